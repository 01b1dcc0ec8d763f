"""Thin ctypes binding over libgrover_mps.so (include/grover_mps.h).

Argument marshalling only: every step of the method runs in the CUDA
library.  The functions keep the C names; `GroverMPS` and `GroverBatch` are
small owners of a handle.  If the library is missing or cannot be loaded the
first call raises RuntimeError: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libgrover_mps.so")

GMPS_C128, GMPS_C64_F64SVD, GMPS_DW = 0, 1, 2
GMPS_APPLY_MPO, GMPS_APPLY_SPLIT, GMPS_APPLY_FUSED, GMPS_APPLY_GATES = 0, 1, 2, 3
DTYPES = {"c128": GMPS_C128, "c64": GMPS_C64_F64SVD, "dw": GMPS_DW}
APPLY = {"mpo": GMPS_APPLY_MPO, "split": GMPS_APPLY_SPLIT, "fused": GMPS_APPLY_FUSED, "gates": GMPS_APPLY_GATES}
STATUS = {0: "OK", 1: "ERR_ARG", 2: "ERR_OOM", 3: "ERR_CUDA", 4: "ERR_TIMEOUT", 5: "ERR_NOCONV",
          6: "ERR_NUMERIC", 7: "ERR_STATE", 8: "ERR_CAPACITY", 9: "ERR_UNSUPPORTED"}

# every symbol include/grover_mps.h declares
EXPORTS = [
    "grover_mps_arena_bytes", "grover_mps_create", "grover_mps_create_ex", "grover_mps_reset",
    "grover_mps_iterate", "grover_mps_iterate_device", "grover_mps_sync", "grover_mps_amplitude",
    "grover_mps_prob_marked", "grover_mps_sample", "grover_mps_sample_device", "grover_mps_backward",
    "grover_mps_stats", "grover_mps_export", "grover_mps_destroy", "grover_mps_last_error",
    "grover_mps_batch_create", "grover_mps_batch_run", "grover_mps_batch_result",
    "grover_mps_batch_amplitude", "grover_mps_batch_stats", "grover_mps_batch_set_threads",
    "grover_mps_batch_destroy",
    "grover_mps_launch_count", "grover_mps_run_noalloc", "grover_mps_diff_batch_create",
    "grover_mps_diff_batch_run", "grover_mps_diff_batch_destroy", "grover_mps_apply_circuit",
    "grover_mps_grover_gates", "grover_mps_debug_fail_allocations",
]
# every symbol include/grover_sv.h declares
SV_EXPORTS = [
    "grover_sv_bytes", "grover_sv_create", "grover_sv_reset", "grover_sv_iterate", "grover_sv_amplitude",
    "grover_sv_prob_marked", "grover_sv_export", "grover_sv_destroy",
]


class gmps_config(C.Structure):
    _fields_ = [("n", C.c_int), ("M", C.c_int), ("marked", C.POINTER(C.c_uint64)), ("dtype", C.c_int),
                ("apply", C.c_int), ("chi_max", C.c_int), ("tol", C.c_double), ("max_sweeps", C.c_int),
                ("threads", C.c_int), ("differentiable", C.c_int), ("checkpoint_every", C.c_int),
                ("max_iters", C.c_int), ("arena", C.c_void_p), ("arena_bytes", C.c_size_t)]


class gmps_gate(C.Structure):
    _fields_ = [("kind", C.c_int), ("site", C.c_int), ("u", C.c_double * 8)]


GATE_1Q, GATE_MCPHASE = 0, 1


class gmps_stats(C.Structure):
    _fields_ = [("iterations", C.c_int64), ("n", C.c_int), ("chi", C.c_int * 65), ("max_bond", C.c_int),
                ("log_norm", C.c_double), ("discarded_weight", C.c_double),
                ("max_jacobi_sweeps", C.c_int), ("jacobi_sweeps", C.c_int64), ("svd_count", C.c_int64),
                ("device_status", C.c_int), ("sm_id", C.c_int), ("t_begin_ns", C.c_int64),
                ("t_end_ns", C.c_int64), ("ctas", C.c_int)]


def _stats_dict(s, n):
    return {"iterations": s.iterations, "chi": list(s.chi[: n + 1]), "max_bond": s.max_bond,
            "log_norm": s.log_norm, "discarded_weight": s.discarded_weight,
            "max_jacobi_sweeps": s.max_jacobi_sweeps, "jacobi_sweeps": s.jacobi_sweeps,
            "svd_count": s.svd_count, "device_status": s.device_status, "sm_id": s.sm_id,
            "t_begin_ns": s.t_begin_ns, "t_end_ns": s.t_end_ns, "ctas": s.ctas}


class GMPSError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


_lib = None


def load():
    """Load libgrover_mps.so (built by paper_2601_03832_gb300.build)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"CUDA library not built: {LIB_PATH} missing (run __graft_entry__.build())")
    lib = C.CDLL(LIB_PATH)
    vp, i32, i64, u64, f64 = C.c_void_p, C.c_int, C.c_int64, C.c_uint64, C.c_double
    P = C.POINTER
    sig = {
        "grover_mps_arena_bytes": [P(gmps_config), P(C.c_size_t)],
        "grover_mps_create": [i32, P(u64), i32, i32, i32, f64, vp, P(vp)],
        "grover_mps_create_ex": [P(gmps_config), vp, P(vp)],
        "grover_mps_reset": [vp],
        "grover_mps_iterate": [vp, i64, P(f64), P(f64)],
        "grover_mps_iterate_device": [vp, i64, vp, vp],
        "grover_mps_sync": [vp],
        "grover_mps_amplitude": [vp, u64, P(f64), P(f64)],
        "grover_mps_prob_marked": [vp, P(f64)],
        "grover_mps_sample": [vp, i64, u64, P(u64)],
        "grover_mps_sample_device": [vp, i64, u64, vp, vp],
        "grover_mps_backward": [vp, f64, P(f64), P(f64)],
        "grover_mps_stats": [vp, P(gmps_stats)],
        "grover_mps_export": [vp, P(f64), C.c_size_t, P(C.c_size_t)],
        "grover_mps_destroy": [vp],
        "grover_mps_batch_create": [i32, P(gmps_config), P(i64), P(P(f64)), P(P(f64)), vp, P(vp)],
        "grover_mps_batch_run": [vp, i32],
        "grover_mps_batch_result": [vp, P(f64), P(i32)],
        "grover_mps_batch_amplitude": [vp, i32, u64, P(f64), P(f64)],
        "grover_mps_batch_stats": [vp, i32, P(gmps_stats)],
        "grover_mps_batch_set_threads": [vp, i32],
        "grover_mps_batch_destroy": [vp],
        "grover_mps_run_noalloc": [i32, P(u64), i32, i32, i32, f64, i64, vp, vp, vp, P(f64), P(f64), P(i32)],
        "grover_mps_apply_circuit": [vp, P(gmps_gate), i64, i64],
        "grover_mps_grover_gates": [i32, P(u64), i32, i64, P(gmps_gate), i64, P(i64)],
        "grover_mps_diff_batch_create": [P(gmps_config), i32, i32, vp, P(vp)],
        "grover_mps_diff_batch_run": [vp, P(f64), P(f64), P(f64), P(f64), P(f64)],
        "grover_mps_diff_batch_destroy": [vp],
        "grover_mps_debug_fail_allocations": [i32],
        "grover_sv_bytes": [i32, i32, P(C.c_size_t)],
        "grover_sv_create": [i32, P(u64), i32, i32, vp, P(vp)],
        "grover_sv_reset": [vp],
        "grover_sv_iterate": [vp, i64, P(f64), P(f64)],
        "grover_sv_amplitude": [vp, u64, P(f64), P(f64)],
        "grover_sv_prob_marked": [vp, P(f64)],
        "grover_sv_export": [vp, P(f64), C.c_size_t],
        "grover_sv_destroy": [vp],
    }
    for name, args in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = C.c_int
    lib.grover_mps_last_error.argtypes = []
    lib.grover_mps_last_error.restype = C.c_char_p
    lib.grover_mps_launch_count.argtypes = []
    lib.grover_mps_launch_count.restype = C.c_int64
    _lib = lib
    return lib


def _check(st):
    if st != 0:
        raise GMPSError(st, load().grover_mps_last_error().decode())


def _dptr(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def launch_count() -> int:
    return int(load().grover_mps_launch_count())


def debug_fail_allocations(count: int):
    """Make the library's next `count` device allocations fail (tests)."""
    _check(load().grover_mps_debug_fail_allocations(count))


def make_config(n, marked, dtype="c128", apply="mpo", chi_max=4, tol=0.0, max_sweeps=0, threads=0,
                differentiable=False, checkpoint_every=0, max_iters=0):
    marked_arr = np.ascontiguousarray(np.asarray(marked, dtype=np.uint64))
    cfg = gmps_config()
    cfg.n = n
    cfg.M = len(marked_arr)
    cfg.marked = marked_arr.ctypes.data_as(C.POINTER(C.c_uint64))
    cfg.dtype = DTYPES[dtype] if isinstance(dtype, str) else int(dtype)
    cfg.apply = APPLY[apply] if isinstance(apply, str) else int(apply)
    cfg.chi_max = chi_max
    cfg.tol = tol
    cfg.max_sweeps = max_sweeps
    cfg.threads = threads
    cfg.differentiable = int(differentiable)
    cfg.checkpoint_every = checkpoint_every
    cfg.max_iters = max_iters
    return cfg, marked_arr


def arena_bytes(n, marked, **kw) -> int:
    cfg, keep = make_config(n, marked, **kw)
    out = C.c_size_t()
    _check(load().grover_mps_arena_bytes(C.byref(cfg), C.byref(out)))
    return int(out.value)


class GroverMPS:
    """One instance: grover_mps_create_ex ... grover_mps_destroy."""

    def __init__(self, n, marked, dtype="c128", apply="mpo", chi_max=4, tol=0.0, stream=None,
                 arena=None, **kw):
        lib = load()
        cfg, self._marked = make_config(n, marked, dtype=dtype, apply=apply, chi_max=chi_max, tol=tol, **kw)
        if arena is not None:   # (device pointer, bytes), e.g. from a torch uint8 tensor
            cfg.arena, cfg.arena_bytes = int(arena[0]), int(arena[1])
        self.n, self.marked = n, [int(x) for x in self._marked]
        h = C.c_void_p()
        _check(lib.grover_mps_create_ex(C.byref(cfg), C.c_void_p(stream or 0), C.byref(h)))
        self.h = h

    def iterate(self, k, phi=None, psi=None):
        lib = load()
        pa = None if phi is None else np.ascontiguousarray(phi, dtype=np.float64)
        sa = None if psi is None else np.ascontiguousarray(psi, dtype=np.float64)
        _check(lib.grover_mps_iterate(self.h, int(k), None if pa is None else _dptr(pa),
                                      None if sa is None else _dptr(sa)))

    def iterate_device(self, k, dev_phi=0, dev_psi=0):
        _check(load().grover_mps_iterate_device(self.h, int(k), C.c_void_p(dev_phi or 0),
                                                C.c_void_p(dev_psi or 0)))

    def sync(self):
        _check(load().grover_mps_sync(self.h))

    def reset(self):
        _check(load().grover_mps_reset(self.h))

    def amplitude(self, bits) -> complex:
        re, im = C.c_double(), C.c_double()
        _check(load().grover_mps_amplitude(self.h, C.c_uint64(int(bits)), C.byref(re), C.byref(im)))
        return complex(re.value, im.value)

    def prob_marked(self) -> float:
        p = C.c_double()
        _check(load().grover_mps_prob_marked(self.h, C.byref(p)))
        return p.value

    def sample(self, shots, seed) -> np.ndarray:
        out = np.zeros(int(shots), dtype=np.uint64)
        _check(load().grover_mps_sample(self.h, int(shots), C.c_uint64(int(seed)),
                                        out.ctypes.data_as(C.POINTER(C.c_uint64))))
        return out

    def sample_device(self, shots, seed, dev_bits, dev_margin=0):
        _check(load().grover_mps_sample_device(self.h, int(shots), C.c_uint64(int(seed)),
                                               C.c_void_p(dev_bits), C.c_void_p(dev_margin or 0)))

    def backward(self, dL_dP=-1.0):
        st = self.stats()
        K = int(st["iterations"])
        gphi, gpsi = np.zeros(K), np.zeros(K)
        _check(load().grover_mps_backward(self.h, float(dL_dP), _dptr(gphi), _dptr(gpsi)))
        return gphi, gpsi

    def stats(self) -> dict:
        s = gmps_stats()
        _check(load().grover_mps_stats(self.h, C.byref(s)))
        return _stats_dict(s, self.n)

    def apply_circuit(self, gates, repeat=1):
        """Apply a gate array (from grover_gates or make_gates) `repeat` times."""
        _check(load().grover_mps_apply_circuit(self.h, gates, len(gates), int(repeat)))

    def export(self):
        """Site tensors as a list of complex128 arrays (chi_l, 2, chi_{l+1})."""
        lib = load()
        need = C.c_size_t()
        _check(lib.grover_mps_export(self.h, None, 0, C.byref(need)))
        buf = np.zeros(need.value, dtype=np.float64)
        _check(lib.grover_mps_export(self.h, _dptr(buf), need.value, C.byref(need)))
        chi = self.stats()["chi"]
        z = buf.view(np.complex128)
        out, o = [], 0
        for l in range(self.n):
            cnt = chi[l] * 2 * chi[l + 1]
            out.append(z[o:o + cnt].reshape(chi[l], 2, chi[l + 1]).copy())
            o += cnt
        return out

    def close(self):
        if getattr(self, "h", None):
            load().grover_mps_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def grover_gates(n, marked, iterations=1):
    """The gates of `iterations` Grover iterations (grover_mps_grover_gates)."""
    lib = load()
    m = np.ascontiguousarray(np.asarray(marked, dtype=np.uint64))
    cnt = C.c_int64()
    mp = m.ctypes.data_as(C.POINTER(C.c_uint64))
    _check(lib.grover_mps_grover_gates(int(n), mp, len(m), int(iterations), None, 0, C.byref(cnt)))
    arr = (gmps_gate * cnt.value)()
    _check(lib.grover_mps_grover_gates(int(n), mp, len(m), int(iterations), arr, cnt.value, C.byref(cnt)))
    return arr


def make_gates(ops):
    """Gate array from (kind, site, 2x2 complex matrix or phase) tuples."""
    arr = (gmps_gate * len(ops))()
    for g, (kind, site, val) in zip(arr, ops):
        g.kind, g.site = kind, site
        if kind == GATE_1Q:
            u = np.asarray(val, dtype=np.complex128).reshape(4)
            for q in range(4):
                g.u[2 * q], g.u[2 * q + 1] = u[q].real, u[q].imag
        else:
            g.u[0] = float(val)
    return arr


def run_noalloc(n, marked, k, apply="mpo", chi_max=4, tol=0.0, dev_phi=0, dev_psi=0, stream=None):
    """grover_mps_run_noalloc: one FP64 instance in the library's static device
    array, for callers that cannot allocate device memory.  Returns
    (P_marked, amplitudes of the marked strings, bond table chi_0..chi_n)."""
    lib = load()
    m = np.ascontiguousarray(np.asarray(marked, dtype=np.uint64))
    p = C.c_double()
    amps = np.zeros(2 * len(m))
    chi = np.zeros(int(n) + 1, dtype=np.int32)
    _check(lib.grover_mps_run_noalloc(int(n), m.ctypes.data_as(C.POINTER(C.c_uint64)), len(m),
                                      APPLY[apply] if isinstance(apply, str) else int(apply), int(chi_max),
                                      float(tol), int(k), C.c_void_p(dev_phi or 0), C.c_void_p(dev_psi or 0),
                                      C.c_void_p(stream or 0), C.byref(p), _dptr(amps),
                                      chi.ctypes.data_as(C.POINTER(C.c_int))))
    return p.value, amps[0::2] + 1j * amps[1::2], [int(x) for x in chi]


class DiffBatch:
    """Loss L = 1 - P_marked and its phase gradients for many phase vectors of
    one problem (grover_mps_diff_batch_*): every stage of the forward and
    reverse sweeps is one launch over all vectors."""

    def __init__(self, n, marked, count, K, dtype="c128", apply="fused", chi_max=None, tol=0.0,
                 checkpoint_every=8, threads=0, stream=None):
        lib = load()
        cfg, self._marked = make_config(n, marked, dtype=dtype, apply=apply,
                                        chi_max=chi_max if chi_max else len(marked) + 1, tol=tol,
                                        threads=threads, checkpoint_every=checkpoint_every)
        h = C.c_void_p()
        _check(lib.grover_mps_diff_batch_create(C.byref(cfg), int(count), int(K), C.c_void_p(stream or 0),
                                                C.byref(h)))
        self.h, self.count, self.K = h, int(count), int(K)

    def run(self, phis, psis):
        """phis, psis: (count, K).  Returns (L[count], dL/dphi, dL/dpsi)."""
        ph = np.ascontiguousarray(phis, dtype=np.float64).reshape(self.count, self.K)
        ps = np.ascontiguousarray(psis, dtype=np.float64).reshape(self.count, self.K)
        loss = np.zeros(self.count)
        gphi = np.zeros((self.count, self.K))
        gpsi = np.zeros((self.count, self.K))
        _check(load().grover_mps_diff_batch_run(self.h, _dptr(ph), _dptr(ps), _dptr(loss), _dptr(gphi),
                                                _dptr(gpsi)))
        return loss, gphi, gpsi

    def close(self):
        if getattr(self, "h", None):
            load().grover_mps_diff_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class GroverSV:
    """Iterative Grover on a dense statevector (grover_sv_*): complex128
    ("c128") or complex64 ("c64") amplitudes in device memory."""

    def __init__(self, n, marked, dtype="c128", stream=None):
        lib = load()
        m = np.ascontiguousarray(np.asarray(marked, dtype=np.uint64))
        self.n, self.marked = n, [int(x) for x in m]
        h = C.c_void_p()
        _check(lib.grover_sv_create(int(n), m.ctypes.data_as(C.POINTER(C.c_uint64)), len(m),
                                    DTYPES[dtype] if isinstance(dtype, str) else int(dtype),
                                    C.c_void_p(stream or 0), C.byref(h)))
        self.h = h

    def reset(self):
        _check(load().grover_sv_reset(self.h))

    def iterate(self, k, phi=None, psi=None):
        pa = None if phi is None else np.ascontiguousarray(phi, dtype=np.float64)
        sa = None if psi is None else np.ascontiguousarray(psi, dtype=np.float64)
        _check(load().grover_sv_iterate(self.h, int(k), None if pa is None else _dptr(pa),
                                        None if sa is None else _dptr(sa)))

    def amplitude(self, bits) -> complex:
        re, im = C.c_double(), C.c_double()
        _check(load().grover_sv_amplitude(self.h, C.c_uint64(int(bits)), C.byref(re), C.byref(im)))
        return complex(re.value, im.value)

    def prob_marked(self) -> float:
        p = C.c_double()
        _check(load().grover_sv_prob_marked(self.h, C.byref(p)))
        return p.value

    def export(self) -> np.ndarray:
        buf = np.zeros(2 << self.n, dtype=np.float64)
        _check(load().grover_sv_export(self.h, _dptr(buf), buf.size))
        return buf.view(np.complex128)

    def close(self):
        if getattr(self, "h", None):
            load().grover_sv_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class GroverBatch:
    """Many instances in one persistent launch (grover_mps_batch_*)."""

    def __init__(self, instances, dtype="c64", apply="fused", tol=0.0, phis=None, psis=None, stream=None):
        lib = load()
        cnt = len(instances)
        cfgs = (gmps_config * cnt)()
        self._keep = []
        ks = np.zeros(cnt, dtype=np.int64)
        for i, inst in enumerate(instances):
            c, m = make_config(inst.n, inst.marked, dtype=dtype, apply=apply, chi_max=inst.chi_max,
                               tol=inst.tol if inst.tol else tol)
            cfgs[i] = c
            self._keep.append(m)
            ks[i] = inst.k
        pp = ps = None
        if phis is not None:
            self._phis = [np.ascontiguousarray(p, dtype=np.float64) for p in phis]
            pp = (C.POINTER(C.c_double) * cnt)(*[_dptr(p) for p in self._phis])
        if psis is not None:
            self._psis = [np.ascontiguousarray(p, dtype=np.float64) for p in psis]
            ps = (C.POINTER(C.c_double) * cnt)(*[_dptr(p) for p in self._psis])
        h = C.c_void_p()
        _check(lib.grover_mps_batch_create(cnt, cfgs, ks.ctypes.data_as(C.POINTER(C.c_int64)), pp, ps,
                                           C.c_void_p(stream or 0), C.byref(h)))
        self.h, self.count, self.ks = h, cnt, ks
        self.ns = [inst.n for inst in instances]

    def set_threads(self, threads):
        _check(load().grover_mps_batch_set_threads(self.h, int(threads)))

    def run(self, use_graph=True):
        _check(load().grover_mps_batch_run(self.h, int(bool(use_graph))))

    def result(self):
        p = np.zeros(self.count)
        st = np.zeros(self.count, dtype=np.int32)
        rc = load().grover_mps_batch_result(self.h, _dptr(p), st.ctypes.data_as(C.POINTER(C.c_int)))
        return p, st, rc

    def stats(self, i) -> dict:
        s = gmps_stats()
        _check(load().grover_mps_batch_stats(self.h, int(i), C.byref(s)))
        return _stats_dict(s, self.ns[i])

    def amplitude(self, i, bits) -> complex:
        re, im = C.c_double(), C.c_double()
        _check(load().grover_mps_batch_amplitude(self.h, int(i), C.c_uint64(int(bits)), C.byref(re), C.byref(im)))
        return complex(re.value, im.value)

    def close(self):
        if getattr(self, "h", None):
            load().grover_mps_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
