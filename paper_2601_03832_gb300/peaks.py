"""Measured peak rates of this GPU: the roofline denominators.

`measure()` times the microbenchmarks of libgmps_peaks.so (FP64 FMA, FP32
FMA, shared-memory reads; include/gmps_peaks.h) with CUDA events on the
current stream, and the TF32 tensor rate with a cuBLAS GEMM through
torch.matmul (8192^3, TF32 allowed).  Each figure is the best of a few
repetitions after a warm-up launch.
"""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libgmps_peaks.so")
FP64_FMA, FP32_FMA, SMEM_READ = 0, 1, 2

_lib = None


def load():
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"peak library not built: {LIB_PATH} missing (run __graft_entry__.build())")
    lib = C.CDLL(LIB_PATH)
    lib.gmps_peak_launch.argtypes = [C.c_int, C.c_int, C.c_int, C.c_longlong, C.c_void_p, C.c_void_p,
                                     C.POINTER(C.c_double)]
    lib.gmps_peak_launch.restype = C.c_int
    _lib = lib
    return lib


def _time_launch(kind, blocks, threads, trips, reps=3):
    import torch
    lib = load()
    stream = torch.cuda.current_stream()
    sink = torch.empty(blocks * threads, dtype=torch.float64, device="cuda")
    work = C.c_double()
    best = None
    for r in range(reps + 1):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record(stream)
        rc = lib.gmps_peak_launch(kind, blocks, threads, trips, C.c_void_p(stream.cuda_stream),
                                  C.c_void_p(sink.data_ptr()), C.byref(work))
        b.record(stream)
        torch.cuda.synchronize()
        if rc != 0:
            raise RuntimeError(f"gmps_peak_launch({kind}) failed with {rc}")
        if r == 0:
            continue  # warm-up
        sec = a.elapsed_time(b) / 1000.0
        best = sec if best is None else min(best, sec)
    return work.value / best, best


def measure():
    """Dict of measured peaks: fp64/fp32 FMA TFLOP/s, shared-memory read
    TB/s (whole chip), TF32 tensor TFLOP/s (cuBLAS), with the launch shapes."""
    import torch
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    out = {"sms": sms}
    fp64, t64 = _time_launch(FP64_FMA, sms * 8, 256, 2000)
    fp32, t32 = _time_launch(FP32_FMA, sms * 8, 256, 40000)
    smem, ts = _time_launch(SMEM_READ, sms * 8, 256, 20000)
    out["fp64_fma_tflops"] = fp64 / 1e12
    out["fp32_fma_tflops"] = fp32 / 1e12
    out["smem_read_tbs"] = smem / 1e12
    out["launch"] = {"blocks": sms * 8, "threads": 256, "seconds": {"fp64": t64, "fp32": t32, "smem": ts}}
    # TF32 tensor rate through cuBLAS (a library GEMM: the denominator for a
    # 3xTF32 contraction)
    prev = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = True
    try:
        n = 8192
        x = torch.randn(n, n, device="cuda", dtype=torch.float32)
        y = torch.randn(n, n, device="cuda", dtype=torch.float32)
        torch.matmul(x, y)
        best = None
        for _ in range(5):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            torch.matmul(x, y)
            b.record()
            torch.cuda.synchronize()
            s = a.elapsed_time(b) / 1000.0
            best = s if best is None else min(best, s)
        out["tf32_tensor_tflops"] = 2.0 * n ** 3 / best / 1e12
        del x, y
    finally:
        torch.backends.cuda.matmul.allow_tf32 = prev
    return out


if __name__ == "__main__":
    import json

    import torch
    torch.cuda.set_device(0)
    print(json.dumps(measure(), indent=1))
