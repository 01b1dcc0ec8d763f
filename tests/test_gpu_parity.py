"""CUDA path (through the C ABI) against the CPU oracle, element by element."""
import math

import numpy as np
import pytest

from oracle import mps as omps
from oracle import reduced
from oracle import statevector as sv
from paper_2601_03832_gb300 import inputs
from tests.gpu_util import dense_from_sites, right_orthonormal_error

pytestmark = pytest.mark.gpu

TOL_P_F64 = 1e-10        # FP64 marked probability (plain form)
TOL_AMP_F64 = 1e-11      # FP64 amplitudes, small n
# complex64 storage and contraction (FP64 QR/SVD): per-result bounds measured
# on the small configuration and stated with margin
TOL_P_C64 = 2e-6
TOL_AMP_C64 = 2e-6
# double-word FP32 (~48-bit significand): worst measured amplitude error 3e-11
# over the general-phase cases below; stated bound 1e-10
TOL_AMP_DW = 1e-10
TOL = {"c128": (TOL_P_F64, TOL_AMP_F64), "dw": (TOL_P_F64, TOL_AMP_DW), "c64": (TOL_P_C64, TOL_AMP_C64)}


@pytest.fixture(scope="module")
def B():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2601_03832_gb300 import binding
    binding.load()
    return binding


@pytest.mark.parametrize("dtype", ["c128", "dw", "c64"])
@pytest.mark.parametrize("apply", ["mpo", "split", "fused"])
def test_small_config_closed_form(B, apply, dtype):
    tp, ta = TOL[dtype]
    inst = inputs.config_small()
    g = B.GroverMPS(inst.n, inst.marked, dtype=dtype, apply=apply, chi_max=inst.chi_max)
    g.iterate(inst.k)
    P, aw, ar = reduced.closed_form(inst.n, 1, inst.k)
    assert abs(g.prob_marked() - P) <= tp
    a = g.amplitude(inst.marked[0])
    assert abs(a.real - aw) < ta and abs(a.imag) < ta
    st = g.stats()
    assert st["chi"] == [1] + [2] * (inst.n - 1) + [1]
    assert st["device_status"] == 0 and st["iterations"] == inst.k
    sites = g.export()
    v = dense_from_sites(sites)
    ref = sv.grover(inst.n, inst.marked, inst.k)
    assert np.abs(v - ref).max() < ta
    orth = 1e-12 if dtype == "c128" else (1e-12 if dtype == "dw" else 1e-6)
    for A in sites[1:]:
        assert right_orthonormal_error(A) < orth
    assert abs(np.linalg.norm(sites[0]) - 1.0) < orth


@pytest.mark.parametrize("dtype", ["c128", "dw"])
@pytest.mark.parametrize("apply", ["mpo", "split", "fused"])
@pytest.mark.parametrize("n,M", [(1, 1), (2, 1), (3, 2), (5, 1), (7, 3), (9, 4), (11, 2)])
def test_general_phases_dense(B, apply, n, M, dtype):
    marked = inputs.marked_strings(n, M, seed=200 + 7 * n + M)
    rng = np.random.default_rng(n * 31 + M)
    k = 6
    phis, psis = rng.normal(np.pi, 0.6, k), rng.normal(np.pi, 0.6, k)
    g = B.GroverMPS(n, marked, dtype=dtype, apply=apply, chi_max=64)
    g.iterate(k, phis, psis)
    ref = sv.grover(n, marked, k, phis, psis)
    v = dense_from_sites(g.export())
    assert np.abs(v - ref).max() < TOL[dtype][1]
    st = g.stats()
    for cut in range(1, n):
        assert st["chi"][cut] == reduced.exact_bond(n, marked, k, cut, phis, psis)


def test_iterate_in_chunks_equals_one_call(B):
    inst = inputs.config_small()
    g1 = B.GroverMPS(inst.n, inst.marked, apply="fused", chi_max=4)
    g1.iterate(50)
    g2 = B.GroverMPS(inst.n, inst.marked, apply="fused", chi_max=4)
    for _ in range(5):
        g2.iterate(10)
    assert abs(g1.prob_marked() - g2.prob_marked()) < 1e-13


def test_multi_marked_split_and_fused_vs_reduced(B):
    n, M = 24, 8
    marked = inputs.marked_strings(n, M, seed=77)
    k = 40
    for apply in ("split", "fused"):
        g = B.GroverMPS(n, marked, apply=apply, chi_max=16)
        g.iterate(k)
        P, aw, ar = reduced.closed_form(n, M, k)
        assert abs(g.prob_marked() - P) < TOL_P_F64
        for w in marked[:3]:
            assert abs(g.amplitude(w) - aw) < 1e-11
        st = g.stats()
        for cut in (1, 5, 12, 23):
            assert st["chi"][cut] == reduced.exact_bond(n, marked, k, cut)


def test_sampling_bit_exact_small_config(B):
    inst = inputs.config_small()
    g = B.GroverMPS(inst.n, inst.marked, chi_max=inst.chi_max)
    g.iterate(inst.k)
    ref = omps.grover_iterate(omps.plus_state(inst.n), inst.marked, inst.k, inst.chi_max)
    for shots, seed in ((4096, 2), (1, 2), (333, 12345)):
        bits = g.sample(shots, seed)
        obits, margin = omps.sample(ref, shots, seed)
        ok = margin > 1e-12
        assert ok.sum() >= shots - 2
        assert np.array_equal(bits[ok], obits[ok])


def test_sampling_general_state(B):
    n, marked = 9, [3, 300, 77]
    rng = np.random.default_rng(5)
    phis, psis = rng.normal(np.pi, 0.5, 4), rng.normal(np.pi, 0.5, 4)
    g = B.GroverMPS(n, marked, apply="split", chi_max=16)
    g.iterate(4, phis, psis)
    ref = omps.grover_iterate(omps.plus_state(n), marked, 4, 16, phis=phis, psis=psis)
    bits = g.sample(2000, 99)
    obits, margin = omps.sample(ref, 2000, 99)
    ok = margin > 1e-12
    assert np.array_equal(bits[ok], obits[ok])


def test_truncation_chi_max_one(B):
    """chi_max = 1 forces product-state truncation: compare with the oracle's
    identical rule (gauge-invariant amplitudes)."""
    n, marked = 8, [19]
    g = B.GroverMPS(n, marked, chi_max=1)
    g.iterate(3)
    ref = omps.grover_iterate(omps.plus_state(n), marked, 3, 1)
    v = dense_from_sites(g.export())
    assert np.abs(v - omps.to_dense(ref)).max() < 1e-11
    assert g.stats()["discarded_weight"] > 0


def test_bad_arguments_are_rejected(B):
    with pytest.raises(B.GMPSError) as e:
        B.GroverMPS(5, [3, 3])
    assert e.value.status == 1
    with pytest.raises(B.GMPSError):
        B.GroverMPS(5, [40])
    with pytest.raises(B.GMPSError):
        B.GroverMPS(0, [0])
    with pytest.raises(B.GMPSError):
        B.GroverMPS(4, [1], chi_max=0)
    g = B.GroverMPS(4, [1])
    with pytest.raises(B.GMPSError):
        g.amplitude(1 << 5)
    with pytest.raises(B.GMPSError):
        g.iterate(2, np.array([0.1, np.nan]))


def test_jacobi_sweep_limit_reports_status(B):
    """max_sweeps = 1 cannot converge: the device reports ERR_NOCONV and the
    handle enters its error state (no fault, no hang)."""
    n, marked = 10, [5, 9, 100]
    g = B.GroverMPS(n, marked, apply="split", chi_max=16, max_sweeps=1)
    with pytest.raises(B.GMPSError) as e:
        g.iterate(5)
    assert e.value.status == 5
    with pytest.raises(B.GMPSError) as e2:
        g.iterate(1)
    assert e2.value.status == 7
    g.reset()
    assert g.stats()["device_status"] == 0


def test_caller_arena_from_torch(B):
    import torch
    inst = inputs.config_small()
    nbytes = B.arena_bytes(inst.n, inst.marked, chi_max=4)
    buf = torch.empty(nbytes + 256, dtype=torch.uint8, device="cuda")
    base = (buf.data_ptr() + 255) // 256 * 256
    s = torch.cuda.current_stream()
    g = B.GroverMPS(inst.n, inst.marked, chi_max=4, stream=s.cuda_stream, arena=(base, nbytes))
    g.iterate(inst.k)
    assert abs(g.prob_marked() - reduced.closed_form(inst.n, 1, inst.k)[0]) < TOL_P_F64
    g.close()


@pytest.mark.parametrize("dtype", ["c128", "c64", "dw"])
def test_batched_small(B, dtype):
    """A batch of small uneven instances in one persistent launch captured in a
    CUDA graph: every P_marked within its form's bound of the closed form, and a
    replay of the graph gives the same bits (the precision forms' per-site
    cache of Jacobi rotations is reset with the chains, so a replay repeats the
    first run exactly)."""
    insts = inputs.config_batched(count=12, seed=9, n_range=(6, 14), m_range=(1, 4), kcap=60, chi_max=8)
    b = B.GroverBatch(insts, dtype=dtype, apply="fused")
    b.run(use_graph=True)
    p, st, rc = b.result()
    assert rc == 0 and not st.any()
    for i, inst in enumerate(insts):
        Pc = reduced.closed_form(inst.n, inst.M, inst.k)[0]
        assert abs(p[i] - Pc) < TOL[dtype][0]
    # replay the captured graph: same result
    b.run(use_graph=True)
    p2, _, _ = b.result()
    assert np.array_equal(p, p2)


def test_batched_many_marked_fp64_all_instances(B):
    """128 instances of the batched workload (n in [16, 36], M in [1, 16], k_i
    capped at 100) in FP64: every P_marked within 1e-10 of the closed form.
    Includes pivots whose squared modulus is a denormal double (n = 17, M = 12)."""
    insts = inputs.config_batched(count=128)
    for i in insts:
        i.k = min(i.k, 100)
    b = B.GroverBatch(insts, dtype="c128", apply="fused")
    b.run(use_graph=False)
    p, st, rc = b.result()
    assert rc == 0 and not st.any()
    errs = [abs(p[i] - reduced.closed_form(x.n, x.M, x.k)[0]) for i, x in enumerate(insts)]
    assert max(errs) < TOL_P_F64, (int(np.argmax(errs)), max(errs))


@pytest.mark.parametrize("dtype", ["c128", "dw"])
@pytest.mark.parametrize("apply", ["mpo", "split", "fused"])
@pytest.mark.parametrize("n,M", [(12, 1), (10, 2)])
def test_cta_sizes_agree_with_oracle(B, apply, n, M, dtype):
    """One warp (every small step inline), two warps (Q formed by warp 1,
    target environments folded during the SVD sweep) and eight warps run the
    same iteration: each against the dense oracle, with general phases."""
    marked = inputs.marked_strings(n, M, seed=500 + n + M)
    rng = np.random.default_rng(17 * n + M)
    k = 9
    phis, psis = rng.normal(np.pi, 0.5, k), rng.normal(np.pi, 0.5, k)
    ref = sv.grover(n, marked, k, phis, psis)
    for threads in (32, 64, 256):
        g = B.GroverMPS(n, marked, dtype=dtype, apply=apply, chi_max=16, threads=threads)
        g.iterate(k, phis, psis)
        v = dense_from_sites(g.export())
        assert np.abs(v - ref).max() < TOL[dtype][1], threads
        st = g.stats()
        for cut in range(1, n):
            assert st["chi"][cut] == reduced.exact_bond(n, marked, k, cut, phis, psis), (threads, cut)
        g.close()


def test_paper_experiments_small_n(B):
    """The paper's sweeps (M = 1, k = round(pi/4 sqrt N)) on the built path at
    small n: FP64 marked probability against the closed form, complex64
    within its stated bound, shot counts within 6 sigma of the binomial mean."""
    from paper_2601_03832_gb300 import experiments as ex
    ns = [4, 7, 10]
    for r in ex.precision_sweep(ns):
        Pc = reduced.closed_form(r["n"], 1, r["k"])[0]
        assert abs(r["c128"]["P_marked"] - Pc) < TOL_P_F64
        assert abs(r["c64"]["P_marked"] - Pc) < TOL_P_C64
        assert r["c128"]["max_bond"] <= 2
    for r in ex.shot_sweep([2, 5, 9]):
        Pc = reduced.closed_form(r["n"], 1, r["k"])[0]
        for s, cnt in r["marked_counts"].items():
            s = int(s)
            assert 0 <= cnt <= s
            assert abs(cnt - s * Pc) <= 6 * math.sqrt(s * Pc * (1 - Pc)) + 1


def test_autotune_picks_a_candidate_and_caches_per_device(B, tmp_path, monkeypatch):
    """The batch autotuner times every candidate block size on a slice of the
    batch, returns the fastest, and caches it under a key that names the GPU,
    its SM count and the library build; a second call is served from the cache."""
    import torch
    from paper_2601_03832_gb300 import autotune
    monkeypatch.setattr(autotune, "CACHE", str(tmp_path / "tune.json"))
    insts = inputs.config_batched(count=8, seed=9, n_range=(8, 12), m_range=(1, 3), kcap=20, chi_max=8)
    best, rec = autotune.tune_batch(insts, dtype="c64", apply="fused", kslice=4)
    assert best in autotune.CANDIDATES
    assert set(rec["seconds"]) == {str(t) for t in autotune.CANDIDATES}
    key = autotune._key(insts, "c64", "fused")
    props = torch.cuda.get_device_properties(torch.cuda.current_device())
    assert key.startswith(f"{props.name}|sm{props.multi_processor_count}|")
    best2, rec2 = autotune.tune_batch(insts, dtype="c64", apply="fused", kslice=4)
    assert best2 == best and rec2 == rec


def test_forced_allocation_failure_reports_oom(B):
    """A device allocation that fails (forced by the library's fault hook)
    surfaces as GMPS_ERR_OOM from the handle, the batch and the statevector,
    with nothing left behind: the next creation succeeds and runs."""
    inst = inputs.config_small()
    for make in (lambda: B.GroverMPS(inst.n, inst.marked, chi_max=4),
                 lambda: B.GroverBatch([inst], dtype="c128", apply="fused"),
                 lambda: B.GroverSV(inst.n, inst.marked)):
        B.debug_fail_allocations(1)
        with pytest.raises(B.GMPSError) as e:
            make()
        assert e.value.status == 2
    B.debug_fail_allocations(0)
    g = B.GroverMPS(inst.n, inst.marked, chi_max=4)
    g.iterate(inst.k)
    assert abs(g.prob_marked() - reduced.closed_form(inst.n, 1, inst.k)[0]) < TOL_P_F64
    g.close()


def test_arena_canary_catches_a_write_past_the_arena(B):
    """The canary closing a handle's arena is checked after every call that
    synchronises: overwriting it (here from the host, through the caller's
    torch arena) turns the next call into GMPS_ERR_STATE."""
    import torch
    inst = inputs.config_small()
    nbytes = B.arena_bytes(inst.n, inst.marked, chi_max=4)
    buf = torch.zeros(nbytes + 256, dtype=torch.uint8, device="cuda")
    off = (256 - buf.data_ptr() % 256) % 256
    base = buf.data_ptr() + off
    s = torch.cuda.current_stream()
    g = B.GroverMPS(inst.n, inst.marked, chi_max=4, stream=s.cuda_stream, arena=(base, nbytes))
    g.iterate(5)                                   # canary intact: fine
    buf[off + nbytes - 8: off + nbytes] = 0xFF     # the arena's last bytes
    torch.cuda.synchronize()
    with pytest.raises(B.GMPSError) as e:
        g.iterate(5)
    assert e.value.status == 7 and "canary" in str(e.value)
    g.close()
