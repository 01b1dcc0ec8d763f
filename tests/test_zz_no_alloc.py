"""grover_mps_run_noalloc: the allocation-free entry point, for callers that
must not allocate device memory (it runs one FP64 instance inside a fixed
device array compiled into the library).  Its results must match the
handle-based entry point -- the same bond table, P_marked and amplitudes
within the FP64 tolerances the other GPU tests use -- on two calls in a row
(the shared array keeps the previous call's contents, so the second call
checks that everything is re-initialised).  This file is collected last so
that a run stopping at the first failure has already run every other test."""
import numpy as np
import pytest

from paper_2601_03832_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL_P = 1e-10     # FP64 marked probability, as in test_gpu_parity.py
TOL_AMP = 1e-11   # FP64 amplitudes
TOL_P_SAME = 1e-12  # same plan and rank rule as the handle path: agreement to rounding


@pytest.fixture(scope="module")
def B():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2601_03832_gb300 import binding
    binding.load()
    return binding


def _reference(B, n, marked, k, apply, chi_max, phi=None, psi=None):
    g = B.GroverMPS(n, marked, dtype="c128", apply=apply, chi_max=chi_max)
    g.iterate(k, phi, psi)
    p = g.prob_marked()
    a = np.array([g.amplitude(w) for w in marked])
    chi = g.stats()["chi"]
    g.close()
    return p, a, chi


@pytest.mark.parametrize("apply", ["mpo", "fused"])
def test_noalloc_matches_handle_path_twice(B, apply):
    inst = inputs.config_small()
    p_ref, a_ref, chi_ref = _reference(B, inst.n, inst.marked, inst.k, apply, inst.chi_max)
    for _ in range(2):
        p, a, chi = B.run_noalloc(inst.n, inst.marked, inst.k, apply=apply, chi_max=inst.chi_max)
        assert chi == chi_ref
        assert abs(p - p_ref) < TOL_P
        assert np.abs(a - a_ref).max() < TOL_AMP


def test_noalloc_long_run_same_bonds_as_handle_path(B):
    """n = 29 (the headline instance) for 1500 iterations: the rank rule is the
    handle path's, so no rounding-noise direction may survive on either side
    and the bond tables agree exactly."""
    inst = inputs.config_n29()
    k = 1500
    p_ref, a_ref, chi_ref = _reference(B, inst.n, inst.marked, k, "fused", inst.chi_max)
    for _ in range(2):
        p, a, chi = B.run_noalloc(inst.n, inst.marked, k, apply="fused", chi_max=inst.chi_max)
        assert chi == chi_ref == [1] + [2] * (inst.n - 1) + [1]
        assert abs(p - p_ref) <= TOL_P_SAME
        assert np.abs(a - a_ref).max() < TOL_AMP


def test_noalloc_general_phases_eight_marked(B):
    import torch
    n, M, k = 18, 8, 40
    marked = inputs.marked_strings(n, M, seed=808)
    rng = np.random.default_rng(8)
    phi, psi = rng.normal(np.pi, 0.5, k), rng.normal(np.pi, 0.5, k)
    p_ref, a_ref, chi_ref = _reference(B, n, marked, k, "fused", 16, phi, psi)
    dphi = torch.tensor(phi, dtype=torch.float64, device="cuda")
    dpsi = torch.tensor(psi, dtype=torch.float64, device="cuda")
    s = torch.cuda.current_stream().cuda_stream
    for _ in range(2):
        p, a, chi = B.run_noalloc(n, marked, k, apply="fused", chi_max=16, dev_phi=dphi.data_ptr(),
                                  dev_psi=dpsi.data_ptr(), stream=s)
        assert chi == chi_ref
        assert abs(p - p_ref) <= TOL_P_SAME
        assert np.abs(a - a_ref).max() < TOL_AMP


def test_noalloc_device_phases_and_back_to_back_instances(B):
    import torch
    n, marked, k = 10, [3, 700, 901], 7
    rng = np.random.default_rng(4)
    phi, psi = rng.normal(np.pi, 0.5, k), rng.normal(np.pi, 0.5, k)
    p_ref, a_ref, chi_ref = _reference(B, n, marked, k, "split", 16, phi, psi)
    dphi = torch.tensor(phi, dtype=torch.float64, device="cuda")
    dpsi = torch.tensor(psi, dtype=torch.float64, device="cuda")
    s = torch.cuda.current_stream().cuda_stream
    for _ in range(2):
        p, a, chi = B.run_noalloc(n, marked, k, apply="split", chi_max=16, dev_phi=dphi.data_ptr(),
                                  dev_psi=dpsi.data_ptr(), stream=s)
        assert chi == chi_ref
        assert abs(p - p_ref) < TOL_P
        assert np.abs(a - a_ref).max() < TOL_AMP
        # a different, larger instance in between must not leak into the next call
        p2, _, chi2 = B.run_noalloc(16, [5], 20, apply="fused", chi_max=4, stream=s)
        p2_ref, _, chi2_ref = _reference(B, 16, [5], 20, "fused", 4)
        assert chi2 == chi2_ref
        assert abs(p2 - p2_ref) < TOL_P


def test_noalloc_accepts_what_the_handle_path_accepts(B):
    """The planner is shared: an MPO-mode instance with M = 7 and
    chi_max = 16 (expanded bond (M+1) x 10 = 80) plans the same bond capacity
    on both paths and gives the same bonds."""
    n, M, k = 12, 7, 3
    marked = inputs.marked_strings(n, M, seed=707)
    p_ref, a_ref, chi_ref = _reference(B, n, marked, k, "mpo", 16)
    p, a, chi = B.run_noalloc(n, marked, k, apply="mpo", chi_max=16)
    assert chi == chi_ref
    assert abs(p - p_ref) < TOL_P


def test_noalloc_rejects_instances_above_the_static_size(B):
    marked = inputs.marked_strings(64, 16, seed=1)
    with pytest.raises(B.GMPSError) as e:
        B.run_noalloc(64, marked, 1, apply="fused", chi_max=32)
    assert e.value.status == 8
    assert "static scratch" in str(e.value)
