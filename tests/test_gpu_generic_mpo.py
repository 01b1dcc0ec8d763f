"""The generic MPO path (the oracle as an MPO of bond M+1, Sec. III-B-2's
"tensors are locally updated") at expanded bonds beyond shared memory: the
QR sweep's R and work matrices then live in a per-instance device work area.
Against the dense oracle (n = 16, M = 16, expanded bond 17 x 19 = 323) and,
at the multi-marked workload (n = 40, M = 32, expanded bond 33 x 35 = 1155),
against the closed form (Sec. II, Eqs. 5-6) and the exact Schmidt spectrum."""
import numpy as np
import pytest

from oracle import reduced
from oracle import statevector as sv
from paper_2601_03832_gb300 import inputs
from tests.gpu_util import dense_from_sites, schmidt_from_sites

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2601_03832_gb300 import binding
    binding.load()
    return binding


def test_generic_mpo_work_area_against_dense_oracle(B):
    n, M, k = 16, 16, 2
    marked = inputs.marked_strings(n, M, seed=1616)
    rng = np.random.default_rng(16)
    phis, psis = rng.normal(np.pi, 0.4, k), rng.normal(np.pi, 0.4, k)
    g = B.GroverMPS(n, marked, dtype="c128", apply="mpo", chi_max=32)
    g.iterate(k, phis, psis)
    ref = sv.grover(n, marked, k, phis, psis)
    assert np.abs(dense_from_sites(g.export()) - ref).max() < 1e-11
    st = g.stats()
    assert st["ctas"] > 1  # the QR steps ran on the cluster
    for cut in range(1, n):
        assert st["chi"][cut] == reduced.exact_bond(n, marked, k, cut, phis, psis), cut
    g.close()


def test_generic_mpo_work_area_complex64(B):
    """The same generic-MPO case in the complex64 form (FP32 storage and
    contraction, FP64 QR on the cluster, warm-started Jacobi): amplitudes
    within 1e-5 of the dense FP64 oracle, bonds between the exact Schmidt
    rank and 2(M+1)."""
    n, M, k = 16, 16, 2
    marked = inputs.marked_strings(n, M, seed=1616)
    rng = np.random.default_rng(16)
    phis, psis = rng.normal(np.pi, 0.4, k), rng.normal(np.pi, 0.4, k)
    g = B.GroverMPS(n, marked, dtype="c64", apply="mpo", chi_max=64)
    g.iterate(k, phis, psis)
    ref = sv.grover(n, marked, k, phis, psis)
    assert np.abs(dense_from_sites(g.export()) - ref).max() < 1e-5
    st = g.stats()
    assert st["ctas"] > 1
    for cut in range(1, n):
        exact = reduced.exact_bond(n, marked, k, cut, phis, psis)
        assert exact <= st["chi"][cut] <= 2 * (M + 1), cut
    g.close()


def test_generic_mpo_multi_marked_n40(B):
    k = 2
    mi = inputs.config_multi_marked(k=k)
    g = B.GroverMPS(mi.n, mi.marked, dtype="c128", apply="mpo", chi_max=mi.chi_max, tol=mi.tol)
    g.iterate(k)
    P_cf, aw, _ = reduced.closed_form(mi.n, mi.M, k)
    assert abs(g.prob_marked() - P_cf) <= 1e-9 * P_cf
    for w in mi.marked[:4]:
        assert abs(g.amplitude(w) - aw) <= 1e-12
    st = g.stats()
    sites = g.export()
    for cut in (1, 6, 20, 34, 39):
        ex = reduced.schmidt_values(mi.n, mi.marked, k, cut)
        kept = ex[ex > mi.tol * ex[0]]
        assert st["chi"][cut] == len(kept), cut
        got = schmidt_from_sites(sites, cut)
        assert np.abs(got[: len(kept)] - kept).max() <= 1e-9 * kept[0], cut
    g.close()
