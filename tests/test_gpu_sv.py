"""The iterative statevector path (grover_sv_*, include/grover_sv.h) against
the dense CPU oracle and the closed form (Sec. II, Eqs. 5-6)."""
import numpy as np
import pytest

from oracle import reduced
from oracle import statevector as sv
from paper_2601_03832_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL_AMP_F64 = 1e-12   # complex128 amplitudes, n <= 17, k <= 90
TOL_AMP_C64 = 2e-6    # complex64 amplitudes (FP64 sums and coefficients)
TOL_P_F64 = 1e-10


@pytest.fixture(scope="module")
def B():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2601_03832_gb300 import binding
    binding.load()
    return binding


@pytest.mark.parametrize("dtype", ["c128", "c64"])
@pytest.mark.parametrize("n,M,k", [(1, 1, 3), (3, 2, 5), (10, 3, 20), (17, 8, 90)])
def test_sv_general_phases_against_dense_oracle(B, dtype, n, M, k):
    marked = inputs.marked_strings(n, M, seed=900 + n + M)
    rng = np.random.default_rng(n + 7 * M)
    phis, psis = rng.normal(np.pi, 0.6, k), rng.normal(np.pi, 0.6, k)
    g = B.GroverSV(n, marked, dtype=dtype)
    g.iterate(k, phis, psis)
    ref = sv.grover(n, marked, k, phis, psis)
    v = g.export()
    tol = TOL_AMP_F64 if dtype == "c128" else TOL_AMP_C64
    assert np.abs(v - ref).max() < tol
    assert abs(g.prob_marked() - sv.prob_marked(ref, marked)) < 10 * tol
    x = int(rng.integers(0, 1 << n))
    assert abs(g.amplitude(x) - ref[x]) < tol
    g.close()


def test_sv_chunks_graph_replay_and_reset(B):
    """k split over calls (graph replays of 64 launches plus single launches,
    a new phase array per call) equals one call; reset returns to |s>."""
    n, marked = 14, [5, 9000]
    rng = np.random.default_rng(3)
    k = 150
    phis, psis = rng.normal(np.pi, 0.3, k), rng.normal(np.pi, 0.3, k)
    g1 = B.GroverSV(n, marked)
    g1.iterate(k, phis, psis)
    g2 = B.GroverSV(n, marked)
    for lo, hi in ((0, 70), (70, 71), (71, 150)):
        g2.iterate(hi - lo, phis[lo:hi], psis[lo:hi])
    assert np.abs(g1.export() - g2.export()).max() < 1e-13
    ref = sv.grover(n, marked, k, phis, psis)
    assert np.abs(g1.export() - ref).max() < 1e-11
    g2.reset()
    assert np.abs(g2.export() - sv.uniform_state(n)).max() < 1e-15


@pytest.mark.parametrize("n", [20, 26])
def test_sv_plain_grover_closed_form(B, n):
    M = 1
    marked = inputs.marked_strings(n, M, seed=1000 + n)
    k = inputs.k_floor(n, M)
    g = B.GroverSV(n, marked)
    g.iterate(k)
    P, aw, ar = reduced.closed_form(n, M, k)
    assert abs(g.prob_marked() - P) < TOL_P_F64
    assert abs(g.amplitude(marked[0]) - aw) < 1e-10
    other = (marked[0] + 12345) % (1 << n)
    assert abs(g.amplitude(other) - ar) < 1e-13
    g.close()
