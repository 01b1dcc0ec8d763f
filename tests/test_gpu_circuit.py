"""Gate-level circuits (grover_mps_apply_circuit): the paper's circuit of
Fig. 1A applied gate by gate, in its "Iterative" (one iteration's gates,
repeated) and "Common" (the whole k-iteration circuit) forms, against the
closed form (Sec. II, Eqs. 5-6) and the dense oracle's gate primitives."""
import numpy as np
import pytest

from oracle import reduced
from oracle import statevector as sv
from paper_2601_03832_gb300 import inputs
from tests.gpu_util import dense_from_sites

pytestmark = pytest.mark.gpu

TOL_P = 1e-10
TOL_AMP = 1e-11


@pytest.fixture(scope="module")
def B():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2601_03832_gb300 import binding
    binding.load()
    return binding


def test_grover_gates_iterative_and_common_match_closed_form(B):
    inst = inputs.config_small()
    k = inst.k
    P, aw, ar = reduced.closed_form(inst.n, 1, k)
    one = B.grover_gates(inst.n, inst.marked, 1)
    zeros = bin(((1 << inst.n) - 1) & ~inst.marked[0]).count("1")
    assert len(one) == 4 * inst.n + 1 + 2 * zeros + 1
    it = B.GroverMPS(inst.n, inst.marked, apply="mpo", chi_max=inst.chi_max)
    it.apply_circuit(one, repeat=k)
    allk = B.grover_gates(inst.n, inst.marked, k)
    assert len(allk) == k * len(one)
    cm = B.GroverMPS(inst.n, inst.marked, apply="mpo", chi_max=inst.chi_max)
    cm.apply_circuit(allk, repeat=1)
    for g in (it, cm):
        assert abs(g.prob_marked() - P) < TOL_P
        # the gates give -G per iteration: amplitudes carry (-1)^k
        assert abs(g.amplitude(inst.marked[0]) - (-1) ** k * aw) < TOL_AMP
        assert g.stats()["chi"] == [1] + [2] * (inst.n - 1) + [1]
    v1, v2 = dense_from_sites(it.export()), dense_from_sites(cm.export())
    assert np.abs(v1 - v2).max() < 1e-13


def test_grover_gates_several_marked_against_dense_oracle(B):
    n, M, k = 9, 3, 4
    marked = inputs.marked_strings(n, M, seed=31)
    g = B.GroverMPS(n, marked, apply="mpo", chi_max=8)
    g.apply_circuit(B.grover_gates(n, marked, 1), repeat=k)
    ref = sv.grover(n, marked, k) * (-1) ** k
    assert np.abs(dense_from_sites(g.export()) - ref).max() < TOL_AMP


def test_random_circuit_against_dense_oracle(B):
    """Random one-qubit unitaries and multi-controlled phases, applied gate by
    gate, against the dense oracle's primitives; both storage forms."""
    n = 8
    rng = np.random.default_rng(7)
    ops = []
    for _ in range(40):
        if rng.random() < 0.2:
            ops.append((B.GATE_MCPHASE, 0, float(rng.uniform(-np.pi, np.pi))))
        else:
            a = rng.normal(size=(2, 2)) + 1j * rng.normal(size=(2, 2))
            q, _ = np.linalg.qr(a)
            ops.append((B.GATE_1Q, int(rng.integers(0, n)), q))
    v = sv.uniform_state(n)
    for kind, site, val in ops:
        v = sv.apply_1q(v, n, site, val) if kind == B.GATE_1Q else sv.apply_mcphase(v, val)
    for dtype, tol in (("c128", 1e-11), ("c64", 2e-6)):
        g = B.GroverMPS(n, [1], dtype=dtype, apply="gates", chi_max=16)
        g.apply_circuit(B.make_gates(ops))
        assert np.abs(dense_from_sites(g.export()) - v).max() < tol


def test_circuit_needs_mpo_or_gate_handle(B):
    g = B.GroverMPS(10, [5], apply="fused", chi_max=4)
    with pytest.raises(B.GMPSError) as e:
        g.apply_circuit(B.grover_gates(10, [5], 1))
    assert e.value.status == 9
    h = B.GroverMPS(10, [5], apply="gates", chi_max=8)
    with pytest.raises(B.GMPSError) as e2:
        h.iterate(1)
    assert e2.value.status == 9
