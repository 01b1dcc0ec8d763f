"""Pins of the CPU oracle against things other than itself: the paper's
closed form (Sec. II, Eqs. 5-6), brute-force dense operators, library
routines (numpy.random.Philox, numpy.linalg.svd) and finite differences."""
import math

import numpy as np
import pytest

from oracle import mps, philox, reduced, statevector as sv
from paper_2601_03832_gb300 import inputs


# ------------------------------------------------------------------ Philox
@pytest.mark.parametrize("key", [0, 1, 0xDEADBEEFCAFEF00D, 2**64 - 1])
def test_philox_matches_numpy(key):
    """numpy.random.Philox is Philox4x64-10; it increments its 256-bit counter
    before each block, so counter c-1 yields the block of counter c."""
    rng = np.random.Generator(np.random.PCG64(123))
    for _ in range(20):
        ctr = [int(x) for x in rng.integers(0, 2**63, size=4, dtype=np.uint64)]
        ctr[0] = max(ctr[0], 1)
        c_int = sum(c << (64 * i) for i, c in enumerate(ctr)) - 1
        ref = np.random.Philox(key=key, counter=c_int).random_raw(4)
        got = philox.philox4x64_10([np.uint64(c) for c in ctr], [np.uint64(key), np.uint64(0)])
        assert [int(x) for x in got] == [int(x) for x in ref]


def test_philox_zero_block():
    """Counter 0, key 0 through numpy (counter -1 wraps to 0)."""
    ref = np.random.Philox(key=0, counter=2**256 - 1).random_raw(4)
    got = philox.philox4x64_10([np.uint64(0)] * 4, [np.uint64(0)] * 2)
    assert [int(x) for x in got] == [int(x) for x in ref]


def test_uniforms_range():
    u = philox.uniforms(7, np.arange(10000, dtype=np.uint64), 3)
    assert u.min() >= 0.0 and u.max() < 1.0
    assert abs(u.mean() - 0.5) < 0.02


# -------------------------------------------------------- closed form pins
@pytest.mark.parametrize("n,M", [(2, 1), (5, 1), (8, 3), (10, 1), (12, 1), (12, 7)])
def test_statevector_closed_form(n, M):
    """Dense statevector at phi = psi = pi against Eqs. 5-6."""
    marked = inputs.marked_strings(n, M, seed=11 + n)
    for k in [0, 1, 3, inputs.k_floor(n, M)]:
        v = sv.grover(n, marked, k)
        P, aw, ar = reduced.closed_form(n, M, k)
        assert abs(sv.prob_marked(v, marked) - P) < 1e-12
        mask = np.zeros(1 << n, bool)
        mask[marked] = True
        assert np.allclose(v[mask], aw, atol=1e-12)
        assert np.allclose(v[~mask], ar, atol=1e-12)
        assert abs(np.linalg.norm(v) - 1) < 1e-12


def test_closed_form_values_small_config():
    """n = 12, M = 1, k = 50: theta = arcsin(2^-6), P = sin^2(101 theta)."""
    th = math.asin(2.0 ** -6)
    assert abs(reduced.theta(12, 1) - th) < 1e-16
    P, aw, ar = reduced.closed_form(12, 1, 50)
    assert abs(P - math.sin(101 * th) ** 2) < 1e-15
    assert abs(P - 0.99994534610911) < 1e-13


def test_paper_fp64_amplitude_is_one():
    """Sec. IV-2/IV-3 (Figs. 3-4): with M = 1 and k = round(pi/4 sqrt N) (Eq. 8)
    the FP64 target value reads 1.0 from n = 13 up to n = 29; the closed form
    gives P > 0.9997 there (1.000 to three decimals)."""
    for n in range(13, 30):
        k = int(round(math.pi / 4 * math.sqrt(2.0 ** n)))
        P = reduced.closed_form(n, 1, k)[0]
        assert P > 0.9997


def test_reduced_model_matches_closed_form_large_n():
    for n, M, k in [(29, 1, 18198), (40, 32, 1000), (20, 4, 64), (60, 5, 1000)]:
        P, aw, ar = reduced.amplitudes(n, M, k)
        Pc, awc, arc = reduced.closed_form(n, M, k)
        assert abs(P - Pc) < 1e-10
        assert abs(aw - awc) < 1e-10 and abs(ar - arc) < 1e-12


# ----------------------------------------------- brute-force dense operators
@pytest.mark.parametrize("n,M", [(1, 1), (3, 2), (4, 1), (5, 3)])
def test_statevector_update_matches_dense_operators(n, M):
    marked = inputs.marked_strings(n, M, seed=3 * n + M)
    rng = np.random.default_rng(n)
    phis, psis = rng.uniform(0, 2 * np.pi, 4), rng.uniform(0, 2 * np.pi, 4)
    v = sv.uniform_state(n)
    ref = v.copy()
    for j in range(4):
        O, D = sv.dense_operators(n, marked, np.exp(1j * phis[j]), np.exp(1j * psis[j]))
        ref = D @ (O @ ref)
    got = sv.grover(n, marked, 4, phis, psis)
    assert np.allclose(got, ref, atol=1e-13)
    # the dense operators are unitary
    assert np.allclose(O.conj().T @ O, np.eye(1 << n), atol=1e-13)
    assert np.allclose(D.conj().T @ D, np.eye(1 << n), atol=1e-13)


@pytest.mark.parametrize("n,M", [(3, 1), (4, 2), (10, 5), (12, 1)])
def test_reduced_model_matches_statevector_general_phases(n, M):
    marked = inputs.marked_strings(n, M, seed=17 + n)
    rng = np.random.default_rng(M)
    k = 9
    phis, psis = rng.normal(np.pi, 0.7, k), rng.normal(np.pi, 0.7, k)
    v = sv.grover(n, marked, k, phis, psis)
    P, aw, ar = reduced.amplitudes(n, M, k, phis, psis)
    mask = np.zeros(1 << n, bool)
    mask[marked] = True
    assert np.allclose(v[mask], aw, atol=1e-12)
    assert np.allclose(v[~mask], ar, atol=1e-12)
    assert abs(sv.prob_marked(v, marked) - P) < 1e-12


# ---------------------------------------------------- Schmidt spectrum pin
@pytest.mark.parametrize("n,M,k", [(6, 1, 3), (8, 3, 5), (10, 4, 2), (12, 1, 50), (9, 8, 1)])
def test_schmidt_spectrum_matches_dense_svd(n, M, k):
    marked = inputs.marked_strings(n, M, seed=5 + n + M)
    rng = np.random.default_rng(n)
    phis, psis = rng.normal(np.pi, 0.3, k), rng.normal(np.pi, 0.3, k)
    v = sv.grover(n, marked, k, phis, psis)
    for cut in range(1, n):
        # x = low (sites < cut) + high * 2^cut: rows = high bits, cols = low bits
        mat = v.reshape(1 << (n - cut), 1 << cut)
        ref = np.linalg.svd(mat, compute_uv=False)
        got = reduced.schmidt_values(n, marked, k, cut, phis, psis)
        r = len(got)
        assert np.allclose(got, ref[:r], atol=1e-12)
        assert np.all(ref[r:] < 1e-12)


def test_exact_bond_two_for_single_marked():
    inst = inputs.config_small()
    for cut in range(1, 12):
        assert reduced.exact_bond(12, inst.marked, 50, cut) == 2
        assert reduced.exact_bond(12, inst.marked, 0, cut) == 1


# ------------------------------------------------------------ MPS oracle
@pytest.mark.parametrize("n", [1, 2, 3, 5])
def test_mpo_builders_match_dense_operators(n):
    marked = inputs.marked_strings(n, min(3, (1 << n) - 1), seed=n)
    phi, psi = 0.37, 2.9
    O, D = sv.dense_operators(n, marked, np.exp(1j * phi), np.exp(1j * psi))
    assert np.allclose(mps.mpo_to_dense(mps.oracle_mpo(n, marked, phi)), O, atol=1e-14)
    assert np.allclose(mps.mpo_to_dense(mps.diffusion_mpo(n, psi)), D, atol=1e-14)


@pytest.mark.parametrize("mode", ["mpo", "split", "fused"])
@pytest.mark.parametrize("n,M", [(1, 1), (2, 1), (4, 2), (7, 3), (10, 1), (11, 6)])
def test_mps_matches_statevector(mode, n, M):
    marked = inputs.marked_strings(n, M, seed=100 + n * M)
    rng = np.random.default_rng(n + M)
    k = 7
    phis, psis = rng.normal(np.pi, 0.5, k), rng.normal(np.pi, 0.5, k)
    st = mps.grover_iterate(mps.plus_state(n), marked, k, chi_max=64, tol=0.0,
                            phis=phis, psis=psis, mode=mode)
    v = sv.grover(n, marked, k, phis, psis)
    assert np.allclose(mps.to_dense(st), v, atol=1e-12)
    for w in marked:
        assert abs(mps.amplitude(st, w) - v[w]) < 1e-12
    assert abs(mps.overlap_plus(st) - v.sum() / math.sqrt(1 << n)) < 1e-12
    # canonical form left by the SVD sweep: right-orthonormal sites, unit norm
    for A in st.sites[1:]:
        assert mps.is_right_orthonormal(A)
    assert abs(np.linalg.norm(st.sites[0]) - 1) < 1e-13
    # exact bonds
    for cut in range(1, n):
        assert st.bonds()[cut] == reduced.exact_bond(n, marked, k, cut, phis, psis)


def test_qr_sweep_left_orthonormal_and_exact():
    n, marked = 8, [5, 200]
    st = mps.grover_iterate(mps.plus_state(n), marked, 3, 16)
    ex = mps.apply_mpo(st, mps.oracle_mpo(n, marked, 1.1))
    q = mps.qr_sweep(ex)
    for A in q.sites[:-1]:
        assert mps.is_left_orthonormal(A)
    assert np.allclose(mps.to_dense(q), mps.to_dense(ex), atol=1e-13)


def test_truncation_rule():
    S = np.array([1.0, 0.5, 1e-13, 1e-17])
    assert mps.keep_count(S, 4, 8, chi_max=8, tol=0.0) == 3
    assert mps.keep_count(S, 4, 8, chi_max=8, tol=1e-12) == 2
    assert mps.keep_count(S, 4, 8, chi_max=1, tol=0.0) == 1
    assert mps.keep_count(np.zeros(3), 3, 3, 4, 0.0) == 1


def test_mps_small_config_closed_form_and_bond_two():
    inst = inputs.config_small()
    st = mps.grover_iterate(mps.plus_state(12), inst.marked, 50, inst.chi_max, 0.0)
    P, aw, ar = reduced.closed_form(12, 1, 50)
    assert abs(mps.prob_marked(st, inst.marked) - P) < 1e-12
    assert abs(mps.amplitude(st, inst.marked[0]) - aw) < 1e-12
    assert st.bonds() == [1] + [2] * 11 + [1]
    other = (inst.marked[0] + 1) % 4096
    assert abs(mps.amplitude(st, other) - ar) < 1e-13


def test_mps_multi_marked_direct_sum_matches_reduced_large_n():
    """n = 40, M = 32 (a few iterations): P against the closed form and sigma
    against the exact Schmidt spectrum; the fused direct sum keeps bond <= 33."""
    inst = inputs.config_multi_marked(k=3)
    st = mps.grover_iterate(mps.plus_state(40), inst.marked, 3, inst.chi_max, inst.tol,
                            mode="fused")
    P = mps.prob_marked(st, inst.marked)
    Pc = reduced.closed_form(40, 32, 3)[0]
    assert abs(P - Pc) < 1e-12 and abs(P - Pc) / Pc < 1e-7
    assert max(st.bonds()) <= 33
    for cut in (1, 5, 20, 39):
        assert st.bonds()[cut] == reduced.exact_bond(40, inst.marked, 3, cut)


# ------------------------------------------------------------- sampling
def test_mps_sampler_matches_dense_marginals():
    n, marked = 7, [3, 77, 100]
    rng = np.random.default_rng(1)
    phis, psis = rng.normal(np.pi, 0.4, 3), rng.normal(np.pi, 0.4, 3)
    st = mps.grover_iterate(mps.plus_state(n), marked, 3, 16, phis=phis, psis=psis)
    v = sv.grover(n, marked, 3, phis, psis)
    shots, seed = 300, 99
    b1, m1 = mps.sample(st, shots, seed)
    b2, m2 = sv.conditional_sample(v, n, lambda s, l: philox.uniforms(seed, s, l), shots)
    ok = np.minimum(m1, m2) > 1e-12
    assert ok.sum() > 0.99 * shots
    assert np.array_equal(b1[ok], b2[ok])


def test_sampler_histogram_binomial():
    """4096 shots at n = 12, k = 50: the marked count is Binomial(4096, P)."""
    from scipy import stats
    inst = inputs.config_small()
    st = mps.grover_iterate(mps.plus_state(12), inst.marked, 50, 4)
    bits, _ = mps.sample(st, 4096, seed=2)
    P = reduced.closed_form(12, 1, 50)[0]
    hits = int(np.sum(bits == inst.marked[0]))
    assert stats.binomtest(hits, 4096, P).pvalue > 1e-4
    # unmarked draws at k = 0 are uniform: chi-square over a tiny n
    st0 = mps.plus_state(4)
    b0, _ = mps.sample(st0, 4096, seed=5)
    counts = np.bincount(b0.astype(np.int64), minlength=16)
    assert stats.chisquare(counts).pvalue > 1e-4


# ------------------------------------------------------------- adjoint
def _fd_grad(n, marked, phis, psis, h=1e-4):
    def L(ph, ps):
        return 1.0 - sv.prob_marked(sv.grover(n, marked, len(ph), ph, ps), marked)
    gphi, gpsi = np.zeros(len(phis)), np.zeros(len(psis))
    for j in range(len(phis)):
        e = np.zeros(len(phis)); e[j] = h
        gphi[j] = (L(phis + e, psis) - L(phis - e, psis)) / (2 * h)
        gpsi[j] = (L(phis, psis + e) - L(phis, psis - e)) / (2 * h)
    return gphi, gpsi


@pytest.mark.parametrize("n,M,K", [(4, 1, 5), (6, 3, 8), (8, 2, 6)])
def test_statevector_adjoint_vs_finite_differences(n, M, K):
    marked = inputs.marked_strings(n, M, seed=n + 40)
    rng = np.random.default_rng(K)
    phis, psis = rng.normal(np.pi, 0.3, K), rng.normal(np.pi, 0.3, K)
    L, gphi, gpsi = sv.adjoint(n, marked, phis, psis)
    fphi, fpsi = _fd_grad(n, marked, phis, psis)
    assert np.allclose(gphi, fphi, atol=1e-7)
    assert np.allclose(gpsi, fpsi, atol=1e-7)
    Lr, rphi, rpsi = reduced.loss_and_grad(n, M, phis, psis)
    assert abs(L - Lr) < 1e-12
    assert np.allclose(gphi, rphi, atol=1e-11)
    assert np.allclose(gpsi, rpsi, atol=1e-11)


# --------------------------------------------------- planted mistakes
def test_pins_catch_planted_sign_error(monkeypatch):
    """A diffusion with the sign of its identity term flipped must fail the
    closed-form pin (the test plants the mistake in the oracle on the CPU)."""
    def bad_diffusion(v, e_psi):
        N = v.size
        return (1.0 - e_psi) * v.sum() / N + v
    monkeypatch.setattr(sv, "apply_diffusion", bad_diffusion)
    v = sv.grover(6, [9], 4)
    assert abs(sv.prob_marked(v, [9]) - reduced.closed_form(6, 1, 4)[0]) > 1e-3


def test_pins_catch_planted_conjugation_error(monkeypatch):
    """O with e^{-i phi} instead of e^{i phi} must fail the reduced-model pin."""
    orig = sv.apply_oracle
    monkeypatch.setattr(sv, "apply_oracle", lambda v, m, e: orig(v, m, np.conj(e)))
    phis, psis = np.array([0.4, 1.2, 2.0]), np.array([2.5, 0.3, 1.0])
    v = sv.grover(5, [7, 20], 3, phis, psis)
    P = reduced.amplitudes(5, 2, 3, phis, psis)[0]
    assert abs(sv.prob_marked(v, [7, 20]) - P) > 1e-6


def test_golden_file_is_current():
    """tests/golden/closed_form.json was written by make_golden.py from the oracle."""
    import json, os
    path = os.path.join(os.path.dirname(__file__), "golden", "closed_form.json")
    g = json.load(open(path))
    e = g["n12_M1_k50"]
    assert e["marked"] == inputs.config_small().marked
    assert abs(e["P"] - 0.99994534610911) < 1e-13
    assert abs(g["n29_M1_k18198"]["P"] - 0.99999999848124) < 1e-13
    assert abs(g["n40_M32_k1000"]["P"] - 1.1652723977320e-4) < 1e-15


def test_paper_iteration_count_rule():
    """Eq. 8, k = round(pi/4 sqrt N): 50 at n = 12, 18198 at n = 29, and 9 at
    n = 7 (where floor would give 8)."""
    from paper_2601_03832_gb300.experiments import k_paper
    assert k_paper(12) == 50 and k_paper(29) == 18198 and k_paper(7) == 9
    assert [k_paper(n) for n in (2, 3, 4, 5)] == [2, 2, 3, 4]


def test_gate_primitives_against_definitions():
    """The dense one-qubit gate and multi-controlled phase: H on every qubit
    of |0...0> is |s> (Eq. 2); X on qubit l flips bit l of a basis state;
    the multi-controlled Z reflects only |1...1>; a one-qubit gate on qubit l
    equals the Kronecker product I (x) u (x) I with u in bit position l."""
    import numpy as np
    from oracle import statevector as sv
    n = 5
    H = np.array([[1, 1], [1, -1]]) / np.sqrt(2)
    X = np.array([[0, 1], [1, 0]])
    v = np.zeros(1 << n, dtype=np.complex128)
    v[0] = 1
    for l in range(n):
        v = sv.apply_1q(v, n, l, H)
    assert np.allclose(v, sv.uniform_state(n), atol=1e-15)
    e = np.zeros(1 << n, dtype=np.complex128)
    e[0b00101] = 1
    f = sv.apply_1q(e, n, 3, X)
    assert f[0b01101] == 1 and np.count_nonzero(f) == 1
    z = sv.apply_mcphase(np.ones(1 << n, dtype=np.complex128), np.pi)
    assert abs(z[-1] + 1) < 1e-15 and np.all(z[:-1] == 1)
    rng = np.random.default_rng(1)
    u = rng.normal(size=(2, 2)) + 1j * rng.normal(size=(2, 2))
    x = rng.normal(size=1 << n) + 1j * rng.normal(size=1 << n)
    for l in range(n):
        K = np.kron(np.kron(np.eye(1 << (n - 1 - l)), u), np.eye(1 << l))
        assert np.allclose(sv.apply_1q(x, n, l, u), K @ x, atol=1e-13)
