"""Dense FP64 statevector oracle (n <= 24).  Test infrastructure only.

The Grover gate of Sec. II, Eq. 3, G = D O with O applied first, in the
phase-generalised form this package computes:

    O(phi) = I - (1 - e^{i phi}) sum_{w in W} |w><w|
    D(psi) = (1 - e^{i psi}) |s><s| - I,   |s> = N^{-1/2} sum_x |x>  (Eq. 2)

phi = psi = pi gives O = I - 2 Pi_W and D = 2|s><s| - I, the standard pair
whose product rotates the {|w>,|r>} plane by 2 theta (Sec. II).  Basis index
x = sum_l b_l 2^l: bit l is qubit / MPS site l.
"""
from __future__ import annotations

import numpy as np


def eiphase(angle):
    """e^{i angle}; None means plain Grover (angle = pi), returned exactly as -1."""
    if angle is None:
        return complex(-1.0, 0.0)
    return complex(np.cos(angle), np.sin(angle))


def _phases(k, phis, psis):
    ph = [eiphase(None if phis is None else phis[j]) for j in range(k)]
    ps = [eiphase(None if psis is None else psis[j]) for j in range(k)]
    return ph, ps


def uniform_state(n: int) -> np.ndarray:
    """|s> of Eq. 2."""
    N = 1 << n
    return np.full(N, 1.0 / np.sqrt(N), dtype=np.complex128)


def apply_oracle(v: np.ndarray, marked, e_phi: complex) -> np.ndarray:
    """O v: multiply the marked amplitudes by e^{i phi}, leave the rest."""
    out = v.copy()
    idx = np.asarray(marked, dtype=np.int64)
    out[idx] = out[idx] * e_phi
    return out


def apply_diffusion(v: np.ndarray, e_psi: complex) -> np.ndarray:
    """D v = (1 - e^{i psi}) <s|v> |s> - v."""
    N = v.size
    s_overlap = v.sum() / np.sqrt(N)          # <s|v>
    return (1.0 - e_psi) * s_overlap / np.sqrt(N) - v


def grover(n: int, marked, k: int, phis=None, psis=None, keep_all: bool = False):
    """|psi_k> = G_k ... G_1 |s>, G_j = D(psi_j) O(phi_j) (Eq. 3, iterative form)."""
    ph, ps = _phases(k, phis, psis)
    v = uniform_state(n)
    hist = [v] if keep_all else None
    for j in range(k):
        v = apply_diffusion(apply_oracle(v, marked, ph[j]), ps[j])
        if keep_all:
            hist.append(v)
    return hist if keep_all else v


def prob_marked(v: np.ndarray, marked) -> float:
    return float(np.sum(np.abs(v[np.asarray(marked, dtype=np.int64)]) ** 2))


def dense_operators(n: int, marked, e_phi: complex, e_psi: complex):
    """Explicit 2^n x 2^n matrices of O and D (tiny n only), from their definitions."""
    N = 1 << n
    Pw = np.zeros((N, N), dtype=np.complex128)
    for w in marked:
        Pw[w, w] = 1.0
    s = uniform_state(n)
    O = np.eye(N, dtype=np.complex128) - (1.0 - e_phi) * Pw
    D = (1.0 - e_psi) * np.outer(s, s.conj()) - np.eye(N, dtype=np.complex128)
    return O, D


def conditional_sample(v: np.ndarray, n: int, uniforms_fn, shots: int):
    """Draw `shots` bitstrings bit by bit, site 0 first, from the exact marginals.

    For shot j at site l with the already drawn low bits `pre`:
    p_b = sum over all x with x mod 2^l = pre and bit l of x = b of |v_x|^2;
    bit l = 1 iff u * (p0 + p1) >= p0, u = uniforms_fn(shots, l).
    Returns (bits uint64 array, margin array) where margin is the smallest
    |u - p0/(p0+p1)| met by each shot (used to flag near-ties).
    """
    prob = np.abs(v) ** 2
    x = np.arange(v.size, dtype=np.int64)
    bits = np.zeros(shots, dtype=np.int64)
    margin = np.full(shots, np.inf)
    for l in range(n):
        u = uniforms_fn(np.arange(shots), l)
        low_mask = (1 << l) - 1
        for j in range(shots):
            sel = (x & low_mask) == bits[j]
            p1 = prob[sel & (((x >> l) & 1) == 1)].sum()
            p0 = prob[sel & (((x >> l) & 1) == 0)].sum()
            tot = p0 + p1
            b = 1 if u[j] * tot >= p0 else 0
            margin[j] = min(margin[j], abs(u[j] - p0 / tot))
            bits[j] |= b << l
    return bits.astype(np.uint64), margin


def adjoint(n: int, marked, phis, psis):
    """Loss L = 1 - P_marked(psi_K) and dL/dphi_k, dL/dpsi_k (k = 1..K), reverse mode.

    psi_k = D_k O_k psi_{k-1};  mu_K = Pi_W psi_K;  nu_k = D_k^dag mu_k;
    dP/dphi_k = 2 Re <nu_k | i e^{i phi_k} Pi_W | psi_{k-1}>
    dP/dpsi_k = 2 Re [ -i e^{i psi_k} <mu_k|s> <s| O_k psi_{k-1}> ]
    mu_{k-1} = O_k^dag nu_k.
    """
    K = len(phis)
    hist = grover(n, marked, K, phis, psis, keep_all=True)
    idx = np.asarray(marked, dtype=np.int64)
    N = 1 << n
    s = uniform_state(n)
    mu = np.zeros(N, dtype=np.complex128)
    mu[idx] = hist[K][idx]
    P = float(np.sum(np.abs(hist[K][idx]) ** 2))
    g_phi = np.zeros(K)
    g_psi = np.zeros(K)
    for k in range(K, 0, -1):
        e_phi = eiphase(phis[k - 1])
        e_psi = eiphase(psis[k - 1])
        prev = hist[k - 1]
        nu = apply_diffusion(mu, np.conj(e_psi))          # D^dag = (1 - e^{-i psi})|s><s| - I
        g_phi[k - 1] = -2.0 * np.real(1j * e_phi * np.vdot(nu[idx], prev[idx]))
        o_prev = apply_oracle(prev, marked, e_phi)
        g_psi[k - 1] = -2.0 * np.real(-1j * e_psi * np.vdot(mu, s) * np.vdot(s, o_prev))
        mu = apply_oracle(nu, marked, np.conj(e_phi))      # O^dag = I - (1 - e^{-i phi}) Pi_W
    return 1.0 - P, g_phi, g_psi


# --------------------------------------------------------- gate-level circuits
def apply_1q(v: np.ndarray, n: int, site: int, u: np.ndarray) -> np.ndarray:
    """A one-qubit gate u (2 x 2) on qubit `site` (bit `site` of the index), the
    elementary gates H and X of the circuit in Fig. 1A."""
    t = v.reshape(1 << (n - 1 - site), 2, 1 << site)
    return np.einsum("st,atb->asb", np.asarray(u, dtype=np.complex128), t).reshape(-1)


def apply_mcphase(v: np.ndarray, phase: float) -> np.ndarray:
    """I - (1 - e^{i phase}) |1...1><1...1|: the multi-controlled phase of
    Fig. 1A (phase pi: the multi-controlled Z)."""
    out = v.copy()
    out[-1] *= complex(np.cos(phase), np.sin(phase))
    return out
