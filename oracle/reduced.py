"""Two-dimensional invariant-plane model of Grover's iteration.  Test
infrastructure only.

Sec. II, Eqs. 1-2: |w> = M^{-1/2} sum_{x in W}|x>, |r> = (N-M)^{-1/2}
sum_{x not in W}|x>, |s> = sin(theta)|w> + cos(theta)|r> with
theta = arcsin sqrt(M/N).  Both operators of the phase-generalised gate
leave span{|w>,|r>} invariant; in the basis (|w>, |r>):

    O(phi) = diag(e^{i phi}, 1)
    D(psi) = (1 - e^{i psi}) s s^T - I,   s = (sin theta, cos theta)

so the state after k gates is the 2-vector a_k = D_k O_k a_{k-1}, a_0 = s.
At phi = psi = pi this is the rotation of Sec. II with the closed form
G^k|s> = sin((2k+1)theta)|w> + cos((2k+1)theta)|r> (Eq. 5) and
P(k) = sin^2((2k+1)theta) (Eq. 6).

This module needs no 2^n memory and serves any n (up to 64).
"""
from __future__ import annotations

import math

import numpy as np


def eiphase(angle):
    if angle is None:
        return complex(-1.0, 0.0)
    return complex(math.cos(angle), math.sin(angle))


def theta(n: int, M: int) -> float:
    """theta = arcsin sqrt(M/N) (Eq. 2)."""
    return math.asin(math.sqrt(M / 2.0 ** n))


def closed_form(n: int, M: int, k: int):
    """(P, marked amplitude, unmarked amplitude) from Eqs. 5-6 at phi = psi = pi."""
    th = theta(n, M)
    N = 2.0 ** n
    a_w = math.sin((2 * k + 1) * th)
    a_r = math.cos((2 * k + 1) * th)
    return a_w ** 2, a_w / math.sqrt(M), a_r / math.sqrt(N - M)


def evolve(n: int, M: int, k: int, phis=None, psis=None) -> np.ndarray:
    """a_k in the (|w>, |r>) basis for the phase sequence (None = pi)."""
    th = theta(n, M)
    s = np.array([math.sin(th), math.cos(th)], dtype=np.complex128)
    a = s.copy()
    for j in range(k):
        e_phi = eiphase(None if phis is None else phis[j])
        e_psi = eiphase(None if psis is None else psis[j])
        a = np.array([e_phi * a[0], a[1]])                     # O
        a = (1.0 - e_psi) * s * np.dot(s, a) - a                # D (s real)
    return a


def amplitudes(n: int, M: int, k: int, phis=None, psis=None):
    """(P_marked, amplitude on each marked x, amplitude on each unmarked x)."""
    a = evolve(n, M, k, phis, psis)
    N = 2.0 ** n
    return float(abs(a[0]) ** 2), a[0] / math.sqrt(M), a[1] / math.sqrt(N - M)


def loss_and_grad(n: int, M: int, phis, psis):
    """L = 1 - |a_w|^2 and its gradient by reverse-mode through the 2x2 products."""
    K = len(phis)
    th = theta(n, M)
    s = np.array([math.sin(th), math.cos(th)], dtype=np.complex128)
    S = np.outer(s, s)
    hist = [s.copy()]
    a = s.copy()
    for j in range(K):
        Om = np.diag([eiphase(phis[j]), 1.0])
        Dm = (1.0 - eiphase(psis[j])) * S - np.eye(2)
        a = Dm @ (Om @ a)
        hist.append(a)
    P = abs(a[0]) ** 2
    # mu_K = Pi_W a_K; dP/dx = 2 Re <mu | dG a_prev> propagated backwards.
    mu = np.array([a[0], 0.0], dtype=np.complex128)
    gphi = np.zeros(K)
    gpsi = np.zeros(K)
    for j in range(K - 1, -1, -1):
        e_phi, e_psi = eiphase(phis[j]), eiphase(psis[j])
        Om = np.diag([e_phi, 1.0])
        Dm = (1.0 - e_psi) * S - np.eye(2)
        dOm = np.diag([1j * e_phi, 0.0])
        dDm = -1j * e_psi * S
        prev = hist[j]
        gphi[j] = -2.0 * np.real(np.vdot(mu, Dm @ (dOm @ prev)))
        gpsi[j] = -2.0 * np.real(np.vdot(mu, dDm @ (Om @ prev)))
        mu = Om.conj().T @ (Dm.conj().T @ mu)
    return 1.0 - P, gphi, gpsi


def _gram_factor(count: int, c: float) -> np.ndarray:
    """F with F F^T = Gram matrix of (count orthonormal basis strings, |+>^{(x)m}),
    where <p|+...+> = c for every basis string p; zero modes dropped."""
    G = np.eye(count + 1)
    G[:count, count] = c
    G[count, :count] = c
    lam, V = np.linalg.eigh(G)
    keep = lam > 1e-13 * lam.max()
    return V[:, keep] * np.sqrt(lam[keep])


def schmidt_values(n: int, marked, k: int, cut: int, phis=None, psis=None) -> np.ndarray:
    """Exact singular values of |psi_k> across the cut (sites < cut | sites >= cut).

    |psi_k> = alpha sum_{x in W}|x> + beta |+>^{(x)n} with
    alpha = a_w/sqrt(M) - a_r/sqrt(N-M), beta = a_r sqrt(N)/sqrt(N-M).
    With the distinct prefixes / suffixes of W and |+> on each side as
    (non-orthogonal) bases, sigma = svd(F_L^T C F_R) for Gram factors F.
    """
    M = len(marked)
    N = 2.0 ** n
    a = evolve(n, M, k, phis, psis)
    alpha = a[0] / math.sqrt(M) - a[1] / math.sqrt(N - M)
    beta = a[1] * math.sqrt(N) / math.sqrt(N - M)
    mask = (1 << cut) - 1
    pre = sorted({w & mask for w in marked})
    suf = sorted({w >> cut for w in marked})
    pi = {p: i for i, p in enumerate(pre)}
    qi = {q: i for i, q in enumerate(suf)}
    C = np.zeros((len(pre) + 1, len(suf) + 1), dtype=np.complex128)
    for w in marked:
        C[pi[w & mask], qi[w >> cut]] += alpha
    C[len(pre), len(suf)] = beta
    FL = _gram_factor(len(pre), 2.0 ** (-cut / 2.0))
    FR = _gram_factor(len(suf), 2.0 ** (-(n - cut) / 2.0))
    return np.linalg.svd(FL.T @ C @ FR, compute_uv=False)


def exact_bond(n: int, marked, k: int, cut: int, phis=None, psis=None, rtol: float = 1e-13) -> int:
    sv = schmidt_values(n, marked, k, cut, phis, psis)
    return int(np.sum(sv > rtol * sv[0]))
