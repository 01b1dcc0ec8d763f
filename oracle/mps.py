"""Plain FP64 matrix-product-state oracle.  Test infrastructure only.

Follows Sec. III-B-2: the state is a chain of site tensors A_l of shape
(chi_l, 2, chi_{l+1}) (chi_0 = chi_n = 1); after each operator the tensors
are updated locally and small singular values are truncated, with the bond
capped at chi_max.  Each Grover gate of Sec. III-A (iterative method: the
state is replaced by G|state> every iteration, G = D O of Eq. 3) is applied
as:

  1. contraction of an operator into the site tensors -- either as a matrix
     product operator (MPO; oracle of bond M+1, diffusion of bond 2) or as
     the equivalent direct sum of the current MPS with product states;
  2. a canonicalising QR sweep, left to right;
  3. a truncated-SVD sweep, right to left, ending with the FP64
     renormalisation of site 0.

Conventions: site l is bit l of the basis index (LSB = site 0); site tensor
index order [left bond][physical][right bond]; complex128 throughout.
Truncation keeps sigma_i > max(tol * sigma_0, max(m, n) * eps * sigma_0) for an
m x n matrix (eps = 2^-52), at least one value, at most chi_max.
"""
from __future__ import annotations

import math

import numpy as np

from .philox import uniforms

EPS = np.finfo(np.float64).eps
PLUS = np.array([1.0, 1.0]) / math.sqrt(2.0)


def eiphase(angle):
    if angle is None:
        return complex(-1.0, 0.0)
    return complex(math.cos(angle), math.sin(angle))


class MPS:
    def __init__(self, sites):
        self.sites = [np.asarray(a, dtype=np.complex128) for a in sites]
        self.log_norm = 0.0       # sum of log(norm) removed by renormalisation
        self.discarded = 0.0      # sum of discarded sigma^2 (relative to the kept norm)

    @property
    def n(self):
        return len(self.sites)

    def bonds(self):
        return [1] + [a.shape[2] for a in self.sites]


# ---------------------------------------------------------------- A0: init
def plus_state(n: int) -> MPS:
    """|s> = |+>^{(x)n} (Eq. 2) as a bond-1 MPS."""
    return MPS([PLUS.reshape(1, 2, 1).astype(np.complex128) for _ in range(n)])


def product_state(bits: int, n: int) -> MPS:
    sites = []
    for l in range(n):
        a = np.zeros((1, 2, 1), dtype=np.complex128)
        a[0, (bits >> l) & 1, 0] = 1.0
        sites.append(a)
    return MPS(sites)


# ------------------------------------------------------- A1/A3: MPO builders
def _close_boundaries(W, left, right):
    """Contract boundary vectors into the first / last MPO tensors."""
    W = [w.copy() for w in W]
    W[0] = np.einsum("a,abst->bst", left, W[0])[None]
    W[-1] = np.einsum("abst,b->ast", W[-1], right)[:, None]
    return W


def oracle_mpo(n: int, marked, phi=None):
    """O = I - (1 - e^{i phi}) sum_w |w><w| as an MPO of bond M+1.

    W_l[a, b, s, s'] = diag(I_2, P_{w_1,l}, ..., P_{w_M,l}) with P_b = |b><b|;
    left boundary (1, e^{i phi}-1, ..., e^{i phi}-1), right boundary all ones.
    """
    M = len(marked)
    c = eiphase(phi) - 1.0
    W = []
    for l in range(n):
        w = np.zeros((M + 1, M + 1, 2, 2), dtype=np.complex128)
        w[0, 0] = np.eye(2)
        for a, x in enumerate(marked, start=1):
            b = (x >> l) & 1
            w[a, a, b, b] = 1.0
        W.append(w)
    left = np.array([1.0] + [c] * M, dtype=np.complex128)
    right = np.ones(M + 1, dtype=np.complex128)
    return _close_boundaries(W, left, right)


def diffusion_mpo(n: int, psi=None):
    """D = (1 - e^{i psi})|s><s| - I as an MPO of bond 2.

    |s><s| = (x)_l |+><+| (Eq. 2), so W_l = diag(I_2, |+><+|), left boundary
    (-1, 1 - e^{i psi}), right boundary (1, 1).
    """
    pp = np.outer(PLUS, PLUS)
    W = []
    for _ in range(n):
        w = np.zeros((2, 2, 2, 2), dtype=np.complex128)
        w[0, 0] = np.eye(2)
        w[1, 1] = pp
        W.append(w)
    left = np.array([-1.0, 1.0 - eiphase(psi)], dtype=np.complex128)
    right = np.ones(2, dtype=np.complex128)
    return _close_boundaries(W, left, right)


def mpo_to_dense(W) -> np.ndarray:
    """Dense 2^n x 2^n matrix of an MPO (tiny n), rows/cols indexed by x = sum b_l 2^l."""
    n = len(W)
    T = W[0][0]                                   # (b, s, t)
    T = T.transpose(1, 2, 0)[..., None]           # (s0, t0, b)->(S, T, b)
    cur = W[0][0].transpose(1, 2, 0)              # S, T, b with S,T over sites so far
    for l in range(1, n):
        cur = np.einsum("STa,abst->SsTtb", cur, W[l])
        S, s, T_, t, b = cur.shape
        # new index: x = S + s * 2^l  -> place s as the higher bit
        cur = cur.transpose(1, 0, 3, 2, 4).reshape(s * S, t * T_, b)
    return cur[..., 0]


# ------------------------------------------------------ A2/A3: contraction
def apply_mpo(state: MPS, W) -> MPS:
    """B_l[(a,i), s, (b,j)] = sum_{s'} W_l[a,b,s,s'] A_l[i,s',j]; bond becomes D*chi."""
    out = []
    for A, w in zip(state.sites, W):
        B = np.einsum("abst,itj->aisbj", w, A)
        a, i, s, b, j = B.shape
        out.append(B.reshape(a * i, s, b * j))
    res = MPS(out)
    res.log_norm, res.discarded = state.log_norm, state.discarded
    return res


def direct_sum(terms, n: int) -> MPS:
    """MPS of sum_t c_t |Phi_t> from (c_t, MPS_t) pairs: block-diagonal site tensors."""
    if n == 1:
        site = sum(c * t.sites[0] for c, t in terms)
        return MPS([site])
    sites = []
    for l in range(n):
        blocks = [t.sites[l] for _, t in terms]
        if l == 0:
            site = np.concatenate([c * b for (c, _), b in zip(terms, blocks)], axis=2)
        elif l == n - 1:
            site = np.concatenate(blocks, axis=0)
        else:
            L = sum(b.shape[0] for b in blocks)
            R = sum(b.shape[2] for b in blocks)
            site = np.zeros((L, 2, R), dtype=np.complex128)
            i0 = j0 = 0
            for b in blocks:
                site[i0:i0 + b.shape[0], :, j0:j0 + b.shape[2]] = b
                i0 += b.shape[0]
                j0 += b.shape[2]
        sites.append(site)
    return MPS(sites)


def apply_oracle_direct(state: MPS, marked, phi=None) -> MPS:
    """O|psi> = |psi> + (e^{i phi} - 1) sum_w psi(w)|w>: bond chi + M."""
    c = eiphase(phi) - 1.0
    terms = [(1.0, state)] + [(c * amplitude(state, w), product_state(w, state.n)) for w in marked]
    res = direct_sum(terms, state.n)
    res.log_norm, res.discarded = state.log_norm, state.discarded
    return res


def apply_diffusion_direct(state: MPS, psi=None) -> MPS:
    """D|phi> = (1 - e^{i psi}) <s|phi> |s> - |phi>: bond chi + 1."""
    c = (1.0 - eiphase(psi)) * overlap_plus(state)
    res = direct_sum([(-1.0, state), (c, plus_state(state.n))], state.n)
    res.log_norm, res.discarded = state.log_norm, state.discarded
    return res


def apply_grover_direct(state: MPS, marked, phi=None, psi=None) -> MPS:
    """G|psi> = D O|psi> in one direct sum (bond chi + M + 1):
    -|psi> - (e^{i phi}-1) sum_w psi(w)|w> + (1-e^{i psi}) <s|O psi> |s>,
    <s|O psi> = <s|psi> + (e^{i phi}-1) 2^{-n/2} sum_w psi(w)."""
    n = state.n
    c = eiphase(phi) - 1.0
    amps = [amplitude(state, w) for w in marked]
    s_o = overlap_plus(state) + c * 2.0 ** (-n / 2.0) * sum(amps)
    terms = [(-1.0, state)] + [(-c * a, product_state(w, n)) for a, w in zip(amps, marked)]
    terms.append(((1.0 - eiphase(psi)) * s_o, plus_state(n)))
    res = direct_sum(terms, n)
    res.log_norm, res.discarded = state.log_norm, state.discarded
    return res


# ------------------------------------------------------------ A4: QR sweep
def qr_sweep(state: MPS) -> MPS:
    """Left-to-right: reshape site l to (2 chi_l) x chi_{l+1}, QR, keep Q, pass R right."""
    s = [a.copy() for a in state.sites]
    for l in range(len(s) - 1):
        cl, _, cr = s[l].shape
        Q, R = np.linalg.qr(s[l].reshape(cl * 2, cr), mode="reduced")
        s[l] = Q.reshape(cl, 2, Q.shape[1])
        s[l + 1] = np.einsum("ij,jsk->isk", R, s[l + 1])
    res = MPS(s)
    res.log_norm, res.discarded = state.log_norm, state.discarded
    return res


# ----------------------------------------------------------- A5: SVD sweep
def keep_count(S: np.ndarray, m: int, n: int, chi_max: int, tol: float) -> int:
    if S.size == 0 or S[0] == 0.0:
        return 1
    thr = max(tol * S[0], max(m, n) * EPS * S[0])
    return max(1, min(int(np.sum(S > thr)), chi_max))


def svd_sweep(state: MPS, chi_max: int, tol: float = 0.0) -> MPS:
    """Right-to-left: reshape site l to chi_l x (2 chi_{l+1}), SVD, truncate, keep V^dag,
    pass U S left; finally renormalise site 0 (FP64) and record log-norm and
    discarded weight."""
    s = [a.copy() for a in state.sites]
    disc = state.discarded
    for l in range(len(s) - 1, 0, -1):
        cl, _, cr = s[l].shape
        m = s[l].reshape(cl, 2 * cr)
        U, S, Vh = np.linalg.svd(m, full_matrices=False)
        k = keep_count(S, m.shape[0], m.shape[1], chi_max, tol)
        tot = float(np.sum(S ** 2))
        if tot > 0:
            disc += float(np.sum(S[k:] ** 2)) / tot
        s[l] = Vh[:k].reshape(k, 2, cr)
        s[l - 1] = np.einsum("isj,jk->isk", s[l - 1], U[:, :k] * S[:k])
    nrm = float(np.linalg.norm(s[0]))
    s[0] = s[0] / nrm
    res = MPS(s)
    res.log_norm = state.log_norm + math.log(nrm)
    res.discarded = disc
    return res


def recompress(state: MPS, chi_max: int, tol: float) -> MPS:
    return svd_sweep(qr_sweep(state), chi_max, tol)


# ------------------------------------------------- the iterative method
def grover_iterate(state: MPS, marked, k: int, chi_max: int, tol: float = 0.0,
                   phis=None, psis=None, mode: str = "mpo") -> MPS:
    """k iterations of the iterative method (Sec. III-A): state <- G_j state.

    mode "mpo":    O as an MPO, QR+SVD sweeps; D as an MPO, QR+SVD sweeps.
    mode "split":  the same two steps with the direct-sum contraction.
    mode "fused":  G = D O as one direct sum, one QR+SVD sweep pair.
    """
    n = state.n
    for j in range(k):
        phi = None if phis is None else phis[j]
        psi = None if psis is None else psis[j]
        if mode == "mpo":
            state = recompress(apply_mpo(state, oracle_mpo(n, marked, phi)), chi_max, tol)
            state = recompress(apply_mpo(state, diffusion_mpo(n, psi)), chi_max, tol)
        elif mode == "split":
            state = recompress(apply_oracle_direct(state, marked, phi), chi_max, tol)
            state = recompress(apply_diffusion_direct(state, psi), chi_max, tol)
        elif mode == "fused":
            state = recompress(apply_grover_direct(state, marked, phi, psi), chi_max, tol)
        else:
            raise ValueError(mode)
    return state


# ---------------------------------------------------- S2: amplitudes
def amplitude(state: MPS, bits: int) -> complex:
    """<bits|psi> = prod_l A_l[:, b_l, :]."""
    v = np.ones(1, dtype=np.complex128)
    for l, A in enumerate(state.sites):
        v = v @ A[:, (bits >> l) & 1, :]
    return complex(v[0])


def overlap_plus(state: MPS) -> complex:
    """<s|psi> = prod_l (A_l[:,0,:] + A_l[:,1,:]) / sqrt 2."""
    v = np.ones(1, dtype=np.complex128)
    for A in state.sites:
        v = v @ ((A[:, 0, :] + A[:, 1, :]) / math.sqrt(2.0))
    return complex(v[0])


def prob_marked(state: MPS, marked) -> float:
    return float(sum(abs(amplitude(state, w)) ** 2 for w in marked))


def to_dense(state: MPS) -> np.ndarray:
    """Full 2^n vector (tiny n), index x = sum_l b_l 2^l."""
    v = state.sites[0][0]                       # (2, chi)
    for l in range(1, state.n):
        v = np.einsum("xa,asb->sxb", v, state.sites[l])
        s, x, b = v.shape
        v = v.reshape(s * x, b)
    return v[:, 0]


# ---------------------------------------------------- S1: perfect sampling
def sample(state: MPS, shots: int, seed: int):
    """Perfect sampling, site 0 first, on a right-canonical MPS (as left by svd_sweep).

    For each shot: v = [1]; at site l, v_b = v A_l[:, b, :], p_b = |v_b|^2,
    bit = 1 iff u (p0 + p1) >= p0 with u = Philox uniform of (shot, l);
    v <- v_bit / sqrt(p_bit).
    Returns (bits as uint64, per-shot smallest |u - p0/(p0+p1)|).
    """
    bits = np.zeros(shots, dtype=np.uint64)
    margin = np.full(shots, np.inf)
    v = np.ones((shots, 1), dtype=np.complex128)
    for l, A in enumerate(state.sites):
        u = uniforms(seed, np.arange(shots, dtype=np.uint64), l)
        v0 = v @ A[:, 0, :]
        v1 = v @ A[:, 1, :]
        p0 = np.sum(np.abs(v0) ** 2, axis=1)
        p1 = np.sum(np.abs(v1) ** 2, axis=1)
        tot = p0 + p1
        b = (u * tot >= p0)
        margin = np.minimum(margin, np.abs(u - p0 / tot))
        bits |= b.astype(np.uint64) << np.uint64(l)
        v = np.where(b[:, None], v1 / np.sqrt(p1)[:, None], v0 / np.sqrt(p0)[:, None])
    return bits, margin


def is_left_orthonormal(A, atol=1e-12) -> bool:
    cl, _, cr = A.shape
    m = A.reshape(cl * 2, cr)
    return np.allclose(m.conj().T @ m, np.eye(cr), atol=atol)


def is_right_orthonormal(A, atol=1e-12) -> bool:
    cl, _, cr = A.shape
    m = A.reshape(cl, 2 * cr)
    return np.allclose(m @ m.conj().T, np.eye(cl), atol=atol)
