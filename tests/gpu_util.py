"""Helpers for the GPU tests (host-side contraction of exported tensors)."""
import numpy as np


def dense_from_sites(sites):
    v = sites[0][0]
    for A in sites[1:]:
        v = np.einsum("xa,asb->sxb", v, A)
        s, x, b = v.shape
        v = v.reshape(s * x, b)
    return v[:, 0]


def right_orthonormal_error(A):
    cl, _, cr = A.shape
    m = A.reshape(cl, 2 * cr)
    return float(np.abs(m @ m.conj().T - np.eye(cl)).max())


def schmidt_from_sites(sites, cut):
    """Schmidt values across `cut` (sites < cut | sites >= cut) of a
    right-canonical chain (sites 1..n-1 right-orthonormal, as the SVD sweep
    leaves it): the singular values of the left block's R factor,
    accumulated by QR from the left."""
    R = np.ones((1, 1), dtype=np.complex128)
    for A in sites[:cut]:
        B = np.einsum("ij,jsk->isk", R, A)
        _, R = np.linalg.qr(B.reshape(-1, B.shape[2]))
    return np.linalg.svd(R, compute_uv=False)
