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
