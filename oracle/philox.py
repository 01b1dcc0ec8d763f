"""Philox4x64-10 (Salmon, Moraes, Dror & Shaw, "Parallel random numbers: as
easy as 1, 2, 3", SC'11), written from the published round function.

Used for the perfect-sampling uniforms (Sec. IV-3, shots): for shot `j` and
site `l` the counter is (j, l, 0, 0) and the key is (seed, 0); the uniform is
u = (word0 >> 11) * 2^-53 in [0, 1).

Test infrastructure only (see oracle/__init__.py).
"""
from __future__ import annotations

import numpy as np

_M0 = np.uint64(0xD2E7470EE14C6C93)
_M1 = np.uint64(0xCA5A826395121157)
_W0 = np.uint64(0x9E3779B97F4A7C15)
_W1 = np.uint64(0xBB67AE8584CAA73B)
_LO32 = np.uint64(0xFFFFFFFF)
_S32 = np.uint64(32)


def _mulhilo(a: np.ndarray, b: np.uint64):
    """(hi, lo) 64-bit halves of the 128-bit product a*b, schoolbook on 32-bit limbs."""
    a0, a1 = a & _LO32, a >> _S32
    b0, b1 = b & _LO32, b >> _S32
    p00, p01, p10, p11 = a0 * b0, a0 * b1, a1 * b0, a1 * b1
    mid = (p00 >> _S32) + (p01 & _LO32) + (p10 & _LO32)
    hi = p11 + (p01 >> _S32) + (p10 >> _S32) + (mid >> _S32)
    lo = a * b
    return hi, lo


def philox4x64_10(ctr, key):
    """Ten Philox4x64 rounds.  `ctr` is a (4, ...) uint64 array, `key` a (2, ...) one.

    Returns the four output words, shape like `ctr`.
    """
    with np.errstate(over="ignore"):
        x0, x1, x2, x3 = (np.asarray(c, dtype=np.uint64).copy() for c in ctr)
        k0, k1 = (np.asarray(k, dtype=np.uint64).copy() for k in key)
        for r in range(10):
            if r > 0:
                k0 = k0 + _W0
                k1 = k1 + _W1
            hi0, lo0 = _mulhilo(x0, _M0)
            hi1, lo1 = _mulhilo(x2, _M1)
            x0, x1, x2, x3 = hi1 ^ x1 ^ k0, lo1, hi0 ^ x3 ^ k1, lo0
    return np.stack([x0, x1, x2, x3])


def uniforms(seed: int, shots: np.ndarray, site: int) -> np.ndarray:
    """u in [0,1) for counters (shot, site, 0, 0), key (seed, 0)."""
    shots = np.asarray(shots, dtype=np.uint64)
    z = np.zeros_like(shots)
    out = philox4x64_10([shots, np.full_like(shots, site), z, z],
                        [np.full_like(shots, seed & 0xFFFFFFFFFFFFFFFF), z])
    return (out[0] >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)
