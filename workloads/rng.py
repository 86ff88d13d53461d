"""Counter-based random start vectors.

Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as
1, 2, 3", SC'11): a 4x32-bit counter and a 2x32-bit key go through ten rounds of
two 32x32->64 multiplies (constants 0xD2511F53, 0xCD9E8D57) with the key bumped
by the Weyl constants (0x9E3779B9, 0xBB67AE85) between rounds.

Element e of a vector stream (flat index over the real-valued [rows][cols]
array, real and imaginary parts as separate elements) uses counter
(e mod 2^32, e div 2^32, 0, 0) and key (seed mod 2^32, seed div 2^32).  Its
Gaussian value is the Box-Muller transform sqrt(-2 ln U_a) cos(2 pi U_b) of two
53-bit uniforms in (0, 1): U_a from output words (0, 1), U_b from words (2, 3),
U = ((w_hi * 2^32 + w_lo) >> 11 + 0.5) * 2^-53.

The paper draws TPQ start vectors uniformly on the d_H-sphere (Sec. 3.5.1); a
normalised Gaussian vector has exactly that distribution.
"""
from __future__ import annotations

import numpy as np

_M0 = np.uint64(0xD2511F53)
_M1 = np.uint64(0xCD9E8D57)
_W0 = 0x9E3779B9
_W1 = 0xBB67AE85
_LO = np.uint64(0xFFFFFFFF)
_S32 = np.uint64(32)


def philox4x32_10(c0, c1, c2, c3, k0: int, k1: int):
    """Vectorised Philox4x32-10 over uint64 arrays holding 32-bit words."""
    c0, c1, c2, c3 = (np.asarray(c, dtype=np.uint64) & _LO for c in (c0, c1, c2, c3))
    for r in range(10):
        kk0 = np.uint64((k0 + r * _W0) & 0xFFFFFFFF)
        kk1 = np.uint64((k1 + r * _W1) & 0xFFFFFFFF)
        p0 = _M0 * c0
        p1 = _M1 * c2
        hi0, lo0 = p0 >> _S32, p0 & _LO
        hi1, lo1 = p1 >> _S32, p1 & _LO
        c0, c1, c2, c3 = hi1 ^ c1 ^ kk0, lo1, hi0 ^ c3 ^ kk1, lo0
    return c0, c1, c2, c3


def _words(first: int, count: int, seed: int):
    e = np.arange(first, first + count, dtype=np.uint64)
    return philox4x32_10(e & _LO, e >> _S32, np.zeros_like(e), np.zeros_like(e),
                         seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF)


def philox_uniform53(w_lo, w_hi):
    x = (np.asarray(w_hi, dtype=np.uint64) << _S32) | np.asarray(w_lo, dtype=np.uint64)
    return ((x >> np.uint64(11)).astype(np.float64) + 0.5) * 2.0 ** -53


def philox_gaussian(first: int, count: int, seed: int) -> np.ndarray:
    """Gaussian values of stream elements first .. first+count-1."""
    w0, w1, w2, w3 = _words(first, count, seed)
    ua = philox_uniform53(w0, w1)
    ub = philox_uniform53(w2, w3)
    return np.sqrt(-2.0 * np.log(ua)) * np.cos(6.283185307179586 * ub)


def random_vectors(rows: int, cols: int, seed: int, complex_: bool = False,
                   normalize: bool = True, chunk: int = 1 << 24) -> np.ndarray:
    """[rows][cols] Gaussian start vectors (complex: re/im interleaved stream).

    With normalize=True each column is scaled to unit 2-norm.
    """
    reals = cols * (2 if complex_ else 1)
    n = rows * reals
    out = np.empty(n, dtype=np.float64)
    for a in range(0, n, chunk):
        b = min(n, a + chunk)
        out[a:b] = philox_gaussian(a, b - a, seed)
    out = out.reshape(rows, reals)
    if complex_:
        out = out.view(np.complex128)
    if normalize:
        out /= np.linalg.norm(out, axis=0, keepdims=True)
    return out


def bootstrap_picks(M: int, P: int, n_samples: int, seed: int) -> np.ndarray:
    """[M][P] sample indices drawn uniformly with replacement from
    0 .. n_samples-1: pick e = m * P + p is floor(U * n_samples) (capped at
    n_samples - 1) with U the 53-bit uniform of output words (0, 1) of the
    Philox stream element e under key `seed` (the resamplings of the TPQ
    bootstrap)."""
    w0, w1, _, _ = _words(0, M * P, seed)
    u = philox_uniform53(w0, w1)
    k = np.floor(u * n_samples).astype(np.int64)
    return np.minimum(k, n_samples - 1).reshape(M, P)
