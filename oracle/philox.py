"""Counter-based Gaussian test matrices for the FRSVT oracle (test infrastructure only).

Alg. 1 samples a standard Gaussian matrix Omega (n x l, or n x p under range
propagation); Sec. 2.4 states that the implementation uses dense Gaussian
matrices drawn entry-wise from N(0, 1).  To let the oracle and the CUDA path
use the *same* Omega without passing it around, both sides implement the
Philox4x64-10 counter-based generator from its published definition (Salmon,
Moraes, Dror and Shaw, "Parallel random numbers: as easy as 1, 2, 3", SC'11),
and the same Box-Muller map.  This module is the oracle's own implementation.

Pins:
- ``philox4x64_10`` is checked bit for bit against numpy's independent
  ``numpy.random.Philox`` bit generator (a library implementation of the same
  published function).
- ``gaussian_matrix`` is checked by closed-form values of the Box-Muller map and by
  moment / Kolmogorov-Smirnov tests against N(0, 1).

Definition of the Omega stream (shared contract, restated independently on the
CUDA side):
    key      = (seed, 0)
    counter  = (row i, column block j, stream t, problem b)
    x0..x3   = philox4x64_10(counter, key)                  (four uint64 words)
    u(x)     = ((x >> 41) + 0.5) * 2**-23                    (23-bit uniform in (0,1))
    (z0, z1) = sqrt(-2 ln u(x0)) * (cos 2 pi u(x1), sin 2 pi u(x1))
    (z2, z3) = sqrt(-2 ln u(x2)) * (cos 2 pi u(x3), sin 2 pi u(x3))
    Omega[i, 4j + k] = z_k
"""
from __future__ import annotations

import numpy as np

_M0 = np.uint64(0xD2E7470EE14C6C93)
_M1 = np.uint64(0xCA5A826395121157)
_W0 = np.uint64(0x9E3779B97F4A7C15)
_W1 = np.uint64(0xBB67AE8584CAA73B)
_MASK32 = np.uint64(0xFFFFFFFF)
_S32 = np.uint64(32)


def _mulhilo64(a: np.uint64, b: np.ndarray):
    """Full 128-bit product of a (scalar) and b (array), as (hi, lo) uint64 words."""
    a = np.uint64(a)
    b = np.asarray(b, dtype=np.uint64)
    a_lo, a_hi = a & _MASK32, a >> _S32
    b_lo, b_hi = b & _MASK32, b >> _S32
    ll = a_lo * b_lo
    lh = a_lo * b_hi
    hl = a_hi * b_lo
    hh = a_hi * b_hi
    mid = (ll >> _S32) + (lh & _MASK32) + (hl & _MASK32)
    lo = (ll & _MASK32) | ((mid & _MASK32) << _S32)
    hi = hh + (lh >> _S32) + (hl >> _S32) + (mid >> _S32)
    return hi, lo


def philox4x64_10(counter, key):
    """Philox4x64 with 10 rounds.

    counter: uint64 array of shape (..., 4); key: uint64 array of shape (..., 2)
    (broadcastable).  Returns a uint64 array of shape (..., 4).
    """
    with np.errstate(over="ignore"):
        c = np.asarray(counter, dtype=np.uint64)
        k = np.asarray(key, dtype=np.uint64)
        c0, c1, c2, c3 = (c[..., t].copy() for t in range(4))
        k0 = np.broadcast_to(k[..., 0], c0.shape).copy()
        k1 = np.broadcast_to(k[..., 1], c0.shape).copy()
        for rnd in range(10):
            if rnd > 0:
                k0 = k0 + _W0
                k1 = k1 + _W1
            hi0, lo0 = _mulhilo64(_M0, c0)
            hi1, lo1 = _mulhilo64(_M1, c2)
            c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
        return np.stack([c0, c1, c2, c3], axis=-1)


def uniform23(x: np.ndarray) -> np.ndarray:
    """23-bit uniform in (0, 1): ((x >> 41) + 1/2) * 2^-23, exact in float32 and float64."""
    return ((np.asarray(x, dtype=np.uint64) >> np.uint64(41)).astype(np.float64) + 0.5) * 2.0 ** -23


def box_muller(u_r: np.ndarray, u_t: np.ndarray):
    """Box-Muller map of two uniforms to two independent standard normals (float64)."""
    rad = np.sqrt(-2.0 * np.log(u_r))
    ang = 2.0 * np.pi * u_t
    return rad * np.cos(ang), rad * np.sin(ang)


def philox_words(rows: int, cols: int, seed: int, stream: int, problem: int = 0) -> np.ndarray:
    """Raw Philox words feeding Omega[:rows, :cols]: shape (rows, ceil(cols/4), 4) uint64."""
    nblk = (cols + 3) // 4
    ii, jj = np.meshgrid(np.arange(rows, dtype=np.uint64), np.arange(nblk, dtype=np.uint64), indexing="ij")
    ctr = np.stack([ii, jj,
                    np.full_like(ii, np.uint64(stream)),
                    np.full_like(ii, np.uint64(problem))], axis=-1)
    key = np.array([np.uint64(seed), np.uint64(0)], dtype=np.uint64)
    return philox4x64_10(ctr, key)


def gaussian_matrix(rows: int, cols: int, seed: int, stream: int, problem: int = 0) -> np.ndarray:
    """Omega[:rows, :cols] of the (seed, stream, problem) Gaussian stream, float64."""
    if rows == 0 or cols == 0:
        return np.zeros((rows, cols))
    w = philox_words(rows, cols, seed, stream, problem)
    z0, z1 = box_muller(uniform23(w[..., 0]), uniform23(w[..., 1]))
    z2, z3 = box_muller(uniform23(w[..., 2]), uniform23(w[..., 3]))
    z = np.stack([z0, z1, z2, z3], axis=-1).reshape(rows, -1)
    return np.ascontiguousarray(z[:, :cols])
