"""Seeded synthetic inputs shaped like the paper's RPCA / WNNM workloads.

This module only draws test data (numpy ``default_rng``); it holds none of the
method's arithmetic and is the one module that both the CUDA-path tests and
the FP64 oracle tests use for inputs.  The paper's own data (its RPCA
generator, videos, face and gait datasets) is not available, so these
generators stand in for it with the shapes and structures below.

- ``lowrank_sparse``: O = L + S, L = G1 G2^T * scale (Gaussian factors), S with
  a fraction of entries at uniformly random positions, values uniform in
  [-amp, amp] (Sec. 4.1 "Robust PCA test": Gaussian low-rank data plus sparse
  corruption).
- ``rpca_300``: 300 x 300, rank 10, 5 % corruption in [-50, 50].
- ``video``: 76800 x 200 (320 x 240 pixels x 200 frames) background of rank 3
  from smooth random bases, about 8 % of pixels covered by moving rectangles,
  Gaussian noise sigma = 0.01 (the weather / background RPCA of Sec. 4.2).
- ``recovery_8192``: 8192 x 8192, rank 100 (factors scaled 1/sqrt(100)), 10 %
  additive corruption in [-10, 10].
- ``wnnm_batch``: 64 x n_i patch groups, n_i uniform in [40, 160], rank-4
  Gaussian product plus N(0, 0.05^2) noise (WNNM, Sec. 1 footnote on WSVT).
- ``unrolled_batch``: 8 x (2048 x 512), rank 8 (factors scaled 1/sqrt(8)),
  5 % outliers in [-20, 20].
- ``subspaces``: columns drawn from a union of independent low-dimensional
  subspaces (orthonormal random bases, Gaussian coefficients), ordered by
  subspace, with a fraction of whole columns corrupted by a large Gaussian
  vector (the sample-specific corruption that the l2,1 term of the
  low-rank-representation problem, Table 6 Type A, models; stands in for the
  motion-segmentation and face data of Sec. 4.3).
"""
from __future__ import annotations

import numpy as np


def lowrank_sparse(m: int, n: int, rank: int, frac: float, amp: float, seed: int,
                   scale: float = 1.0, additive: bool = True, dtype=np.float64):
    """Return (O, L, S) with O = L + S (additive) or O = L outside supp(S), S inside."""
    rng = np.random.default_rng(seed)
    G1 = rng.standard_normal((m, rank))
    G2 = rng.standard_normal((n, rank))
    L = (G1 @ G2.T) * scale
    S = np.zeros((m, n))
    cnt = int(round(frac * m * n))
    if cnt:
        pos = rng.choice(m * n, size=cnt, replace=False)
        S.flat[pos] = rng.uniform(-amp, amp, size=cnt)
    if additive:
        O = L + S
    else:
        O = L.copy()
        O.flat[pos] = S.flat[pos]
        S = O - L
    return O.astype(dtype), L.astype(dtype), S.astype(dtype)


def rpca_300(seed: int = 1001):
    """300 x 300, L = U V^T (U, V 300 x 10 standard normal), 5 % of entries set in [-50, 50]."""
    return lowrank_sparse(300, 300, 10, 0.05, 50.0, seed)


def recovery_8192(seed: int = 1003, n: int = 8192, dtype=np.float32):
    """n x n, rank 100 with factors scaled 1/sqrt(100), 10 % additive corruption in [-10, 10]."""
    return lowrank_sparse(n, n, 100, 0.10, 10.0, seed, scale=1.0 / np.sqrt(100.0), dtype=dtype)


def unrolled_batch(seed: int = 1005, batch: int = 8, m: int = 2048, n: int = 512):
    """batch x (m x n): rank 8 (factors / sqrt(8)), 5 % additive outliers in [-20, 20]."""
    out = [lowrank_sparse(m, n, 8, 0.05, 20.0, seed + 7919 * b, scale=1.0 / np.sqrt(8.0))
           for b in range(batch)]
    return tuple(np.stack([o[t] for o in out]) for t in range(3))


def _smooth_image(rng, h: int, w: int, k: int = 8) -> np.ndarray:
    """Image from k x k random low-frequency cosine coefficients, normalized to [0, 1]."""
    c = rng.standard_normal((k, k))
    y = np.cos(np.pi * np.outer(np.arange(h) + 0.5, np.arange(k)) / h)   # h x k
    x = np.cos(np.pi * np.outer(np.arange(w) + 0.5, np.arange(k)) / w)   # w x k
    img = y @ c @ x.T
    img -= img.min()
    return img / max(img.max(), 1e-12)


def video(seed: int = 1002, h: int = 240, w: int = 320, frames: int = 200, rank: int = 3,
          n_blobs: int = 4, noise: float = 0.01, dtype=np.float32):
    """Video-background RPCA input: O (h*w x frames), background L and foreground mask.

    Background: sum of ``rank`` separable terms u_k v_k^T, u_k a smooth random
    image, v_k a 4-term random cosine series over time, normalized.  Foreground:
    ``n_blobs`` textured rectangles (sides 20..60 px, values uniform in [0, 1])
    moving with constant velocity (at most 3 px/frame, wrapping at the border)
    that replace the background; about 8 % of pixels per frame.  Noise N(0, noise^2).
    """
    rng = np.random.default_rng(seed)
    t = np.arange(frames)
    U = np.stack([_smooth_image(rng, h, w).ravel() for _ in range(rank)], axis=1)
    V = np.empty((frames, rank))
    for k in range(rank):
        a = rng.standard_normal(4)
        f = rng.uniform(0.2, 4.0, size=4)
        ph = rng.uniform(0, 2 * np.pi, size=4)
        v = (a[None, :] * np.cos(2 * np.pi * f[None, :] * t[:, None] / frames + ph[None, :])).sum(1)
        v -= v.min()
        V[:, k] = 0.2 + v / max(v.max(), 1e-12)
    V /= rank
    L = U @ V.T
    O = L.copy()
    mask = np.zeros((h * w, frames), dtype=bool)
    for _ in range(n_blobs):
        bh, bw = rng.integers(20, 61, size=2)
        y0, x0 = rng.uniform(0, h), rng.uniform(0, w)
        vy, vx = rng.uniform(-3, 3, size=2)
        tex = rng.uniform(0.0, 1.0, size=(bh, bw))
        for fr in range(frames):
            ys = (int(y0 + vy * fr) + np.arange(bh)) % h
            xs = (int(x0 + vx * fr) + np.arange(bw)) % w
            idx = (ys[:, None] * w + xs[None, :]).ravel()
            O[idx, fr] = tex.ravel()
            mask[idx, fr] = True
    O += noise * rng.standard_normal(O.shape)
    return O.astype(dtype), L.astype(dtype), mask


def wnnm_batch(seed: int = 1004, batch: int = 16384, m: int = 64, nmin: int = 40,
               nmax: int = 160, rank: int = 4, noise: float = 0.05):
    """List of float32 patch-group matrices 64 x n_i (rank-4 product + noise) and their n_i."""
    rng = np.random.default_rng(seed)
    ns = rng.integers(nmin, nmax + 1, size=batch)
    mats = []
    for n_i in ns:
        A = rng.standard_normal((m, rank)) @ rng.standard_normal((rank, int(n_i)))
        A += noise * rng.standard_normal(A.shape)
        mats.append(A.astype(np.float32))
    return mats, ns.astype(np.int32)


def snow_video(seed: int = 1006, h: int = 288, w: int = 384, frames: int = 20, density: float = 0.03):
    """Weather-artifact workload (Type B, semi-online removal): frames of a static scene (a smooth
    image under a per-frame illumination gain in [0.95, 1.05]: rank 1) with a 24 x 24 square moving
    4 px per frame, and snow: a `density` fraction of each frame's pixels replaced by U[0.85, 1].
    Returns (O (h*w x frames) float32, the clean frames, the snow mask)."""
    rng = np.random.default_rng(seed)
    bg = _smooth_image(rng, h, w)
    gain = rng.uniform(0.95, 1.05, size=frames)
    clean = np.empty((h * w, frames), dtype=np.float64)
    mask = np.zeros((h * w, frames), dtype=bool)
    O = np.empty((h * w, frames), dtype=np.float64)
    y0, x0 = h // 2 - 12, 16
    for t in range(frames):
        img = bg * gain[t]
        xs = x0 + 4 * t
        img[y0:y0 + 24, xs:xs + 24] = 0.9
        clean[:, t] = img.reshape(-1)
        flakes = rng.random(h * w) < density
        mask[:, t] = flakes
        o = clean[:, t].copy()
        o[flakes] = rng.uniform(0.85, 1.0, size=int(flakes.sum()))
        O[:, t] = o
    return O.astype(np.float32), clean, mask


def subspaces(seed: int = 1007, d: int = 60, k: int = 4, dim: int = 3, per: int = 15, frac: float = 0.1,
              amp: float = 3.0):
    """O (d x k*per): `per` columns from each of `k` random `dim`-dimensional subspaces of R^d
    (coefficients N(0, 1)), ordered by subspace; round(frac * n) columns, chosen at random, get
    amp * N(0, I_d) / sqrt(d) added.  Returns (O, the clean columns, labels, the corrupted mask)."""
    rng = np.random.default_rng(seed)
    n = k * per
    clean = np.empty((d, n))
    labels = np.repeat(np.arange(k), per)
    for i in range(k):
        B, _ = np.linalg.qr(rng.standard_normal((d, dim)))
        clean[:, i * per:(i + 1) * per] = B @ rng.standard_normal((dim, per))
    mask = np.zeros(n, dtype=bool)
    mask[rng.choice(n, size=int(round(frac * n)), replace=False)] = True
    O = clean.copy()
    O[:, mask] += amp * rng.standard_normal((d, int(mask.sum()))) / np.sqrt(d)
    return O, clean, labels, mask
