"""Helpers shared by the GPU parity tests (inputs and comparisons only)."""
import numpy as np


def rel_fro(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    den = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / (den if den > 0 else 1.0))


def spectrum_matrix(m, n, rank, decay, noise, seed):
    """m x n float64 matrix with a decaying spectrum sigma_j = 100 * decay^j (j < rank) plus noise."""
    rng = np.random.default_rng(seed)
    U, _ = np.linalg.qr(rng.standard_normal((m, rank)))
    V, _ = np.linalg.qr(rng.standard_normal((n, rank)))
    s = 100.0 * decay ** np.arange(rank)
    A = (U * s) @ V.T + noise * rng.standard_normal((m, n))
    return A, s


def to_gpu(A, ld=None):
    """float32 CUDA copy of A; the leading dimension is ld, or n rounded up to a multiple of 4."""
    import torch
    A32 = np.asarray(A, dtype=np.float32)
    m, n = A32.shape
    if ld is None:
        ld = (n + 3) // 4 * 4
    if ld == n:
        return torch.from_numpy(np.ascontiguousarray(A32)).cuda()
    buf = torch.zeros((m, ld), dtype=torch.float32, device="cuda")
    buf[:, :n] = torch.from_numpy(np.ascontiguousarray(A32)).cuda()
    return buf[:, :n]
