"""Pins of the oracle's factorizations against LAPACK and their defining properties."""
import numpy as np
import pytest

from oracle import linalg


SHAPES = [(1, 1), (4, 3), (3, 4), (7, 7), (50, 20), (20, 50), (120, 120), (600, 30)]


@pytest.mark.parametrize("shape", SHAPES)
def test_jacobi_svd_matches_lapack(shape):
    rng = np.random.default_rng(sum(shape))
    A = rng.standard_normal(shape)
    U, s, Vt = linalg.jacobi_svd(A)
    s_ref = np.linalg.svd(A, compute_uv=False)
    k = min(shape)
    assert U.shape == (shape[0], k) and Vt.shape == (k, shape[1])
    assert np.max(np.abs(s - s_ref)) <= 1e-12 * s_ref[0]
    assert np.linalg.norm((U * s) @ Vt - A) <= 1e-12 * np.linalg.norm(A)
    assert np.linalg.norm(U.T @ U - np.eye(k)) <= 1e-11
    assert np.linalg.norm(Vt @ Vt.T - np.eye(k)) <= 1e-11
    assert np.all(np.diff(s) <= 0)


def test_jacobi_svd_rank_deficient_and_zero():
    rng = np.random.default_rng(3)
    A = rng.standard_normal((40, 4)) @ rng.standard_normal((4, 25))
    U, s, Vt = linalg.jacobi_svd(A)
    assert np.all(s[4:] <= 1e-12 * s[0])
    assert np.linalg.norm(U.T @ U - np.eye(25)) <= 1e-11
    assert np.linalg.norm((U * s) @ Vt - A) <= 1e-12 * np.linalg.norm(A)
    U, s, Vt = linalg.jacobi_svd(np.zeros((6, 4)))
    assert np.all(s == 0) and np.linalg.norm(U.T @ U - np.eye(4)) < 1e-12


def test_jacobi_svd_graded_spectrum():
    rng = np.random.default_rng(4)
    Uq, _ = np.linalg.qr(rng.standard_normal((60, 20)))
    Vq, _ = np.linalg.qr(rng.standard_normal((20, 20)))
    s_true = np.logspace(0, -10, 20)
    A = (Uq * s_true) @ Vq.T
    _, s, _ = linalg.jacobi_svd(A)
    assert np.max(np.abs(s - s_true) / s_true) < 1e-6       # Jacobi keeps small singular values accurate


@pytest.mark.parametrize("n", [1, 2, 5, 16, 33, 120])
def test_jacobi_eig_matches_lapack(n):
    rng = np.random.default_rng(n)
    B = rng.standard_normal((n, n))
    S = B + B.T
    d, V = linalg.jacobi_eig(S)
    d_ref = np.sort(np.linalg.eigvalsh(S))[::-1]
    assert np.max(np.abs(d - d_ref)) <= 1e-12 * max(1.0, np.abs(d_ref).max())
    assert np.linalg.norm(V.T @ V - np.eye(n)) <= 1e-12
    assert np.linalg.norm((V * d) @ V.T - S) <= 1e-12 * np.linalg.norm(S)


@pytest.mark.parametrize("n", [1, 3, 10, 40])
def test_newton_polar_matches_svd_polar(n):
    rng = np.random.default_rng(10 + n)
    C = rng.standard_normal((n, n))
    W, P, it = linalg.newton_polar(C)
    U, s, Vt = np.linalg.svd(C)
    assert np.linalg.norm(W - U @ Vt) <= 1e-11 * n
    assert np.linalg.norm(P - (Vt.T * s) @ Vt) <= 1e-11 * np.linalg.norm(C)
    assert np.linalg.norm(W @ P - C) <= 1e-12 * np.linalg.norm(C) * n
    assert np.min(np.linalg.eigvalsh(P)) > 0
    assert it <= 20


def test_qr_cp_rank_cut_and_span():
    rng = np.random.default_rng(5)
    Y = rng.standard_normal((80, 3)) @ rng.standard_normal((3, 10))
    Q = linalg.qr_cp(Y)
    assert Q.shape == (80, 3)
    assert np.linalg.norm(Q.T @ Q - np.eye(3)) < 1e-13
    assert np.linalg.norm(Y - Q @ (Q.T @ Y)) < 1e-12 * np.linalg.norm(Y)
    Yf = rng.standard_normal((80, 10))
    assert linalg.qr_cp(Yf).shape == (80, 10)
    assert linalg.qr_cp(np.zeros((5, 3))).shape == (5, 0)


def test_mgs_partial_orthogonalization():
    rng = np.random.default_rng(6)
    Qt, _ = np.linalg.qr(rng.standard_normal((50, 4)))
    Y = rng.standard_normal((50, 3))
    Y[:, 1] = Qt @ rng.standard_normal(4)           # lies in span(Qt): dropped
    QY = linalg.mgs(Qt, Y)
    assert QY.shape == (50, 2)
    Q = np.hstack([Qt, QY])
    assert np.linalg.norm(Q.T @ Q - np.eye(6)) < 1e-13
    assert np.array_equal(Q[:, :4], Qt)             # the propagated block is untouched
    # span([Qt, QY]) == span([Qt, Y])
    M = np.hstack([Qt, Y])
    assert np.linalg.norm(M - Q @ (Q.T @ M)) < 1e-12 * np.linalg.norm(M)
