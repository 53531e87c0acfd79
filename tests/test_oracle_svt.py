"""Pins of the oracle's SVT operators (Def. 1 / Eq. 2-3, Def. 3, Prop. 1-2, Lemma 2, Theorem 3, Alg. 1)."""
import numpy as np
import pytest
import scipy.optimize

from oracle import linalg, svt
from oracle.philox import gaussian_matrix


def nnm_objective(X, A, tau):
    """Eq. 2: tau ||X||_* + 1/2 ||X - A||_F^2 (nuclear norm from LAPACK singular values)."""
    return tau * np.linalg.svd(X, compute_uv=False).sum() + 0.5 * np.sum((X - A) ** 2)


def factored_minimizer(A, tau, weights=None, starts=6, seed=0):
    """Minimize Eq. 2 without any SVD: ||X||_* = min_{X = U V^T} (||U||_F^2 + ||V||_F^2) / 2.

    BFGS over the factors (U: m x n, V: n x n) of the smooth objective
    tau/2 (||U||^2 + ||V||^2) + 1/2 ||U V^T - A||^2 from several random starts;
    returns the best X = U V^T.
    """
    m, n = A.shape
    rng = np.random.default_rng(seed)

    def fg(z):
        U, V = z[: m * n].reshape(m, n), z[m * n:].reshape(n, n)
        R = U @ V.T - A
        f = 0.5 * tau * (np.sum(U * U) + np.sum(V * V)) + 0.5 * np.sum(R * R)
        gU = tau * U + R @ V
        gV = tau * V + R.T @ U
        return f, np.concatenate([gU.ravel(), gV.ravel()])

    best = None
    for _ in range(starts):
        z0 = rng.standard_normal(m * n + n * n)
        res = scipy.optimize.minimize(fg, z0, jac=True, method="BFGS", options={"gtol": 1e-12, "maxiter": 20000})
        if best is None or res.fun < best.fun:
            best = res
    U, V = best.x[: m * n].reshape(m, n), best.x[m * n:].reshape(n, n)
    return U @ V.T


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_exact_svt_brute_force_4x3(seed):
    """Eq. 2 minimized by an SVD-free method agrees with the oracle's exact SVT on 4 x 3 inputs."""
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((4, 3)) * 2.0
    tau = np.linalg.svd(A, compute_uv=False)[1] * 0.9      # some singular values survive, some do not
    X, r = svt.exact_svt(A, tau)
    Xb = factored_minimizer(A, tau, seed=seed)
    assert nnm_objective(X, A, tau) <= nnm_objective(Xb, A, tau) + 1e-12
    assert np.linalg.norm(X - Xb) < 1e-6 * np.linalg.norm(A)     # strong convexity: unique minimizer


@pytest.mark.parametrize("shape", [(4, 3), (30, 20), (20, 45)])
def test_exact_svt_strong_convexity_certificate(shape):
    """f(X* + D) >= f(X*) + 1/2 ||D||^2 for the 1-strongly convex Eq. 2 at its minimizer."""
    rng = np.random.default_rng(7)
    A = rng.standard_normal(shape)
    tau = 0.5 * np.linalg.svd(A, compute_uv=False)[0]
    X, _ = svt.exact_svt(A, tau)
    f0 = nnm_objective(X, A, tau)
    for k in range(50):
        D = rng.standard_normal(shape) * 10.0 ** rng.uniform(-6, 0)
        assert nnm_objective(X + D, A, tau) >= f0 + 0.5 * np.sum(D ** 2) - 1e-11 * max(1.0, f0)


def test_exact_svt_diagonal_closed_form():
    d = np.array([5.0, -3.0, 1.5, 0.2, -0.7])
    A = np.zeros((7, 5))
    A[np.arange(5), np.arange(5)] = d
    X, r = svt.exact_svt(A, 1.0)
    ref = np.zeros((7, 5))
    ref[np.arange(5), np.arange(5)] = np.sign(d) * np.maximum(np.abs(d) - 1.0, 0.0)
    assert np.allclose(X, ref, atol=1e-13)
    assert r == 3


def test_exact_svt_orthogonal_invariance():
    rng = np.random.default_rng(8)
    A = rng.standard_normal((25, 15))
    U, _ = np.linalg.qr(rng.standard_normal((25, 25)))
    V, _ = np.linalg.qr(rng.standard_normal((15, 15)))
    tau = 2.0
    X1, _ = svt.exact_svt(U @ A @ V.T, tau)
    X0, _ = svt.exact_svt(A, tau)
    assert np.linalg.norm(X1 - U @ X0 @ V.T) < 1e-12 * np.linalg.norm(X0)


def test_exact_svt_prox_optimality_and_rank():
    """A - X = P_tau(A) (Def. 3, Lemma 1), ||A - X||_2 = min(sigma_1, tau), U_r^T (A - X) V_r = tau I."""
    rng = np.random.default_rng(9)
    A = rng.standard_normal((40, 30))
    s = np.linalg.svd(A, compute_uv=False)
    tau = 0.5 * (s[5] + s[6])
    X, r = svt.exact_svt(A, tau)
    assert r == 6 == np.linalg.matrix_rank(X, tol=1e-9 * s[0])
    G = A - X
    assert np.linalg.norm(G - svt.ball_projection(A, tau)) < 1e-12 * np.linalg.norm(A)
    assert abs(np.linalg.norm(G, 2) - min(s[0], tau)) < 1e-12 * s[0]
    U, sx, Vt = np.linalg.svd(X)
    Ur, Vr = U[:, :r], Vt[:r].T
    assert np.allclose(Ur.T @ G @ Vr, tau * np.eye(r), atol=1e-11)
    # split of A into S_tau(A) + P_tau(A)
    assert np.linalg.norm(X + svt.ball_projection(A, tau) - A) < 1e-12 * np.linalg.norm(A)
    # tau above sigma_1 gives zero
    X0, r0 = svt.exact_svt(A, s[0] * 1.0001)
    assert r0 == 0 and np.all(X0 == 0)


def test_pseudo_contractions():
    """Prop. 2 (Frobenius) and Prop. 3 with C = 2 (spectral) on random pairs."""
    rng = np.random.default_rng(10)
    for _ in range(10):
        A = rng.standard_normal((12, 9))
        B = A + rng.standard_normal((12, 9)) * rng.uniform(0.01, 1.0)
        tau = rng.uniform(0.5, 3.0)
        SA, _ = svt.exact_svt(A, tau)
        SB, _ = svt.exact_svt(B, tau)
        PA, PB = svt.ball_projection(A, tau), svt.ball_projection(B, tau)
        lhs = np.sum((SA - SB) ** 2)
        assert lhs <= np.sum((A - B) ** 2) - np.sum((PA - PB) ** 2) + 1e-10
        assert np.linalg.norm(SA - SB, 2) <= 2 * np.linalg.norm(A - B, 2) - np.linalg.norm(PA - PB, 2) + 1e-10


def test_lemma2_tail_sum():
    """||P_tau(A) - P_tau(A_k)||_F^2 = sum_{j>k} min(sigma_j, tau)^2 for the best rank-k projection."""
    rng = np.random.default_rng(11)
    A = rng.standard_normal((30, 20))
    U, s, Vt = np.linalg.svd(A, full_matrices=False)
    k, tau = 5, 0.5 * s[3]
    Ak = U[:, :k] @ (U[:, :k].T @ A)
    lhs = np.sum((svt.ball_projection(A, tau) - svt.ball_projection(Ak, tau)) ** 2)
    assert abs(lhs - np.sum(np.minimum(s[k:], tau) ** 2)) < 1e-10 * lhs


# ---------------------------------------------------------------- FRSVT (Alg. 1)

@pytest.mark.parametrize("shape,rank,l,q", [((200, 80), 5, 10, 0), ((200, 80), 5, 10, 2),
                                            ((60, 150), 8, 8, 1), ((90, 90), 12, 20, 1)])
def test_frsvt_exact_when_rank_le_l(shape, rank, l, q):
    """FRSVT is exact when rank(A) <= l (remark after Cor. 2)."""
    rng = np.random.default_rng(rank)
    A = rng.standard_normal((shape[0], rank)) @ rng.standard_normal((rank, shape[1]))
    s = np.linalg.svd(A, compute_uv=False)
    tau = 0.5 * (s[rank // 2] + s[rank // 2 + 1])
    Xe, re = svt.exact_svt(A, tau)
    out = svt.frsvt(A, tau, l, q, seed=3, stream=0)
    assert out.r == re
    assert out.s == rank                        # the pivoted QR cut the basis to rank(A)
    assert np.linalg.norm(out.X - Xe) <= 1e-10 * np.linalg.norm(Xe)


def test_frsvt_range_propagation_exact_when_basis_captures_range():
    rng = np.random.default_rng(12)
    A = rng.standard_normal((150, 6)) @ rng.standard_normal((6, 70))     # tall: short side is 70
    tau = 0.3 * np.linalg.svd(A, compute_uv=False)[3]
    first = svt.frsvt(A, tau, 10, 1, seed=1, stream=0)
    assert first.Q_tilde.shape == (70, min(first.r, 8))
    B = A + 1e-3 * rng.standard_normal(A.shape) @ np.diag(np.ones(70))   # slightly perturbed next iterate
    second = svt.frsvt(B, tau, 10, 1, seed=1, stream=1, Q_prev=first.Q_tilde)
    Xe, _ = svt.exact_svt(B, tau)
    assert np.linalg.norm(second.X - Xe) <= 1e-6 * np.linalg.norm(Xe)


def test_frsvt_depends_only_on_span_of_Q(monkeypatch):
    """Prop. 1: X = Q S_tau(Q^T A) is invariant to the orthonormalization used."""
    rng = np.random.default_rng(13)
    A = rng.standard_normal((120, 60))
    tau = 0.5 * np.linalg.svd(A, compute_uv=False)[4]
    X1 = svt.frsvt(A, tau, 12, 1, seed=5, stream=2).X
    monkeypatch.setattr(linalg, "qr_cp", lambda Y, tol=1e-12: np.linalg.qr(Y)[0])
    X2 = svt.frsvt(A, tau, 12, 1, seed=5, stream=2).X
    assert np.linalg.norm(X1 - X2) <= 1e-11 * np.linalg.norm(X1)


def test_frsvt_equals_projected_exact_svt():
    """With Q from the same Omega, FRSVT(A) = Q S_tau(Q^T A) computed by the exact SVT (Prop. 1)."""
    rng = np.random.default_rng(14)
    A = rng.standard_normal((90, 40))            # tall: work on A^T (40 x 90), Omega has 90 rows
    tau, l, q = 3.0, 10, 1
    out = svt.frsvt(A, tau, l, q, seed=9, stream=4)
    Ah = A.T
    Om = gaussian_matrix(90, l, 9, 4)
    Q = np.linalg.qr(Ah @ Om)[0]
    Q = np.linalg.qr(Ah @ (Ah.T @ Q))[0]
    Xs, _ = svt.exact_svt(Q.T @ Ah, tau)
    assert np.linalg.norm(out.X - (Q @ Xs).T) <= 1e-11 * np.linalg.norm(out.X)


def test_frsvt_theorem3_average_bound():
    """E ||S_tau(A) - S_tau(A_k_hat)||_F^2 <= (1 + k/(p-1)) sum_{j>k} sigma_j^2 - G(A), q = 0 (Eq. 9)."""
    rng = np.random.default_rng(15)
    U, _ = np.linalg.qr(rng.standard_normal((80, 40)))
    V, _ = np.linalg.qr(rng.standard_normal((40, 40)))
    s = 1.0 / (1.0 + np.arange(40)) ** 1.2 * 10
    A = (U * s) @ V.T                         # tall 80 x 40: short side 40
    k, p, tau = 6, 4, 0.5 * s[3]
    Xe, _ = svt.exact_svt(A, tau)
    errs = [np.sum((svt.frsvt(A, tau, k + p, 0, seed=21, stream=t).X - Xe) ** 2) for t in range(200)]
    tail = np.sum(s[k:] ** 2)
    bound = (1 + k / (p - 1)) * tail - np.sum(np.minimum(s[k:], tau) ** 2)
    assert np.mean(errs) <= bound


def test_frsvt_polar_route_matches_jacobi_svd_of_core():
    """Steps 16-19: the polar + eigen route gives the SVD of B (D = singular values of B)."""
    rng = np.random.default_rng(16)
    A = rng.standard_normal((70, 50))
    out = svt.frsvt(A, 1.0, 15, 1, seed=2, stream=0)
    Ah = A.T
    Q = np.linalg.qr(Ah @ gaussian_matrix(70, 15, 2, 0))[0]
    Q = np.linalg.qr(Ah @ (Ah.T @ Q))[0]
    _, sB, _ = linalg.jacobi_svd(Q.T @ Ah)
    assert np.max(np.abs(out.sigma - sB)) <= 1e-12 * sB[0]


def test_frsvt_edge_cases():
    A = np.zeros((10, 6))
    out = svt.frsvt(A, 1.0, 4, 1, 0, 0)
    assert np.all(out.X == 0) and out.r == 0
    out = svt.frsvt(np.zeros((0, 5)), 1.0, 4, 1, 0, 0)
    assert out.X.shape == (0, 5)
    rng = np.random.default_rng(17)
    A = rng.standard_normal((30, 8))
    out = svt.frsvt(A, 0.0, 20, 1, 0, 0)        # l > short side: exact (s = 8), tau = 0 gives A back
    assert np.linalg.norm(out.X - A) < 1e-12 * np.linalg.norm(A)


# ---------------------------------------------------------------- weighted SVT

def test_wsvt_reduces_to_svt_for_constant_weights():
    rng = np.random.default_rng(18)
    A = rng.standard_normal((20, 12))
    assert np.allclose(svt.wsvt(A, np.full(12, 1.3)), svt.exact_svt(A, 1.3)[0], atol=1e-12)


@pytest.mark.parametrize("seed", [0, 1])
def test_wsvt_brute_force_nondescending_weights(seed):
    """argmin sum_j w_j sigma_j(X) + 1/2 ||X - A||^2 for non-descending w is U max(Sigma - w, 0) V^T."""
    rng = np.random.default_rng(40 + seed)
    A = rng.standard_normal((4, 3)) * 2
    w = np.sort(rng.uniform(0.3, 1.5, size=3))
    X = svt.wsvt(A, w)
    f = lambda x: (np.sort(np.linalg.svd(x.reshape(4, 3), compute_uv=False))[::-1] @ w
                   + 0.5 * np.sum((x.reshape(4, 3) - A) ** 2))
    best = min((scipy.optimize.minimize(f, st, method="Powell",
                                        options={"xtol": 1e-10, "ftol": 1e-14, "maxfev": 200000})
                for st in (A.ravel(), np.zeros(12), rng.standard_normal(12))), key=lambda r: r.fun)
    assert f(X.ravel()) <= best.fun + 1e-9


def test_wnnm_weights_rule():
    w = svt.wnnm_weights(100, 2.8, 1e-8)(np.array([4.0, 1.0]))
    assert np.allclose(w, [28.0 / (4.0 + 1e-8), 28.0 / (1.0 + 1e-8)], rtol=1e-14, atol=0)


@pytest.mark.parametrize("shape", [(64, 100), (64, 64), (64, 40)])
def test_weighted_frsvt_equals_wsvt_when_rank_fits(shape):
    """rank(A) <= l: D are the exact singular values, so the weighted FRSVT is the exact WSVT."""
    rng = np.random.default_rng(52)
    m, n = shape
    A = rng.standard_normal((m, 4)) @ rng.standard_normal((4, n))
    w = svt.wnnm_weights(n, 2.8, 1e-8)
    X = svt.frsvt(A, 0.0, 12, 1, 3, 0, problem=5, weights=w).X
    Xe = svt.wsvt(A, w)
    assert np.linalg.norm(X - Xe) <= 1e-10 * np.linalg.norm(Xe)
    # the weights kill some but not all directions: X is neither A nor 0
    assert 0 < np.linalg.norm(Xe) < np.linalg.norm(A)


def test_weighted_frsvt_constant_weights_is_frsvt():
    rng = np.random.default_rng(53)
    A = rng.standard_normal((64, 120))
    a = svt.frsvt(A, 2.5, 12, 1, 7, 1, problem=3)
    b = svt.frsvt(A, 0.0, 12, 1, 7, 1, problem=3, weights=lambda d: np.full_like(d, 2.5))
    assert np.array_equal(a.X, b.X) and a.r == b.r


def test_wsvt_batch_matches_per_problem_calls():
    rng = np.random.default_rng(54)
    mats = [rng.standard_normal((64, n)) for n in (40, 64, 97)]
    ex = svt.wsvt_batch(mats, 2.8, 1e-8, "exact")
    fr = svt.wsvt_batch(mats, 2.8, 1e-8, "frsvt", l=12, q=1, seed=9, stream=2)
    for b, A in enumerate(mats):
        w = svt.wnnm_weights(A.shape[1], 2.8, 1e-8)
        assert np.array_equal(ex[b], svt.wsvt(A, w))
        assert np.array_equal(fr[b], svt.frsvt(A, 0.0, 12, 1, 9, 2, problem=b, weights=w).X)


def test_psvt_keeps_leading_values():
    rng = np.random.default_rng(19)
    A = rng.standard_normal((15, 10))
    U, s, Vt = np.linalg.svd(A, full_matrices=False)
    X = svt.psvt(A, 0.8, 1)
    sx = np.linalg.svd(X, compute_uv=False)
    assert abs(sx[0] - s[0]) < 1e-12 * s[0]
    assert np.allclose(np.sort(sx[1:])[::-1][: np.sum(s[1:] > 0.8)], (s[1:] - 0.8)[s[1:] > 0.8], atol=1e-12)


def test_partial_frsvt_equals_psvt_when_rank_fits():
    """FRSVT with partial thresholding (Table 6, Type B) is exact when rank(A) <= l, like the plain
    operator: it equals the partial SVT computed from the full SVD."""
    rng = np.random.default_rng(23)
    U, _ = np.linalg.qr(rng.standard_normal((60, 4)))
    V, _ = np.linalg.qr(rng.standard_normal((9, 4)))
    A = (U * np.array([9.0, 5.0, 2.0, 0.6])) @ V.T
    for k in (1, 2):
        out = svt.frsvt(A, 1.0, 6, 1, 4, 0, partial_k=k)
        assert np.allclose(out.X, svt.psvt(A, 1.0, k), atol=1e-12)
        assert out.r == 3                        # kept + the values above tau


def test_ialm_partial_svt_separates_rank_one_background():
    """Type B iALM (truncated nuclear norm, k = 1) on a short window: a rank-1 scene plus sparse
    bright outliers is separated, by the exact partial SVT and by FRSVT with partial thresholding."""
    from oracle import rpca
    rng = np.random.default_rng(5)
    m, n = 400, 5
    bg = rng.uniform(0.2, 0.8, size=m)
    L = np.outer(bg, rng.uniform(0.9, 1.1, size=n))
    S = np.zeros((m, n))
    pos = rng.choice(m * n, size=int(0.05 * m * n), replace=False)
    S.flat[pos] = rng.uniform(0.5, 1.0, size=pos.size)
    O = L + S
    ex = rpca.ialm_rpca(O, method="exact", partial_k=1, fixed_iters=60)
    fr = rpca.ialm_rpca(O, method="frsvt", l=3, q=2, seed=1, partial_k=1, fixed_iters=60)
    assert ex.history[-1] < 1e-12 and ex.ranks[-1] == 1
    assert np.linalg.norm(ex.L - L) / np.linalg.norm(L) < 0.1     # the rank-1 scene, up to the model's bias
    assert np.linalg.norm(fr.L - ex.L) / np.linalg.norm(ex.L) < 1e-5
    assert fr.ranks[-1] == 1


# ---------------------------------------------------------------- SVT adjoint

@pytest.mark.parametrize("shape", [(7, 5), (5, 7), (6, 6)])
def test_svt_vjp_matches_central_differences(shape):
    """<Abar, E> and taubar against central differences of exact_svt (FP64, h = 1e-6)."""
    rng = np.random.default_rng(61)
    m, n = shape
    A = rng.standard_normal((m, n))
    s = np.linalg.svd(A, compute_uv=False)
    tau = 0.5 * (s[1] + s[2])                     # away from every sigma_i
    Xbar = rng.standard_normal((m, n))
    Abar, taubar = svt.svt_vjp(A, tau, Xbar)
    h = 1e-6
    for _ in range(4):
        E = rng.standard_normal((m, n))
        fd = np.sum(Xbar * (svt.exact_svt(A + h * E, tau)[0] - svt.exact_svt(A - h * E, tau)[0])) / (2 * h)
        assert abs(np.sum(Abar * E) - fd) < 1e-6 * max(1.0, abs(fd))
    fdt = np.sum(Xbar * (svt.exact_svt(A, tau + h)[0] - svt.exact_svt(A, tau - h)[0])) / (2 * h)
    assert abs(taubar - fdt) < 1e-6 * max(1.0, abs(fdt))


def test_svt_vjp_full_gradient_entrywise():
    """Every entry of Abar against a one-entry central difference on a 4 x 3 input."""
    rng = np.random.default_rng(62)
    A = rng.standard_normal((4, 3)) * 2
    s = np.linalg.svd(A, compute_uv=False)
    tau = 0.5 * (s[0] + s[1])
    Xbar = rng.standard_normal((4, 3))
    Abar, _ = svt.svt_vjp(A, tau, Xbar)
    h = 1e-6
    for i in range(4):
        for j in range(3):
            E = np.zeros((4, 3))
            E[i, j] = 1.0
            fd = np.sum(Xbar * (svt.exact_svt(A + h * E, tau)[0] - svt.exact_svt(A - h * E, tau)[0])) / (2 * h)
            assert abs(Abar[i, j] - fd) < 1e-6


def test_svt_vjp_tau_zero_is_identity_map():
    """tau = 0 (all sigma > 0): X = A, so Abar = Xbar and taubar = -trace(U^T Xbar V)."""
    rng = np.random.default_rng(63)
    A = rng.standard_normal((6, 4))
    Xbar = rng.standard_normal((6, 4))
    Abar, taubar = svt.svt_vjp(A, 0.0, Xbar)
    assert np.allclose(Abar, Xbar, atol=1e-12)
    U, s, Vt = np.linalg.svd(A, full_matrices=False)
    assert abs(taubar + np.trace(U.T @ Xbar @ Vt.T)) < 1e-12


def _residual_problem(ns, nl, spectrum, k, seed):
    """Ah = U diag(spectrum) V^T (ns x nl) and Q = U[:, :k]: (I - Q Q^T) Ah has the spectrum[k:] tail."""
    rng = np.random.default_rng(seed)
    U, _ = np.linalg.qr(rng.standard_normal((ns, len(spectrum))))
    V, _ = np.linalg.qr(rng.standard_normal((nl, len(spectrum))))
    return (U * np.asarray(spectrum, dtype=np.float64)) @ V.T, U[:, :k]


def test_prop4_rank_one_residual_failure_rate():
    """Prop. 4 with a rank-one residual sigma u v^T: ||(I - QQ^T) A omega|| = sigma |g|, g ~ N(0, 1), so the
    bound alpha sqrt(2/pi) sigma |g| >= sigma fails exactly when |g| < c = 1 / (alpha sqrt(2/pi)),
    with probability erf(c / sqrt(2)).  At alpha = 2 that is 0.469 (0.383 without the sqrt(2/pi) factor,
    0.683 with 1 / alpha dropped), so the count over 4000 draws pins the constant."""
    from scipy.special import erf
    Ah, Q = _residual_problem(30, 200, [9.0, 4.0, 2.5], 2, seed=401)
    tail = 2.5                                        # ||(I - QQ^T) Ah||_2
    assert np.linalg.norm(Ah - Q @ (Q.T @ Ah), 2) == pytest.approx(tail, rel=1e-12)
    rng = np.random.default_rng(402)
    N, alpha = 4000, 2.0
    fails = sum(svt.residual_estimate(Q, Ah @ rng.standard_normal(200), alpha) < tail for _ in range(N))
    p = erf(1.0 / (alpha * np.sqrt(2.0 / np.pi)) / np.sqrt(2.0))
    assert p == pytest.approx(0.469, abs=1e-3)
    assert abs(fails - N * p) <= 4.0 * np.sqrt(N * p * (1 - p)), (fails, N * p)


def test_prop4_mean_residual_and_guarantee():
    """E ||(I - QQ^T) A omega|| = sqrt(2/pi) sigma for a rank-one residual (E|g| = sqrt(2/pi)); with a
    rank-three residual the alpha = 20 bound holds in at least 1 - 1/alpha = 95 % of the draws."""
    Ah, Q = _residual_problem(30, 200, [9.0, 4.0, 2.5], 2, seed=403)
    rng = np.random.default_rng(404)
    r = np.array([svt.residual_norm(Q, Ah @ rng.standard_normal(200)) for _ in range(4000)])
    se = 2.5 * np.sqrt(1.0 - 2.0 / np.pi) / np.sqrt(r.size)
    assert abs(r.mean() - 2.5 * np.sqrt(2.0 / np.pi)) <= 4.0 * se
    Ah3, Q3 = _residual_problem(30, 200, [9.0, 4.0, 1.0, 0.8, 0.5], 2, seed=405)
    bound = np.linalg.norm(Ah3 - Q3 @ (Q3.T @ Ah3), 2)
    assert bound == pytest.approx(1.0, rel=1e-12)
    ok = np.mean([svt.residual_estimate(Q3, Ah3 @ rng.standard_normal(200), 20.0) >= bound for _ in range(2000)])
    assert ok >= 0.95


def test_prop4_zero_residual_when_basis_spans_range():
    """rank(A) <= k and Q = the leading left singular vectors: the residual vanishes, so does the estimate."""
    Ah, Q = _residual_problem(30, 200, [9.0, 4.0, 2.5], 3, seed=406)
    y = Ah @ np.random.default_rng(407).standard_normal(200)
    assert svt.residual_estimate(Q, y) <= 1e-13 * np.linalg.norm(y)


def test_frsvt_reports_prop4_residual_of_first_new_column():
    """Under range propagation frsvt reports ||(I - Q~ Q~^T) A^T omega_0|| for the first new Omega column
    (short side = columns of a tall A); without a propagated basis it reports -1.  A propagated basis
    that spans the whole row space leaves no residual."""
    rng = np.random.default_rng(408)
    m, n, l = 300, 40, 10
    U, _ = np.linalg.qr(rng.standard_normal((m, 6)))
    V, _ = np.linalg.qr(rng.standard_normal((n, 6)))
    s = np.array([50.0, 30.0, 20.0, 12.0, 3.0, 1.0])
    A = (U * s) @ V.T + 1e-3 * rng.standard_normal((m, n))
    first = svt.frsvt(A, 2.0, l, 1, seed=5, stream=0)
    assert first.extra["rp_residual"] == -1.0
    Qp = first.Q_tilde
    assert Qp.shape[1] == 5                                     # min(r, l - 2) with r = #{sigma > 2} = 5
    second = svt.frsvt(A, 2.0, l, 1, seed=5, stream=1, Q_prev=Qp)
    omega0 = gaussian_matrix(m, l - Qp.shape[1], 5, 1, 0)[:, 0]
    y = A.T @ omega0
    direct = np.linalg.norm(y - Qp @ np.linalg.lstsq(Qp, y, rcond=None)[0])
    assert second.extra["rp_residual"] == pytest.approx(direct, rel=1e-10)
    # the residual is what the five kept directions miss: sigma_6 and the noise
    assert 0.5 < second.extra["rp_residual"] / np.linalg.norm(y - V[:, :5] @ (V[:, :5].T @ y)) < 2.0
    low = (U[:, :3] * s[:3]) @ V[:, :3].T
    f1 = svt.frsvt(low, 2.0, l, 1, seed=5, stream=0)
    f2 = svt.frsvt(low, 2.0, l, 1, seed=5, stream=1, Q_prev=f1.Q_tilde)
    assert f1.Q_tilde.shape[1] == 3 and f2.extra["rp_residual"] <= 1e-12 * np.linalg.norm(low)


@pytest.mark.parametrize("q", [2, 3])
def test_frsvt_orth_last_same_result(q):
    """Sec. 2.5: skipping the orthonormalisation of the intermediate power steps leaves span(Q), hence X,
    unchanged in exact arithmetic; in FP64 on a moderately conditioned spectrum the two agree to 1e-9.
    The basis handed to the core is still orthonormal (the last step keeps its QR)."""
    rng = np.random.default_rng(501)
    m, n, l = 400, 60, 12
    U, _ = np.linalg.qr(rng.standard_normal((m, n)))
    V, _ = np.linalg.qr(rng.standard_normal((n, n)))
    s = 10.0 * 0.8 ** np.arange(n)
    A = (U * s) @ V.T
    tau = float(0.5 * (s[5] + s[6]))
    ref = svt.frsvt(A, tau, l, q, seed=3, stream=0)
    alt = svt.frsvt(A, tau, l, q, seed=3, stream=0, orth_last=True)
    assert alt.r == ref.r
    assert np.linalg.norm(alt.X - ref.X) <= 1e-9 * np.linalg.norm(ref.X)
    QV = alt.extra["QV"]
    assert np.abs(QV.T @ QV - np.eye(QV.shape[1])).max() <= 1e-12
    # with range propagation as well
    ref2 = svt.frsvt(A, tau, l, q, seed=3, stream=1, Q_prev=ref.Q_tilde)
    alt2 = svt.frsvt(A, tau, l, q, seed=3, stream=1, Q_prev=ref.Q_tilde, orth_last=True)
    assert np.linalg.norm(alt2.X - ref2.X) <= 1e-9 * np.linalg.norm(ref2.X)


def test_frsvt_orth_last_q1_identical():
    """q = 1 has no intermediate power step: the option changes nothing."""
    rng = np.random.default_rng(502)
    A = rng.standard_normal((120, 40))
    a = svt.frsvt(A, 1.0, 8, 1, seed=4, stream=0)
    b = svt.frsvt(A, 1.0, 8, 1, seed=4, stream=0, orth_last=True)
    assert np.array_equal(a.X, b.X)


# ---------------------------------------------------------------- FRSVT-map adjoint

def _frsvt_tau(A, l, q, seed, stream):
    """tau halfway across the widest gap among the leading singular values of FRSVT's B."""
    d = svt.frsvt(A, 0.0, l, q, seed, stream).sigma
    gaps = d[:-1] - d[1:]
    i = int(np.argmax(gaps[: max(1, len(gaps) - 1)]))
    return float(0.5 * (d[i] + d[i + 1]))


@pytest.mark.parametrize("shape,l,q", [((9, 6), 3, 0), ((9, 6), 3, 1), ((11, 7), 4, 2), ((6, 10), 3, 1),
                                       ((8, 8), 5, 2)])
def test_frsvt_vjp_entrywise_central_differences(shape, l, q):
    """Every entry of Abar and taubar of the FRSVT-map adjoint against one-entry central differences
    of the oracle's Alg. 1 (pivoted QR, Newton polar and Jacobi route) with the same Omega."""
    rng = np.random.default_rng(71 + shape[0] + q)
    m, n = shape
    A = rng.standard_normal((m, n)) * 2.0
    seed, stream = 13, 4
    tau = _frsvt_tau(A, l, q, seed, stream)
    Xbar = rng.standard_normal((m, n))
    Abar, taubar, X = svt.frsvt_vjp(A, tau, l, q, seed, stream, Xbar)
    assert np.linalg.norm(X - svt.frsvt(A, tau, l, q, seed, stream).X) < 1e-12 * np.linalg.norm(A)
    h = 1e-6
    fd = np.empty((m, n))
    for i in range(m):
        for j in range(n):
            E = np.zeros((m, n))
            E[i, j] = h
            fd[i, j] = np.sum(Xbar * (svt.frsvt(A + E, tau, l, q, seed, stream).X
                                      - svt.frsvt(A - E, tau, l, q, seed, stream).X)) / (2 * h)
    assert np.max(np.abs(Abar - fd)) < 1e-6 * max(1.0, np.max(np.abs(fd)))
    fdt = np.sum(Xbar * (svt.frsvt(A, tau + h, l, q, seed, stream).X
                         - svt.frsvt(A, tau - h, l, q, seed, stream).X)) / (2 * h)
    assert abs(taubar - fdt) < 1e-6 * max(1.0, abs(fdt))


@pytest.mark.parametrize("shape,q", [((9, 5), 0), ((9, 5), 2), ((5, 8), 1)])
def test_frsvt_vjp_full_basis_is_exact_svt_adjoint(shape, q):
    """With l = min(m, n) the basis spans the short side, FRSVT is the exact SVT, and the FRSVT-map
    adjoint reduces to the divided-difference adjoint of the exact SVT (every QR adjoint cancels)."""
    rng = np.random.default_rng(81 + q)
    A = rng.standard_normal(shape)
    s = np.linalg.svd(A, compute_uv=False)
    tau = 0.5 * (s[1] + s[2])
    Xbar = rng.standard_normal(shape)
    Abar, taubar, _ = svt.frsvt_vjp(A, tau, min(shape), q, 3, 1, Xbar)
    Ae, te = svt.svt_vjp(A, tau, Xbar)
    assert np.max(np.abs(Abar - Ae)) < 1e-10 * max(1.0, np.max(np.abs(Ae)))
    assert abs(taubar - te) < 1e-10 * max(1.0, abs(te))
