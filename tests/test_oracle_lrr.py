"""Pins of the low-rank-representation oracle (Table 6, Type A) on synthetic union-of-subspaces data."""
import numpy as np
import pytest

from oracle import lrr
from paper_1509_00296_gb300 import synth


def test_colshrink_is_the_l21_proximal_map():
    """colshrink_t(Q) minimises t ||S||_{2,1} + 1/2 ||S - Q||_F^2: its KKT conditions hold column by column
    (q_i - s_i = t s_i / ||s_i|| where s_i != 0, ||q_i|| <= t where s_i = 0), and random perturbations
    never lower the objective."""
    rng = np.random.default_rng(601)
    Q = rng.standard_normal((5, 6)) * np.array([0.2, 0.5, 1.0, 2.0, 3.0, 0.05])
    t = 0.8
    S = lrr.colshrink(Q, t)
    for i in range(Q.shape[1]):
        si, qi = S[:, i], Q[:, i]
        if np.linalg.norm(si) > 0:
            assert np.allclose(qi - si, t * si / np.linalg.norm(si), atol=1e-12)
        else:
            assert np.linalg.norm(qi) <= t
    f = lambda X: t * lrr.l21(X) + 0.5 * np.sum((X - Q) ** 2)
    f0 = f(S)
    for _ in range(200):
        assert f(S + 1e-3 * rng.standard_normal(S.shape)) >= f0 - 1e-12


@pytest.fixture(scope="module")
def clean_data():
    O, clean, labels, mask = synth.subspaces(seed=1007)
    return clean, labels


def test_lrr_noiseless_solution_is_the_shape_interaction_matrix(clean_data):
    """Without corruption and with a large lam the problem becomes min ||L||_* s.t. O = O L, whose solution
    is V V^T for the skinny SVD O = U S V^T (rank r = 4 subspaces x 3 dimensions)."""
    O, labels = clean_data
    r = lrr.lrr_ialm(O, 10.0, rho=1.2)
    U, s, Vt = np.linalg.svd(O, full_matrices=False)
    k = int(np.sum(s > 1e-10 * s[0]))
    assert k == 12
    VVt = Vt[:k].T @ Vt[:k]
    assert np.linalg.norm(r.L - VVt) <= 1e-6 * np.linalg.norm(VVt)
    assert np.abs(r.S).max() <= 1e-8


def test_lrr_block_diagonal_for_independent_subspaces(clean_data):
    """L links only columns of the same subspace: the entries between different subspaces vanish."""
    O, labels = clean_data
    r = lrr.lrr_ialm(O, 10.0, rho=1.2)
    same = labels[:, None] == labels[None, :]
    assert np.abs(r.L[~same]).max() <= 1e-6 * np.abs(r.L).max()
    assert np.abs(r.L[same]).max() > 0.1


@pytest.fixture(scope="module")
def corrupted_run():
    O, clean, labels, mask = synth.subspaces(seed=1007)
    return O, mask, lrr.lrr_ialm(O, 0.25, rho=1.2)


def ladmap(O, lam, iters=4000, mu=1e-2, rho=1.05, mu_max=1e3):
    """A second, independent solver of the same problem: linearised ADMM with two blocks (L by a
    linearised SVT step with eta > ||O||_2^2, S by the l2,1 proximal map), which converges for any
    bounded penalty.  Only numpy's SVD and the proximal map are shared with the oracle."""
    eta = 1.01 * np.linalg.norm(O, 2) ** 2
    L = np.zeros((O.shape[1], O.shape[1]))
    S = np.zeros_like(O)
    Y = np.zeros_like(O)
    for _ in range(iters):
        G = L + O.T @ (O - O @ L - S + Y / mu) / eta
        U, sg, Vt = np.linalg.svd(G, full_matrices=False)
        L = (U * np.maximum(sg - 1.0 / (mu * eta), 0.0)) @ Vt
        S = lrr.colshrink(O - O @ L + Y / mu, lam / mu)
        Y = Y + mu * (O - O @ L - S)
        mu = min(rho * mu, mu_max)
    return L, S


def test_lrr_s_step_optimality(corrupted_run):
    """The returned point is feasible (O = Z L + S, L = J) and satisfies the S-step optimality exactly:
    Y1 lies in lam times the l2,1 subdifferential at S (y_i = lam s_i / ||s_i|| on the non-zero columns,
    ||y_i|| <= lam on the others)."""
    O, mask, r = corrupted_run
    lam = 0.25
    assert np.linalg.norm(O - O @ r.L - r.S) <= 1e-7 * np.linalg.norm(O)
    assert np.abs(r.L - r.J).max() <= 1e-7
    for i in range(O.shape[1]):
        si, yi = r.S[:, i], r.Y1[:, i]
        if np.linalg.norm(si) > 1e-9:
            assert np.allclose(yi, lam * si / np.linalg.norm(si), atol=1e-6 * lam)
        else:
            assert np.linalg.norm(yi) <= lam * (1 + 1e-6)


def test_lrr_reaches_the_optimum_of_an_independent_solver():
    """With a slowly growing penalty (rho = 1.02) the iALM point attains the optimal value
    ||L||_* + lam ||S||_{2,1} that a two-block linearised ADMM converges to (2e-5 relative; a fast
    growth such as rho = 1.2 freezes the iterate at a feasible point ~2e-3 above the optimum)."""
    O, clean, labels, mask = synth.subspaces(seed=1009, d=40, k=3, dim=2, per=10, frac=0.1)
    lam = 0.3
    f = lambda L, S: np.linalg.svd(L, compute_uv=False).sum() + lam * lrr.l21(S)
    r = lrr.lrr_ialm(O, lam, rho=1.02, max_iter=5000)
    La, Sa = ladmap(O, lam, iters=20000)
    assert np.linalg.norm(O - O @ La - Sa) <= 1e-6 * np.linalg.norm(O)
    assert np.linalg.norm(O - O @ r.L - r.S) <= 1e-7 * np.linalg.norm(O)
    assert abs(f(r.L, r.S) - f(La, Sa)) <= 2e-5 * f(La, Sa)


def test_lrr_error_columns_are_the_corrupted_samples(corrupted_run):
    """The corrupted samples carry the largest columns of S, with a clear gap to the clean ones."""
    O, mask, r = corrupted_run
    sn = np.linalg.norm(r.S, axis=0)
    top = np.argsort(-sn)[:int(mask.sum())]
    assert set(top.tolist()) == set(np.flatnonzero(mask).tolist())
    assert sn[mask].min() > 2.0 * sn[~mask].max()


def test_lrr_frsvt_full_basis_reproduces_exact_svt():
    """With a full basis (l = n) FRSVT is exact (Sec. 3.1), so the iALM iterates coincide with the exact-SVT
    run; with range propagation and l = 24 the fixed point is the same optimum."""
    O, clean, labels, mask = synth.subspaces(seed=1008, d=40, k=3, dim=2, per=10, frac=0.1)
    ref = lrr.lrr_ialm(O, 0.3, rho=1.3)
    full = lrr.lrr_ialm(O, 0.3, rho=1.3, method="frsvt", l=O.shape[1], q=1, seed=9, range_prop=False)
    assert full.iters == ref.iters
    assert np.linalg.norm(full.L - ref.L) <= 1e-8 * np.linalg.norm(ref.L)
    part = lrr.lrr_ialm(O, 0.3, rho=1.3, method="frsvt", l=12, q=2, seed=9)
    assert np.linalg.norm(part.L - ref.L) <= 1e-5 * np.linalg.norm(ref.L)
    assert np.linalg.norm(part.S - ref.S) <= 1e-5 * max(np.linalg.norm(ref.S), 1e-12)
