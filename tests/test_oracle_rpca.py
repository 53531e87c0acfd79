"""Pins of the oracle's inexact-ALM RPCA host loop (Sec. 4.1 Robust PCA test, Table 5)."""
import numpy as np
import pytest

from oracle import rpca
from paper_1509_00296_gb300 import synth


def _small_problem():
    O, L, S = synth.lowrank_sparse(90, 70, 3, 0.05, 10.0, seed=31)
    return O, L, S


def test_ialm_exact_recovers_planted_lowrank_sparse():
    O, L, S = _small_problem()
    res = rpca.ialm_rpca(O, method="exact", tol=1e-7)
    assert res.history[-1] < 1e-7
    assert np.linalg.norm(res.L - L) / np.linalg.norm(L) < 1e-5
    assert np.sum(np.abs(res.S) > 1e-6) == pytest.approx(np.count_nonzero(S), rel=0.02)
    # dual feasibility of the ALM iterate: ||Y||_2 <= 1 + eps, ||Y||_inf <= lambda + eps
    lam = 1 / np.sqrt(90)
    assert np.max(np.abs(res.Y)) <= lam * (1 + 1e-6)


def test_ialm_frsvt_rp_matches_exact_iterations_and_solution():
    """Table 5: FRSVT-RP takes the same number of iALM iterations and reaches the same accuracy."""
    O, L, S = _small_problem()
    ex = rpca.ialm_rpca(O, method="exact", tol=1e-7)
    fr = rpca.ialm_rpca(O, method="frsvt", l=12, q=2, seed=5, range_prop=True, tol=1e-7)
    assert fr.iters == ex.iters
    assert np.linalg.norm(fr.L - ex.L) / np.linalg.norm(ex.L) < 1e-6
    assert fr.ranks[-1] == ex.ranks[-1] == 3


def test_ialm_frsvt_rpca_300():
    """300 x 300, rank 10, 5 % corruption, l = 20, q = 1, 30 iterations (RPCA 300 x 300 workload)."""
    O, L, S = synth.rpca_300()
    res = rpca.ialm_rpca(O, method="frsvt", l=20, q=1, seed=2001, fixed_iters=30)
    assert np.linalg.norm(res.L - L) / np.linalg.norm(L) < 1e-5
    assert res.ranks[-1] == 10
    assert np.all(np.diff(res.history[10:]) < 0) or res.history[-1] < 1e-7


def test_ialm_init_constants():
    O, _, _ = _small_problem()
    lam = 1 / np.sqrt(90)
    Y0, mu0 = rpca.ialm_init(O, lam)
    s1 = np.linalg.norm(O, 2)
    assert mu0 == pytest.approx(1.25 / s1, rel=1e-12)
    J = max(np.linalg.norm(Y0, 2), np.max(np.abs(Y0)) / lam)
    assert J == pytest.approx(1.0, rel=1e-12)


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_ialm_adaptive_rank_prediction_matches_exact():
    """Adaptive rank prediction (Sec. 2.3, Eq. 7) with range propagation, p = +2 (the Table 4/5
    setting): the same number of iALM iterations and the same solution as exact SVT (Table 5);
    the sampling rate starts at ceil(0.1 b) and settles just above the rank."""
    O, L, _ = synth.lowrank_sparse(150, 120, 6, 0.05, 10.0, seed=33)
    ex = rpca.ialm_rpca(O, method="exact", tol=1e-7)
    fr = rpca.ialm_rpca(O, method="frsvt", q=1, seed=3, tol=1e-7, ap=dict(a=2, rho=0.05, gamma=0.2))
    assert fr.iters == ex.iters
    assert _rel(fr.L, ex.L) < 1e-6
    assert fr.ranks[-1] == ex.ranks[-1] == 6
    assert fr.ls[0] == 3                        # b = ceil(0.2 * 120) = 24, l_0 = ceil(0.1 b)
    assert fr.ls[-1] == fr.ranks[-1] + 2        # r < l: over-sample by a once the rank is found
    O3, L3, _ = synth.rpca_300()
    fr3 = rpca.ialm_rpca(O3, method="frsvt", q=1, seed=2001, tol=1e-7, ap=dict(a=2, rho=0.05, gamma=0.1))
    assert _rel(fr3.L, L3) < 1e-5
    assert fr3.ls[:3] == [3, 18, 12]            # r_0 = l_0 = 3: + ceil(0.05 * 300); then r = 10 < 18: + 2


def test_fixed_small_sampling_rate_needs_prediction():
    """Sec. 4.1 (Fig. 7 discussion): with a fixed small over-sampled rank iALM-FRSVT does not reach
    the ground truth, while the same start under Eq. 7 does."""
    O, L, _ = synth.rpca_300()
    fixed = rpca.ialm_rpca(O, method="frsvt", l=5, q=1, seed=2001, fixed_iters=40)
    ap = rpca.ialm_rpca(O, method="frsvt", q=1, seed=2001, fixed_iters=40, ap=dict(a=2, rho=0.05, gamma=0.1))
    assert _rel(fixed.L, L) > 1e-2
    assert _rel(ap.L, L) < 1e-5
