"""Pins of the oracle's Omega generator (Alg. 1 step 4; Sec. 2.4 dense Gaussian Omega)."""
import numpy as np
import pytest
import scipy.stats

from oracle import philox


def _numpy_philox(counter, key):
    """numpy.random.Philox increments its 256-bit counter before each block."""
    c = np.array(counter, dtype=np.uint64).copy()
    for w in range(4):                      # subtract one with borrow
        if c[w] > 0:
            c[w] -= np.uint64(1)
            break
        c[w] = np.uint64(2**64 - 1)
    return np.random.Philox(counter=c, key=np.array(key, dtype=np.uint64)).random_raw(4)


@pytest.mark.parametrize("trial", range(8))
def test_philox_matches_numpy_library(trial):
    rng = np.random.default_rng(100 + trial)
    ctr = rng.integers(0, 2**63, size=4, dtype=np.uint64) * np.uint64(2) + np.uint64(trial % 2)
    key = rng.integers(0, 2**63, size=2, dtype=np.uint64) * np.uint64(3)
    assert np.array_equal(philox.philox4x64_10(ctr, key), _numpy_philox(ctr, key))


def test_philox_counter_edges_match_numpy():
    for ctr in ([0, 0, 0, 0], [1, 0, 0, 0], [0, 1, 0, 0], [2**64 - 1, 5, 0, 9], [7, 2**64 - 1, 2**64 - 1, 3]):
        for key in ([0, 0], [2**64 - 1, 2**64 - 1], [12345, 0]):
            assert np.array_equal(philox.philox4x64_10(np.array(ctr, dtype=np.uint64), key),
                                  _numpy_philox(ctr, key))


def test_philox_vectorized_equals_scalar():
    words = philox.philox_words(5, 9, seed=42, stream=3, problem=2)
    for i in range(5):
        for j in range(3):
            ref = philox.philox4x64_10(np.array([i, j, 3, 2], dtype=np.uint64), [42, 0])
            assert np.array_equal(words[i, j], ref)


def test_uniform23_closed_form():
    x = np.array([0, 2**64 - 1, 1 << 41, (1 << 63)], dtype=np.uint64)
    u = philox.uniform23(x)
    assert u[0] == 2.0 ** -24
    assert u[1] == 1.0 - 2.0 ** -24
    assert u[2] == 1.5 * 2.0 ** -23
    assert u[3] == 0.5 + 2.0 ** -24
    assert np.all((u > 0) & (u < 1))
    assert np.all(u.astype(np.float32).astype(np.float64) == u)   # exact in float32


def test_box_muller_closed_form():
    z0, z1 = philox.box_muller(np.array([np.exp(-0.5)]), np.array([0.25]))
    assert abs(z0[0]) < 1e-15 and abs(z1[0] - 1.0) < 1e-15
    z0, z1 = philox.box_muller(np.array([np.exp(-2.0)]), np.array([0.5]))
    assert abs(z0[0] + 2.0) < 1e-15 and abs(z1[0]) < 1e-15


def test_gaussian_matrix_statistics():
    Z = philox.gaussian_matrix(40000, 8, seed=7, stream=11)
    x = Z.ravel()
    assert abs(x.mean()) < 4.0 / np.sqrt(x.size)
    assert abs(x.var() - 1.0) < 6.0 * np.sqrt(2.0 / x.size)
    assert scipy.stats.kstest(x, "norm").pvalue > 1e-3
    C = np.corrcoef(Z.T)
    assert np.max(np.abs(C - np.eye(8))) < 5.0 / np.sqrt(Z.shape[0])


def test_gaussian_matrix_streams_and_prefix():
    A = philox.gaussian_matrix(100, 10, seed=1, stream=0)
    B = philox.gaussian_matrix(100, 3, seed=1, stream=0)
    assert np.array_equal(A[:, :3], B)                      # column prefix: Omega_p of range propagation
    C = philox.gaussian_matrix(100, 10, seed=1, stream=1)
    D = philox.gaussian_matrix(100, 10, seed=2, stream=0)
    E = philox.gaussian_matrix(100, 10, seed=1, stream=0, problem=1)
    for other in (C, D, E):
        assert abs(np.corrcoef(A.ravel(), other.ravel())[0, 1]) < 0.1
    assert philox.gaussian_matrix(0, 4, 1, 0).shape == (0, 4)
