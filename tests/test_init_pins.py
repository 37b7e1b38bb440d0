"""Pins of the oracle's seeded random orthogonal W^0 (Algorithm 1's
initialisation, oracle/init.py), independent of the oracle's own code:

* its Philox4x64-10 equals NumPy's Philox bit generator, a library routine
  that implements the same published definition (NumPy advances the counter
  by one before its first block);
* the uniforms lie in (0, 1), and the Box-Muller normals have the moments and
  the distribution of N(0, 1) (Kolmogorov-Smirnov against scipy's normal
  CDF), with independent pairs;
* W^0 has orthonormal columns and is the Q of a QR of the normal matrix with
  a positive-diagonal R (W^T G upper triangular, positive diagonal), the
  only such Q, and its distribution is invariant: E[W W^T] = (k / v) I.
A planted mistake in the generator (a wrong multiplier, a dropped key
increment, a swapped output word) breaks the first pin; a wrong sign rule or
a transposed G breaks the third."""
import numpy as np
import pytest

from oracle.init import haar_w0, philox4x64_10, standard_normals, unit_open


@pytest.mark.parametrize("key,ctr", [((0, 0), (0, 0, 0, 0)), ((123, 456), (5, 7, 0, 0)),
                                     ((2 ** 64 - 1, 2 ** 63 + 11), (2 ** 64 - 2, 3, 2 ** 40, 9))])
def test_philox_matches_numpy(key, ctr):
    # NumPy adds one to the 256-bit counter (word 0 lowest) before its first block
    c = sum(int(x) << (64 * j) for j, x in enumerate(ctr))
    c = (c - 1) % 2 ** 256
    before = [(c >> (64 * j)) & (2 ** 64 - 1) for j in range(4)]
    bg = np.random.Philox(key=np.array(key, dtype=np.uint64), counter=np.array(before, dtype=np.uint64))
    ref = bg.random_raw(4)
    got = philox4x64_10([np.uint64(x) for x in ctr], key)
    assert [int(g) for g in got] == [int(r) for r in ref]


def test_philox_vectorised_matches_scalar():
    b = np.arange(50, dtype=np.uint64)
    got = philox4x64_10([b, np.full(50, 3, np.uint64), np.zeros(50, np.uint64), np.zeros(50, np.uint64)], (9, 0))
    for j in (0, 17, 49):
        one = philox4x64_10([np.uint64(j), np.uint64(3), np.uint64(0), np.uint64(0)], (9, 0))
        assert [int(g[j]) for g in got] == [int(x) for x in one]


def test_uniforms_and_normals():
    scipy_stats = pytest.importorskip("scipy.stats")
    w = np.array([0, 2 ** 64 - 1, 2 ** 11 - 1, 2 ** 11], dtype=np.uint64)
    u = unit_open(w)
    assert np.all((u > 0) & (u < 1))
    z = standard_normals(2024, 5, 200_000)
    assert abs(z.mean()) < 0.01 and abs(z.var() - 1) < 0.01
    assert abs(np.mean(z ** 3)) < 0.02 and abs(np.mean(z ** 4) - 3) < 0.05
    assert scipy_stats.kstest(z, "norm").pvalue > 1e-3
    zz = z.reshape(-1, 2)
    assert abs(np.corrcoef(zz[:, 0], zz[:, 1])[0, 1]) < 0.01
    # the subject index and the seed change the stream
    assert not np.allclose(standard_normals(2024, 6, 100), z[:100])
    assert not np.allclose(standard_normals(2025, 5, 100), z[:100])
    np.testing.assert_array_equal(standard_normals(2024, 5, 100), z[:100])


@pytest.mark.parametrize("v,k", [(7, 1), (40, 6), (300, 50), (64, 64)])
def test_haar_w0_is_the_positive_qr_factor(v, k):
    W = haar_w0(11, 2, v, k)
    G = standard_normals(11, 2, v * k).reshape(v, k)
    np.testing.assert_allclose(W.T @ W, np.eye(k), atol=1e-12)
    R = W.T @ G
    np.testing.assert_allclose(np.tril(R, -1), 0, atol=1e-10 * np.abs(R).max())
    assert np.all(np.diag(R) > 0)
    np.testing.assert_allclose(W @ R, G, atol=1e-10 * np.abs(G).max())


def test_haar_w0_is_rotation_invariant_in_mean():
    v, k, n = 6, 2, 4000
    acc = np.zeros((v, v))
    for s in range(n):
        W = haar_w0(s, 0, v, k)
        acc += W @ W.T
    np.testing.assert_allclose(acc / n, (k / v) * np.eye(v), atol=0.02)
