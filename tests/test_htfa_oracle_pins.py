"""Pins of the HTFA oracle (oracle/htfa.py) to facts that do not come from
the oracle itself.

Factor matrix (Eq. 14, F[k, v] = exp(-||p_v - mu_k||^2 / lambda_k)):
* closed forms: 1 at the center; e^-1 at distance sqrt(lambda) along any
  axis; exp(-3 s^2 / lambda) on the diagonal;
* the Gaussian integral: over a fine grid, sum F * cell volume equals
  (pi lambda)^(3/2).  A wrong width scaling (lambda^2, 2 lambda), a dropped
  axis or a wrong sign fails it;
* separability: F(p) = F(p_x, mu_y, mu_z) F(mu_x, p_y, mu_z) F(mu_x, mu_y, p_z),
  an identity of the exponential, not of the code;
* rejection of non-positive widths.

Residual (Frobenius term of eq:htfa_subject_update_rbfs):
* a hand-worked integer example;
* zero when X = W F; ||X||^2 when W = 0;
* exact rational arithmetic (fractions) on small integer matrices through
  the trace expansion ||X||^2 - 2 tr(W^T X F^T) + tr(W^T W F F^T);
* the least-squares optimum: with W = X F^+ the residual is
  ||X||^2 - ||X F^+ F||^2 (Pythagoras).

z-score (Sec. IV-A): equal to scipy.stats.zscore (ddof 0) on non-constant
columns; mean 0 and unit population variance; invariance under x -> a x + b
(a > 0); a constant column becomes zeros (reading of the paper's silence).
"""
import math
from fractions import Fraction

import numpy as np
import pytest

import oracle


def test_factor_closed_forms():
    mu = np.array([[1.0, -2.0, 0.5], [10.0, 3.0, -4.0]])
    lam = np.array([2.0, 7.5])
    s = 0.9
    pts = [mu[0], mu[1],
           mu[0] + [math.sqrt(lam[0]), 0, 0], mu[1] + [0, -math.sqrt(lam[1]), 0], mu[1] + [0, 0, math.sqrt(lam[1])],
           mu[0] + [s, s, s]]
    F = oracle.rbf_factors(np.array(pts), mu, lam)
    assert F[0, 0] == 1.0 and F[1, 1] == 1.0
    assert F[0, 2] == pytest.approx(math.exp(-1.0), rel=1e-14)
    assert F[1, 3] == pytest.approx(math.exp(-1.0), rel=1e-14)
    assert F[1, 4] == pytest.approx(math.exp(-1.0), rel=1e-14)
    assert F[0, 5] == pytest.approx(math.exp(-3 * s * s / lam[0]), rel=1e-14)
    # symmetric about the center and decreasing with distance
    d = np.linspace(0, 6, 25)[:, None] * np.array([[0.3, -0.5, 0.8]])
    fp = oracle.rbf_factors(mu[0] + d, mu[:1], lam[:1])[0]
    fm = oracle.rbf_factors(mu[0] - d, mu[:1], lam[:1])[0]
    np.testing.assert_allclose(fp, fm, rtol=1e-13)
    assert np.all(np.diff(fp) < 0)


@pytest.mark.parametrize("lam", [0.7, 4.0, 19.0])
def test_factor_gaussian_integral(lam):
    h = 0.1 * math.sqrt(lam)
    r = 7.0 * math.sqrt(lam)
    ax = np.arange(-r, r + h / 2, h)
    g = np.stack(np.meshgrid(ax, ax, ax, indexing="ij"), axis=-1).reshape(-1, 3)
    mu = np.array([[0.013, -0.021, 0.007]])
    F = oracle.rbf_factors(g, mu, np.array([lam]))
    total = F.sum() * h ** 3
    assert total == pytest.approx((math.pi * lam) ** 1.5, rel=1e-6)


def test_factor_separability():
    rng = np.random.default_rng(3)
    mu = rng.uniform(-5, 5, (4, 3))
    lam = rng.uniform(1, 20, 4)
    p = rng.uniform(-8, 8, (30, 3))
    F = oracle.rbf_factors(p, mu, lam)
    for k in range(4):
        prod = np.ones(30)
        for a in range(3):
            q = np.tile(mu[k], (30, 1))
            q[:, a] = p[:, a]
            prod *= oracle.rbf_factors(q, mu[k:k + 1], lam[k:k + 1])[0]
        np.testing.assert_allclose(F[k], prod, rtol=1e-13)


@pytest.mark.parametrize("bad", [0.0, -1.0, float("nan")])
def test_factor_rejects_bad_width(bad):
    with pytest.raises(ValueError):
        oracle.rbf_factors(np.zeros((2, 3)), np.zeros((1, 3)), np.array([bad]))


def test_residual_hand_example():
    X = np.array([[1.0, 2.0], [3.0, 4.0]])
    W = np.array([[1.0], [0.0]])
    F = np.array([[1.0, 1.0]])
    # X - W F = [[0, 1], [3, 4]] -> 0 + 1 + 9 + 16
    assert oracle.htfa_residual(X, W, F) == 26.0


def test_residual_special_cases():
    rng = np.random.default_rng(4)
    W = rng.standard_normal((9, 3))
    F = rng.standard_normal((3, 11))
    assert oracle.htfa_residual(W @ F, W, F) == pytest.approx(0.0, abs=1e-20)
    X = rng.standard_normal((9, 11))
    assert oracle.htfa_residual(X, np.zeros((9, 3)), F) == pytest.approx(float(np.sum(X * X)), rel=1e-15)


def test_residual_exact_rational_trace_form():
    rng = np.random.default_rng(5)
    T, K, V = 5, 3, 7
    X = rng.integers(-9, 10, (T, V))
    W = rng.integers(-4, 5, (T, K))
    F = rng.integers(-3, 4, (K, V))
    Xf = [[Fraction(int(x)) for x in row] for row in X]
    Wf = [[Fraction(int(x)) for x in row] for row in W]
    Ff = [[Fraction(int(x)) for x in row] for row in F]
    xx = sum(x * x for row in Xf for x in row)
    XFt = [[sum(Xf[t][v] * Ff[k][v] for v in range(V)) for k in range(K)] for t in range(T)]
    cross = sum(Wf[t][k] * XFt[t][k] for t in range(T) for k in range(K))
    WtW = [[sum(Wf[t][a] * Wf[t][b] for t in range(T)) for b in range(K)] for a in range(K)]
    FFt = [[sum(Ff[a][v] * Ff[b][v] for v in range(V)) for b in range(K)] for a in range(K)]
    quad = sum(WtW[a][b] * FFt[a][b] for a in range(K) for b in range(K))
    exact = xx - 2 * cross + quad
    assert oracle.htfa_residual(X, W, F) == float(exact)


def test_residual_least_squares_pythagoras():
    rng = np.random.default_rng(6)
    X = rng.standard_normal((20, 40))
    F = rng.standard_normal((6, 40))
    W = X @ np.linalg.pinv(F)
    P = W @ F
    assert oracle.htfa_residual(X, W, F) == pytest.approx(float(np.sum(X * X) - np.sum(P * P)), rel=1e-10)


def test_zscore_matches_scipy_and_invariants():
    stats = pytest.importorskip("scipy.stats")
    rng = np.random.default_rng(7)
    X = rng.normal(5.0, 2.0, (37, 13)) * rng.uniform(0.1, 10, 13)
    Z = oracle.zscore(X)
    np.testing.assert_allclose(Z, stats.zscore(X, axis=0, ddof=0), rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(Z.mean(axis=0), 0, atol=1e-13)
    np.testing.assert_allclose((Z * Z).mean(axis=0), 1, rtol=1e-12)
    np.testing.assert_allclose(oracle.zscore(3.5 * X - 11.0), Z, rtol=1e-10, atol=1e-11)


def test_zscore_constant_column_is_zero():
    X = np.ones((6, 3))
    X[:, 1] = np.arange(6)
    X[:, 2] = 0.1
    Z = oracle.zscore(X)
    np.testing.assert_array_equal(Z[:, 0], 0)
    np.testing.assert_array_equal(Z[:, 2], 0)
    assert Z[:, 1].std() == pytest.approx(1.0)


def test_input_recipe_follows_the_subsampling_rule():
    """The local step's subsample (Sec. V-A): the mean of 25 % of the voxels
    and 3000, and of 10 % of the TRs and 300.  Greeneyes (42,855 voxels,
    475 TRs): (10,713.75 + 3000) / 2 and (47.5 + 300) / 2."""
    import synth.htfa_inputs as hi
    assert hi.subsample_counts(42855, 475) == (6857, 174)
    spec = hi.HTFA_CONFIGS["greeneyes-subsampled-like"]
    assert (spec.n_subjects, spec.V, spec.T, spec.K) == (40, 6857, 174, 100)
    d = hi.draw(hi.HTFA_CONFIGS["ragged-small"])
    mask = {tuple(r) for r in hi.brain_mask(hi.HTFA_CONFIGS["ragged-small"].brain_voxels)}
    assert all(tuple(r) in mask for r in d["vox"].reshape(-1, 3))        # voxels inside the brain
    assert d["lam"].min() >= 0.04 * d["diameter"] and d["lam"].max() <= 1.8 * d["diameter"]
    # positions are read off the axes by the indices
    for a in range(3):
        np.testing.assert_array_equal(d["positions"][..., a], d["axes"][a][d["vox"][..., a]])
