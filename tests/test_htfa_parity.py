"""Parity of the HTFA kernels (srm_htfa_factors, srm_htfa_residual,
srm_zscore) with the FP64 oracle, element by element, on the same seeded
FP32 inputs.

Every bar is an a-priori bound of the FP32 arithmetic, computed here from
the oracle's data (u = 2^-24, twice the bound for margin):

* factors: each axis's argument d^2 / lambda carries at most 4u relative
  error (one rounding each in the difference, square and division), which
  multiplies the factor by exp(4u a); three expf (at most 2 ulp each) and
  two products add 14u: |F - F_o| <= 2 (4 a + 14) u F_o + 2^-125, with
  a = ||p - mu||^2 / lambda.  The absolute term covers results below the
  FP32 normal range;
* residual: per element the product carries at most g (|W| |F|)_tv and
  the difference one more u |r|; squaring and summing 64 terms per thread
  add gamma_64 r^2:
  |R - R_o| <= 2 sum (2 |r| (u |r| + g (|W| |F|)_tv) + gamma_64 r^2).
  For K > 128 the FP32 FMA chain runs, g = gamma_K.  For K <= 128 the
  tensor cores form W F from three BF16 pieces of each operand, which leave
  at most 4 u |W| |F| (the pieces' remainders and three dropped products).
  Their FP32 accumulator rounds once per MMA, 6 ceil(K / 16) times, each
  allowed 2 u (a truncating rounding), so g = (4 + 12 ceil(K / 16)) u;
* z-score: the shifted sums over at most ceil(T/8) + 8 terms bound the
  error of the mean by (T/8 + 10) u max|x - x_0| and that of the variance
  likewise; the bound on z follows.
"""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
U = 2.0 ** -24


@pytest.fixture(scope="module", autouse=True)
def _build():
    from paper_1608_04647_gb300 import _build as b
    b.build()


def _cuda(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _factor_bound(pos, mu, lam, Fo):
    diff = pos[None, :, :].astype(np.float64) - mu[:, None, :].astype(np.float64)
    a = np.sum(diff * diff, axis=2) / lam.astype(np.float64)[:, None]
    return 2 * (4 * a + 14) * U * Fo + 2.0 ** -125


def _check_factors(d, F_gpu):
    import oracle
    worst = 0.0
    for i in range(F_gpu.shape[0]):
        Fo = oracle.rbf_factors(d["positions"][i], d["mu"][i], d["lam"][i])
        err = np.abs(F_gpu[i].astype(np.float64) - Fo)
        bound = _factor_bound(d["positions"][i], d["mu"][i], d["lam"][i], Fo)
        assert np.all(err <= bound), (i, float((err / bound).max()))
        worst = max(worst, float((err / bound).max()))
    return worst


def _product_gamma(K):
    if K <= 128:  # tensor cores, three BF16 pieces per operand
        return (4 + 12 * math.ceil(K / 16)) * U
    return K * U / (1 - K * U)


def _residual_bound(X, W, F, K):
    X, W, F = (np.asarray(a, dtype=np.float64) for a in (X, W, F))
    r = X - W @ F
    gk = _product_gamma(K)
    g64 = 64 * U / (1 - 64 * U)
    per = 2 * np.abs(r) * (U * np.abs(r) + gk * (np.abs(W) @ np.abs(F))) + g64 * r * r
    return 2 * float(per.sum()) + 1e-300


def _gpu_factors(d):
    import torch

    from paper_1608_04647_gb300 import htfa
    grid = htfa.GridPositions([torch.from_numpy(a) for a in d["axes"]], _cuda(d["vox"]))
    flag = torch.zeros(1, dtype=torch.int32, device="cuda")
    F = htfa.factors(grid, _cuda(d["mu"]), _cuda(d["lam"]), flag=flag)
    return F, int(flag.item())


@pytest.mark.parametrize("name", ["ragged-small", "greeneyes-subsampled-like"])
def test_factors_match_oracle(name):
    import synth.htfa_inputs as hi
    d = hi.draw(hi.HTFA_CONFIGS[name])
    F, flag = _gpu_factors(d)
    assert flag == 0
    worst = _check_factors(d, F.cpu().numpy())
    print(name, "worst error / bound", worst)


@pytest.mark.parametrize("K,V", [(1, 1), (130, 1500), (5, 2049)])
def test_factors_shapes(K, V):
    import dataclasses

    import synth.htfa_inputs as hi
    spec = dataclasses.replace(hi.HTFA_CONFIGS["ragged-small"], n_subjects=2, K=K, V=V, T=3)
    d = hi.draw(spec)
    F, flag = _gpu_factors(d)
    assert flag == 0 and tuple(F.shape) == (2, K, V)
    _check_factors(d, F.cpu().numpy())


def test_factors_long_axis_uses_several_table_chunks():
    """nx = 4000: a block holds the tables of only 3 factors at once."""
    import torch

    import oracle
    from paper_1608_04647_gb300 import htfa
    rng = np.random.default_rng(21)
    ax = [np.linspace(-200, 200, 4000).astype(np.float32), np.array([0.0], np.float32),
          np.array([1.5], np.float32)]
    V, K = 3000, 7
    vox = np.zeros((V, 3), np.int32)
    vox[:, 0] = rng.integers(0, 4000, V)
    pos = np.stack([ax[0][vox[:, 0]], np.zeros(V, np.float32), np.full(V, 1.5, np.float32)], axis=1)
    mu = rng.uniform(-150, 150, (K, 3)).astype(np.float32)
    lam = rng.uniform(50, 2000, K).astype(np.float32)
    grid = htfa.GridPositions([torch.from_numpy(a) for a in ax], _cuda(vox))
    F = htfa.factors(grid, _cuda(mu), _cuda(lam)).cpu().numpy()
    Fo = oracle.rbf_factors(pos, mu, lam)
    assert np.all(np.abs(F - Fo) <= _factor_bound(pos, mu, lam, Fo))


def test_factors_flag_bad_voxels_and_widths():
    import torch

    import oracle
    import synth.htfa_inputs as hi
    from paper_1608_04647_gb300 import htfa
    d = hi.draw(hi.HTFA_CONFIGS["ragged-small"])
    vox = d["vox"][0].copy()
    vox[5, 0] = 61          # one past the x axis
    vox[9, 2] = -1
    lam = d["lam"][0].copy()
    lam[3] = 0.0
    lam[4] = -2.0
    grid = htfa.GridPositions([torch.from_numpy(a) for a in d["axes"]], _cuda(vox))
    flag = torch.zeros(1, dtype=torch.int32, device="cuda")
    F = htfa.factors(grid, _cuda(d["mu"][0]), _cuda(lam), flag=flag).cpu().numpy()
    assert int(flag.item()) == htfa.FLAG_BAD_VOXEL | htfa.FLAG_BAD_WIDTH
    assert np.all(np.isnan(F[:, 5])) and np.all(np.isnan(F[:, 9]))
    assert np.all(np.isnan(F[3])) and np.all(np.isnan(F[4]))
    good_k = [k for k in range(F.shape[0]) if k not in (3, 4)]
    good_v = [v for v in range(F.shape[1]) if v not in (5, 9)]
    Fo = oracle.rbf_factors(d["positions"][0][good_v], d["mu"][0][good_k], d["lam"][0][good_k])
    sub = F[np.ix_(good_k, good_v)]
    assert np.all(np.abs(sub - Fo) <= _factor_bound(d["positions"][0][good_v], d["mu"][0][good_k],
                                                    d["lam"][0][good_k], Fo))


def _residual_case(d, V=None):
    import oracle
    n = d["W"].shape[0]
    Fs, Xs = [], []
    for i in range(n):
        Fo = oracle.rbf_factors(d["positions"][i], d["mu"][i], d["lam"][i]).astype(np.float32)
        Xs.append((d["W"][i].astype(np.float64) @ Fo + d["E"][i]).astype(np.float32))
        Fs.append(Fo)
    X, F = np.stack(Xs), np.stack(Fs)
    if V is not None:
        X, F = X[:, :, :V].copy(), F[:, :, :V].copy()
    return X, d["W"], F


@pytest.mark.parametrize("name,V", [("ragged-small", None), ("ragged-small", 699), ("greeneyes-subsampled-like", None)])
def test_residual_matches_oracle(name, V):
    import oracle
    import synth.htfa_inputs as hi
    from paper_1608_04647_gb300 import htfa
    d = hi.draw(hi.HTFA_CONFIGS[name])
    X, W, F = _residual_case(d, V)
    K = W.shape[-1]
    r1 = htfa.residual(_cuda(X), _cuda(W), _cuda(F)).cpu().numpy()
    r2 = htfa.residual(_cuda(X), _cuda(W), _cuda(F)).cpu().numpy()
    assert np.array_equal(r1, r2), "repeated calls must give identical bits"
    for i in range(X.shape[0]):
        ro = oracle.htfa_residual(X[i], W[i], F[i])
        bound = _residual_bound(X[i], W[i], F[i], K)
        assert abs(r1[i] - ro) <= bound, (i, r1[i], ro, bound)
    print(name, "relative error", float(np.max(np.abs(r1 - oracle.htfa_residual_batch(X, W, F)) / r1)))


# tensor-core tiles (128 x 64, K in steps of 16): ragged in T, V and K, two K
# atoms (K > 64), the largest K of that path (128); and K > 128 (FP32 FMA path)
@pytest.mark.parametrize("T,V,K", [(1, 1, 1), (1, 5, 3), (65, 63, 17), (64, 64, 16), (3, 1000, 1),
                                   (129, 65, 65), (300, 513, 100), (128, 64, 128), (70, 200, 150)])
def test_residual_small_shapes(T, V, K):
    import oracle
    from paper_1608_04647_gb300 import htfa
    rng = np.random.default_rng(T * 1000 + V + K)
    X = rng.standard_normal((T, V)).astype(np.float32)
    W = rng.standard_normal((T, K)).astype(np.float32)
    F = rng.uniform(0, 1, (K, V)).astype(np.float32)
    r = float(htfa.residual(_cuda(X), _cuda(W), _cuda(F)).item())
    assert abs(r - oracle.htfa_residual(X, W, F)) <= _residual_bound(X, W, F, K)


def test_residual_empty_is_zero():
    import torch

    from paper_1608_04647_gb300 import htfa
    X = torch.empty((3, 0, 10), device="cuda")
    W = torch.empty((3, 0, 4), device="cuda")
    F = torch.ones((3, 4, 10), device="cuda")
    out = torch.full((3,), 7.0, dtype=torch.float64, device="cuda")
    htfa.residual(X, W, F, out=out)
    assert out.cpu().numpy().tolist() == [0.0, 0.0, 0.0]


def _zscore_bound(X, Zo):
    X = np.asarray(X, dtype=np.float64)
    T = X.shape[0]
    dev = X - X[:1]
    A = np.abs(dev).max(axis=0)
    m1 = dev.mean(axis=0)
    S2 = (dev * dev).mean(axis=0)
    var = np.maximum(S2 - m1 * m1, 1e-300)
    s = np.sqrt(var)
    c = (T / 8 + 10) * U
    dm = c * A
    dvar = c * S2 + 2 * np.abs(m1) * dm + 2 * U * S2
    ds = dvar / (2 * var) + 3 * U
    return 2 * (dm / s + np.abs(Zo) * ds + 4 * U * np.abs(Zo) + U * A / s) + 1e-30


@pytest.mark.parametrize("T,V,inplace", [(150, 700, False), (174, 6857, True), (1000, 333, False),
                                         (1000, 64, True), (1, 40, False)])
def test_zscore_matches_oracle(T, V, inplace):
    import oracle
    from paper_1608_04647_gb300 import htfa
    rng = np.random.default_rng(T + V)
    X = (rng.normal(0, 1, (2, T, V)) * rng.uniform(0.1, 5, (2, 1, V)) + rng.uniform(-20, 20, (2, 1, V)))
    X = X.astype(np.float32)
    X[1, :, 3 % V] = 0.1     # a constant column
    Xg = _cuda(X)
    Z = (htfa.zscore(Xg, out=Xg) if inplace else htfa.zscore(Xg)).cpu().numpy()
    for i in range(2):
        Zo = oracle.zscore(X[i])
        err = np.abs(Z[i].astype(np.float64) - Zo)
        assert np.all(err <= _zscore_bound(X[i], Zo)), (i, float(err.max()))
    assert np.all(Z[1, :, 3 % V] == 0)


def test_jacobian_example_full_size():
    """One subject of V = 50,000 voxels, T = 2,000 samples, K = 100 factors
    (the size of the paper's Jacobian example, Sec. III-B), in the launch
    configuration of the bench: every element of F and the residual, with
    the oracle's sum taken over blocks of rows."""
    import torch

    import oracle
    import synth.htfa_inputs as hi
    from paper_1608_04647_gb300 import htfa
    spec = hi.HTFA_CONFIGS["jacobian-example-like"]
    d = hi.draw(spec)
    F, flag = _gpu_factors(d)
    assert flag == 0
    Fg = F.cpu().numpy()
    _check_factors(d, Fg)
    Fo = oracle.rbf_factors(d["positions"][0], d["mu"][0], d["lam"][0]).astype(np.float32)
    W = d["W"][0]
    X = np.empty((spec.T, spec.V), np.float32)
    for t0 in range(0, spec.T, 250):
        X[t0:t0 + 250] = (W[t0:t0 + 250].astype(np.float64) @ Fo + d["E"][0, t0:t0 + 250]).astype(np.float32)
    r = float(htfa.residual(_cuda(X), _cuda(W), _cuda(Fo)).item())
    ro, bound = 0.0, 0.0
    for t0 in range(0, spec.T, 250):
        ro += oracle.htfa_residual(X[t0:t0 + 250], W[t0:t0 + 250], Fo)
        bound += _residual_bound(X[t0:t0 + 250], W[t0:t0 + 250], Fo, spec.K)
    print("residual", r, "oracle", ro, "bound", bound, "relative error", abs(r - ro) / ro)
    assert abs(r - ro) <= bound
    del F
    torch.cuda.empty_cache()
