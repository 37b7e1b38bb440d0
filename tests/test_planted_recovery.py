"""Planted recovery on the GPU matches the oracle's.

The model has several exact optima: (W_i R, R^T S, R^T Sigma_s R) are equally
likely for any orthogonal R.  So recovery of the planted parameters is
measured without reference to a rotation:

* the largest principal-angle sine between each fitted W_i and the planted
  W_i;
* the relative error of E[S] against the planted (demeaned) S, after the
  orthogonal Procrustes rotation that best aligns them.

Both are computed for the GPU's and for the oracle's fit of the same seeded
inputs.  The difference between GPU and oracle must stay within 1e-3 for the
FP32 form and 1e-2 for the BF16 form.  At the raider-like shapes the
planted parameters are not recoverable at all.  The signal variance per
voxel is about k sigma^2 / v_i ~ 0.007, against a noise variance rho_i^2 of
0.1-1, and with v_i / T ~ 7 the noise's leading sample directions dominate.
There the test checks only that the GPU lands where the oracle does.  A
high-SNR case (v_i = 200, T = 4000) requires recovery itself:
sin theta < 0.1 and an S error below 0.1."""
import math

import numpy as np
import pytest

from gpu_cases import Case, make_inputs, run_gpu, run_oracle

pytestmark = pytest.mark.gpu
BAR = {"f32": 1e-3, "bf16": 1e-2}


@pytest.fixture(scope="module", autouse=True)
def _build():
    from paper_1608_04647_gb300 import _build as b
    b.build()


def _recovery(W, ES, W_true, S_true):
    from scipy.linalg import orthogonal_procrustes, subspace_angles
    sin_w = [float(np.sin(subspace_angles(a, b)).max()) for a, b in zip(W, W_true)]
    Sc = S_true - S_true.mean(axis=1, keepdims=True)
    R, _ = orthogonal_procrustes(ES.T, Sc.T)
    err_s = float(np.linalg.norm(ES.T @ R - Sc.T) / np.linalg.norm(Sc))
    return np.array(sin_w), err_s


@pytest.mark.parametrize("store", ["f32", "bf16"])
def test_raider_like_recovery_matches_oracle(store):
    pytest.importorskip("scipy")
    case = Case("raider-like", [2000] * 4, 300, 10, 10, seed=0)
    d = make_inputs(case)
    o = run_oracle(d, case.n_iter)
    g = run_gpu(d, case.k, case.n_iter, store=store)
    sw_g, es_g = _recovery(g["W"], g["ES"], d["W_true"], d["S_true"])
    sw_o, es_o = _recovery(o["W"], o["ES"], d["W_true"], d["S_true"])
    print(store, "sin theta gpu", np.round(sw_g, 4), "oracle", np.round(sw_o, 4), "S err", es_g, es_o)
    assert np.abs(sw_g - sw_o).max() <= BAR[store]
    assert abs(es_g - es_o) <= BAR[store]


@pytest.mark.parametrize("store", ["f32", "bf16"])
def test_high_snr_recovery(store):
    pytest.importorskip("scipy")
    import torch

    import oracle
    import paper_1608_04647_gb300 as srm
    import synth
    rng = np.random.default_rng(15)
    k, T = 5, 4000
    S = np.diag(np.sqrt(np.linspace(20, 5, k))) @ rng.standard_normal((k, T))
    X, Wt, W0 = [], [], []
    for _ in range(3):
        w = synth.random_orthonormal(rng, 200, k)
        X.append((w @ S + rng.standard_normal((200, 1)) +
                  math.sqrt(rng.uniform(0.1, 0.3)) * rng.standard_normal((200, T))).astype(np.float32))
        Wt.append(w)
        W0.append(synth.random_orthonormal(rng, 200, k).astype(np.float32))
    o = oracle.fit([x.astype(np.float64) for x in X], [w.astype(np.float64) for w in W0], 40)
    m = srm.SRM([torch.from_numpy(x).cuda() for x in X], [torch.from_numpy(w).cuda() for w in W0], k, store=store)
    m.fit(40)
    Wg = [m.get_w(i).cpu().numpy().astype(np.float64) for i in range(3)]
    ESg = m.get_s().cpu().numpy().astype(np.float64)
    sw_g, es_g = _recovery(Wg, ESg, Wt, S)
    sw_o, es_o = _recovery(o["W"], o["ES"], Wt, S)
    print(store, "sin theta gpu", np.round(sw_g, 4), "oracle", np.round(sw_o, 4), "S err", es_g, es_o)
    assert sw_g.max() < 0.1 and es_g < 0.1
    assert np.abs(sw_g - sw_o).max() <= BAR[store]
    assert abs(es_g - es_o) <= BAR[store]
