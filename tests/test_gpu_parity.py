"""GPU parity: the library (through the C ABI) against the FP64 oracle on the
same seeded planted inputs.  Bars: 1e-5 relative (max-norm) for the plain
FP32 form, 2e-2 for the BF16-storage tensor-core form, for W_i, E[S],
rho_i^2, Sigma_s and the log-likelihood trace after the fixed schedule."""
import numpy as np
import pytest

from gpu_cases import Case, check_ll_trace, make_inputs, rel_errors, run_gpu, run_oracle

pytestmark = pytest.mark.gpu

TOL_F32 = 1e-5
TOL_BF16 = 2e-2

PLAIN_CASES = [
    # the raider-like workload itself (4 x 2000 voxels, 300 TRs, k = 10)
    Case("raider-like", [2000] * 4, 300, 10, 10, seed=0),
    # uneven voxel counts, ragged tiles, k not a multiple of 16, odd T
    Case("uneven-k50", [2999, 4100, 3333], 333, 50, 8, seed=1),
    # the high-resolution shape scaled down: k = 100, T not a multiple of 64
    Case("k100", [5000, 4321], 700, 100, 5, seed=3, rho2_range=(0.5, 2.0)),
    # smallest shapes: one subject, k = 1, v barely above k
    Case("tiny", [7], 9, 1, 6, seed=5),
    Case("k-odd", [130, 129, 257], 64, 17, 6, seed=6),
    # data of magnitude 1e4 (Gram entries near 1e20), k > 64: the eigen-solver path
    Case("k80-scaled-1e4", [3000, 2600], 400, 80, 4, seed=12, scale=1e4),
    Case("k50-scaled-1e4", [2500, 3100, 2000], 500, 50, 4, seed=13, scale=1e4),
    # the largest k of the Newton-Schulz polar path (64) and the smallest past it (65)
    Case("k64-boundary", [900, 1300], 130, 64, 4, seed=14),
    Case("k65-eigen-path", [1000, 1200], 131, 65, 4, seed=15),
    # the largest k the library accepts (128; the k x k kernels' shared memory)
    Case("k128-max", [1500, 1300], 300, 128, 3, seed=16),
    # more subjects than SMs: the polar factors run two CTAs per SM
    Case("subjects-beyond-sms", [int(x) for x in np.random.default_rng(18).integers(80, 200, size=200)], 120, 30, 3,
         seed=18),
    # more subjects than E-step reduction groups: several subjects per group
    Case("grouped-subjects", [int(x) for x in np.random.default_rng(11).integers(40, 250, size=150)], 1500, 8, 4,
         seed=11),
]


@pytest.fixture(scope="module", autouse=True)
def _build():
    from paper_1608_04647_gb300 import _build as b
    b.build()


@pytest.mark.parametrize("case", PLAIN_CASES, ids=lambda c: c.name)
def test_plain_fp32_matches_oracle(case):
    d = make_inputs(case)
    o = run_oracle(d, case.n_iter)
    g = run_gpu(d, case.k, case.n_iter, store="f32")
    err = rel_errors(g, o)
    print(case.name, {k: f"{v:.2e}" for k, v in err.items()})
    for key, e in err.items():
        assert e <= TOL_F32, (key, e)
    for w in g["W"]:
        np.testing.assert_allclose(w.T @ w, np.eye(case.k), atol=1e-5)
    check_ll_trace(g["ll"], o["ll"], "f32")


def test_plain_graph_equals_eager():
    case = PLAIN_CASES[1]
    d = make_inputs(case)
    a = run_gpu(d, case.k, case.n_iter, store="f32", graph=False)
    b = run_gpu(d, case.k, case.n_iter, store="f32", graph=True)
    np.testing.assert_array_equal(a["ll"], b["ll"])
    np.testing.assert_array_equal(a["ES"], b["ES"])


def test_plain_deterministic_and_checkpoint():
    import torch

    import paper_1608_04647_gb300 as srm
    case = PLAIN_CASES[1]
    d = make_inputs(case)
    a = run_gpu(d, case.k, 6, store="f32", final_ll=False)
    b = run_gpu(d, case.k, 6, store="f32", final_ll=False)
    np.testing.assert_array_equal(a["ll"], b["ll"])
    for x, y in zip(a["W"], b["W"]):
        np.testing.assert_array_equal(x, y)
    # fit(6) == fit(3) + checkpoint into a fresh context + fit(3)
    X = [torch.from_numpy(x).cuda() for x in d["X"]]
    W0 = [torch.from_numpy(w).cuda() for w in d["W0"]]
    m1 = srm.SRM(X, W0, case.k, store="f32")
    m1.fit(3)
    st = m1.state()
    m2 = srm.SRM(X, W0, case.k, store="f32")
    m2.set_state(st)
    m2.fit(3)
    np.testing.assert_array_equal(m2.ll(), a["ll"])
    np.testing.assert_array_equal(m2.get_w(0).cpu().numpy(), a["W"][0].astype(np.float32))


def test_transform_matches_oracle():
    import oracle
    import torch
    case = PLAIN_CASES[1]
    d = make_inputs(case)
    o = run_oracle(d, case.n_iter, final_ll=False)
    g = run_gpu(d, case.k, case.n_iter, store="f32", final_ll=False)
    rng = np.random.default_rng(3)
    for i in range(len(d["X"])):
        Xn = rng.standard_normal((d["X"][i].shape[0], 77)).astype(np.float32) + 2.0
        S = g["model"].transform(i, torch.from_numpy(Xn).cuda()).cpu().numpy()
        So = oracle.transform(o["W"][i], Xn.astype(np.float64))
        assert np.abs(S - So).max() / np.abs(So).max() <= 1e-5


def test_map_between_subjects_matches_oracle():
    """srm_map: W_j W_i^T (x - mean_t x) for new data, against the oracle's
    mappings (the same fit), including i == j (the projection onto span W_i)."""
    import oracle
    import torch
    case = PLAIN_CASES[1]
    d = make_inputs(case)
    o = run_oracle(d, case.n_iter, final_ll=False)
    g = run_gpu(d, case.k, case.n_iter, store="f32", final_ll=False)
    rng = np.random.default_rng(4)
    for i, j in [(0, 1), (1, 1), (2, 0)]:
        Xn = rng.standard_normal((d["X"][i].shape[0], 70)).astype(np.float32) - 1.0
        Y = g["model"].map(i, j, torch.from_numpy(Xn).cuda()).cpu().numpy()
        Yo = oracle.map_subjects(o["W"][i], o["W"][j], Xn.astype(np.float64))
        assert Y.shape == Yo.shape
        assert np.abs(Y - Yo).max() / np.abs(Yo).max() <= 1e-5


def test_transform_before_fit_uses_w0():
    import oracle
    import torch

    import paper_1608_04647_gb300 as srm
    case = PLAIN_CASES[0]
    d = make_inputs(case)
    X = [torch.from_numpy(x).cuda() for x in d["X"]]
    W0 = [torch.from_numpy(w).cuda() for w in d["W0"]]
    m = srm.SRM(X, W0, case.k, store="f32")
    S = m.transform(1, X[1]).cpu().numpy()
    So = oracle.transform(d["W0"][1].astype(np.float64), d["X"][1].astype(np.float64))
    assert np.abs(S - So).max() / np.abs(So).max() <= 1e-5


def test_call_order_errors():
    import torch

    import paper_1608_04647_gb300 as srm
    case = PLAIN_CASES[3]
    d = make_inputs(case)
    X = [torch.from_numpy(x).cuda() for x in d["X"]]
    W0 = [torch.from_numpy(w).cuda() for w in d["W0"]]
    m = srm.SRM(X, W0, case.k, store="f32")
    with pytest.raises(srm.SrmError) as e:
        m.mstep()
    assert e.value.status == srm.SRM_ERR_STATE
    with pytest.raises(srm.SrmError) as e:
        m.get_s()
    assert e.value.status == srm.SRM_ERR_STATE
    m.estep()
    m.mstep()
    m.synchronize()


def test_rank_deficient_subject_is_reported():
    """A subject whose data are constant over time has X^_i = 0, so A_i = 0 and
    its polar factor is undefined: the next synchronising call reports
    SRM_ERR_NUMERIC (no device fault)."""
    import torch

    import paper_1608_04647_gb300 as srm
    case = PLAIN_CASES[0]
    d = make_inputs(case)
    d["X"][2][:] = 3.0
    X = [torch.from_numpy(x).cuda() for x in d["X"]]
    W0 = [torch.from_numpy(w).cuda() for w in d["W0"]]
    m = srm.SRM(X, W0, case.k, store="f32")
    with pytest.raises(srm.SrmError) as e:
        m.fit(1)
    assert e.value.status == srm.SRM_ERR_NUMERIC
