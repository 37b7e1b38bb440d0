"""Whole-fit parity at the scale of the benchmarked workloads.

Algorithm 1's fixed schedule runs on the GPU and in the FP64 oracle from the
same seeded inputs and the same W^0.  Each result is compared after the last
iteration: W_i, E[S], rho_i^2, Sigma_s and the whole log-likelihood trace.
The bars are 1e-5 relative (max-norm) for the plain FP32 form and 2e-2 for
the batched BF16 form.  The oracle consumes the unrounded FP32 input, so the
BF16 errors include the rounding of X^.

* greeneyes-like, the full workload: 16 subjects, v_i ~ U[20000, 60000],
  T = 1000, k = 50, 20 iterations.  It is fitted in both forms, each in the
  launch configuration the bench times (CUDA graph; the BF16 form autotuned).
  Planted recovery of the two fits is compared with the oracle's.
* forrest-like shape: T = 3500, k = 100 (padded to 128), rho_i^2 ~
  U[0.5, 2], 10 iterations, on three subjects of 20,000-60,000 voxels.  The
  E-pass runs seven 512-wide T-blocks, and the M-pass streams E[S] in 64-wide
  chunks at kld = 128.  The BF16 form runs under the tuned plan and under
  M-pass stages of 1 and 2 boxes per stage (4 boxes do not fit in shared
  memory beside the streamed E[S] chunks at kld = 128: that case checks that
  the library refuses the plan, then skips).

The oracle's fits take about a minute on 16 host cores."""
import dataclasses

import numpy as np
import pytest

from gpu_cases import check_ll_trace, rel_errors

pytestmark = pytest.mark.gpu
TOL = {"f32": 1e-5, "bf16": 2e-2}


@pytest.fixture(scope="module", autouse=True)
def _build():
    from paper_1608_04647_gb300 import _build as b
    b.build()


def _dataset(spec, voxels):
    import synth
    d = synth.planted_dataset(spec, voxel_counts=voxels, dtype=np.float32)
    d["W0"] = [w.astype(np.float32) for w in d["W0"]]
    return d


def _oracle(d, n_iter):
    import oracle
    return oracle.fit([x.astype(np.float64) for x in d["X"]], [w.astype(np.float64) for w in d["W0"]], n_iter,
                      final_ll=True)


def _gpu(d, k, n_iter, store, tune=False, plan=None):
    import torch

    import paper_1608_04647_gb300 as srm
    X = [torch.from_numpy(x).cuda() for x in d["X"]]
    W0 = [torch.from_numpy(w).cuda() for w in d["W0"]]
    m = srm.SRM(X, W0, k, store=store, graph=True, final_ll=True, max_iter=n_iter + 16)
    chosen = None
    if tune:
        chosen, _, _ = m.autotune(None, iters=2)
    if plan:
        if not _set_plan_fitting(m, plan):
            m.close()
            return None
        chosen = m.plan()
    ll = m.fit(n_iter)
    out = {"ll": ll, "W": [m.get_w(i).cpu().numpy().astype(np.float64) for i in range(len(X))],
           "ES": m.get_s().cpu().numpy().astype(np.float64), "plan": chosen}
    out["rho2"], out["Sigma_s"] = m.params()
    m.close()
    del X, W0
    torch.cuda.empty_cache()
    return out


def _set_plan_fitting(m, fields):
    """Apply plan fields with the largest M-pass stage count that fits in
    shared memory under them (srm_set_plan refuses plans that do not fit).
    Returns False if no stage count fits."""
    import paper_1608_04647_gb300 as srm
    for stages in range(8, 1, -1):
        try:
            m.set_plan(**dict(fields, m_stages=stages))
            return True
        except srm.SrmError as e:
            if e.status != srm.SRM_ERR_ARG:
                raise
    return False


def _check(g, o, store, name):
    err = rel_errors(g, o)
    print(name, store, g.get("plan"), {k: f"{v:.2e}" for k, v in err.items()})
    for key, e in err.items():
        assert e <= TOL[store], (name, store, key, e)
    for w in g["W"]:
        np.testing.assert_allclose(w.T @ w, np.eye(w.shape[1]), atol=1e-5 if store == "f32" else 2e-2)
    check_ll_trace(g["ll"], o["ll"], store)


# ------------------------------------------------------------------ greeneyes-like
@pytest.fixture(scope="module")
def greeneyes():
    import synth
    spec = synth.config_spec(1)
    vox = synth.draw_voxel_counts(spec)
    d = _dataset(spec, vox)
    o = _oracle(d, spec.n_iter)
    return spec, d, o


@pytest.mark.parametrize("store", ["f32", "bf16"])
def test_greeneyes_like_full_schedule(greeneyes, store):
    spec, d, o = greeneyes
    g = _gpu(d, spec.k, spec.n_iter, store, tune=(store == "bf16"))
    _check(g, o, store, "greeneyes-like")


def test_greeneyes_like_planted_recovery(greeneyes):
    """sin theta of each fitted W_i against the planted one, and the
    Procrustes-aligned E[S] error against the planted S: the GPU's fits land
    where the oracle's does (1e-3 FP32, 1e-2 BF16)."""
    pytest.importorskip("scipy")
    from scipy.linalg import orthogonal_procrustes, subspace_angles
    spec, d, o = greeneyes

    def recovery(W, ES):
        sw = np.array([float(np.sin(subspace_angles(a, b)).max()) for a, b in zip(W, d["W_true"])])
        Sc = d["S_true"] - d["S_true"].mean(axis=1, keepdims=True)
        R, _ = orthogonal_procrustes(ES.T, Sc.T)
        return sw, float(np.linalg.norm(ES.T @ R - Sc.T) / np.linalg.norm(Sc))

    sw_o, es_o = recovery(o["W"], o["ES"])
    for store, bar in (("f32", 1e-3), ("bf16", 1e-2)):
        g = _gpu(d, spec.k, spec.n_iter, store, tune=(store == "bf16"))
        sw_g, es_g = recovery(g["W"], g["ES"])
        print(store, "max sin theta gpu %.4f oracle %.4f; S error gpu %.4f oracle %.4f" %
              (sw_g.max(), sw_o.max(), es_g, es_o))
        assert np.abs(sw_g - sw_o).max() <= bar
        assert abs(es_g - es_o) <= bar


# ------------------------------------------------------------------ forrest-like shape
@pytest.fixture(scope="module")
def forrest_shape():
    import synth
    spec = dataclasses.replace(synth.config_spec(3), n_subjects=3,
                               name="forrest-like shape, 3 subjects v~U[2e4,6e4] T=3500 k=100")
    vox = [int(v) for v in np.random.default_rng(33).integers(20000, 60001, size=3)]
    d = _dataset(spec, vox)
    o = _oracle(d, spec.n_iter)
    return spec, d, o


PLANS = [
    ("tuned", None),
    ("boxes1", {"single_pass": 0, "m_resident_es": 0, "m_boxes": 1}),
    ("boxes2", {"single_pass": 0, "m_resident_es": 0, "m_boxes": 2}),
    ("boxes4", {"single_pass": 0, "m_resident_es": 0, "m_boxes": 4}),
]


@pytest.mark.parametrize("name,plan", PLANS, ids=[p[0] for p in PLANS])
def test_forrest_like_shape_bf16(forrest_shape, name, plan):
    spec, d, o = forrest_shape
    g = _gpu(d, spec.k, spec.n_iter, "bf16", tune=(plan is None), plan=plan)
    if g is None:
        # a stage holds m_boxes X^ boxes (64 t x 128 rows, 16 KB each) and, with
        # E[S] streamed, as many E[S] chunks (64 t x kld, 16 KB at kld = 128):
        # 128 KB per stage at 4 boxes, so two stages exceed the 227 KB per CTA
        assert plan["m_boxes"] == 4
        pytest.skip("4 boxes per stage with streamed E[S] at kld = 128 do not fit in shared memory "
                    "(2 stages x 128 KB > 227 KB); the library refuses the plan")
    if plan:
        assert g["plan"]["m_boxes"] == plan["m_boxes"]
    _check(g, o, "bf16", "forrest-like/" + name)


def test_forrest_like_shape_f32(forrest_shape):
    spec, d, o = forrest_shape
    g = _gpu(d, spec.k, spec.n_iter, "f32")
    _check(g, o, "f32", "forrest-like")
