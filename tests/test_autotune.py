"""GPU tests of the launch plans and the autotuner (srm_get_plan,
srm_set_plan, srm_autotune).

A plan changes how the two contractions are tiled and pipelined, never what
they compute.  So every plan must match the FP64 oracle within the bar of
the BF16 form.  Plans that differ only in pipelining (stages, Gram buffers,
E[S] residency, prefetch) must give bitwise identical results.  The tuner
must leave the context as srm_init left it, so a tuned fit is the fit an
untuned context runs under the chosen plan.  The cache file must replay the
choice without timing anything."""
import numpy as np
import pytest

from gpu_cases import Case, make_inputs, rel_errors, run_oracle

pytestmark = pytest.mark.gpu
TOL_BF16 = 2e-2

CASE = Case("tune-greeneyes-small", [3000, 2500, 1800, 2222], 1000, 50, 5, seed=23)
CASE_T500 = Case("tune-t500", [2100, 1900, 2600], 500, 20, 4, seed=31)
CASE_K100 = Case("tune-k100", [2600, 3100], 600, 100, 3, seed=32)


@pytest.fixture(scope="module", autouse=True)
def _build():
    from paper_1608_04647_gb300 import _build as b
    b.build()


def _model(d, k, final_ll=True, **kw):
    import torch

    import paper_1608_04647_gb300 as srm
    X = [torch.from_numpy(x).cuda() for x in d["X"]]
    W0 = [torch.from_numpy(w).cuda() for w in d["W0"]]
    return srm.SRM(X, W0, k, store="bf16", final_ll=final_ll, **kw)


def _results(m, n_iter):
    ll = m.fit(n_iter)
    out = {"ll": ll, "W": [m.get_w(i).cpu().numpy().astype(np.float64) for i in range(m.N)],
           "ES": m.get_s().cpu().numpy().astype(np.float64)}
    out["rho2"], out["Sigma_s"] = m.params()
    return out


@pytest.mark.parametrize("case", [CASE, CASE_T500, CASE_K100], ids=lambda c: c.name)
def test_autotuned_fit_matches_oracle_and_cache_replays(case, tmp_path):
    d = make_inputs(case)
    o = run_oracle(d, case.n_iter)
    cache = str(tmp_path / "plans.txt")
    m = _model(d, case.k, graph=True)
    plan, ms, rep = m.autotune(cache, iters=2)
    print(rep)
    assert ms > 0 and "chosen:" in rep
    assert plan == m.plan()
    if case.k > 64:
        assert plan["single_pass"] == 0
    # the single pass's 16 KB-slot forms are candidates where one CTA takes a tile (T <= 512)
    fine_tried = any(" fsl=9 " in ln or " fsl=8 " in ln for ln in rep.splitlines() if ln.startswith("fpass"))
    assert fine_tried == (case.k <= 64 and case.T <= 512), rep
    g = _results(m, case.n_iter)
    err = rel_errors(g, o)
    print(case.name, plan, {k: f"{v:.2e}" for k, v in err.items()})
    for key, e in err.items():
        assert e <= TOL_BF16, (key, e)
    # the tuner restored the initial state: same results as an untuned
    # context set to the chosen plan (bitwise: same plan, same launches)
    u = _model(d, case.k, graph=True)
    u.set_plan(**plan)
    h = _results(u, case.n_iter)
    np.testing.assert_array_equal(g["ll"], h["ll"])
    np.testing.assert_array_equal(g["ES"], h["ES"])
    # a second context of the same shapes replays the cached plan
    m2 = _model(d, case.k, graph=True)
    plan2, ms2, rep2 = m2.autotune(cache, iters=2)
    assert rep2.startswith("cached:")
    assert plan2 == plan and abs(ms2 - ms) < 1e-3 * ms + 1e-6


def test_every_plan_matches_oracle():
    import paper_1608_04647_gb300 as srm
    d = make_inputs(CASE)
    o = run_oracle(d, CASE.n_iter)
    plans = [dict(single_pass=0, e_reserve=0), dict(single_pass=0, e_reserve=32),
             dict(single_pass=0, m_stages=2, m_gram_bufs=1, m_resident_es=0, m_prefetch=0),
             dict(single_pass=0, m_stages=2, m_gram_bufs=1, m_resident_es=0, m_prefetch=0, m_boxes=4),
             dict(single_pass=1, f_prefetch=0), dict(single_pass=1, f_prefetch=3, f_l2_hints=7),
             dict(single_pass=1, f_prefetch=1, f_l2_hints=6), dict(single_pass=1, f_first_stages=1),
             dict(single_pass=1, f_first_stages=3, f_prefetch=2), dict(single_pass=1, f_first_stages=4),
             dict(single_pass=1, f_reserve=0), dict(single_pass=1, f_reserve=30, f_first_stages=1),
             dict(single_pass=1, f_first_stages=2, f_lead=1), dict(single_pass=1, f_first_stages=2, f_lead=3)]
    for fields in plans:
        m = _model(d, CASE.k, graph=True)
        m.set_plan(**fields)
        p = m.plan()
        for key, v in fields.items():
            assert p[key] == v, (key, p)
        err = rel_errors(_results(m, CASE.n_iter), o)
        print(fields, {k: f"{v:.2e}" for k, v in err.items()})
        for key, e in err.items():
            assert e <= TOL_BF16, (fields, key, e)
    # out-of-range plans are refused before anything runs
    m = _model(d, CASE.k)
    for bad in (dict(m_stages=9), dict(m_gram_bufs=3), dict(e_reserve=-1), dict(f_prefetch=99),
                dict(f_l2_hints=8), dict(f_first_stages=0), dict(f_first_stages=5), dict(m_boxes=3),
                dict(single_pass=1, f_reserve=-1), dict(f_lead=5), dict(f_slots=7),
                dict(f_slots=8, f_first_stages=7), dict(f_slots=9, f_first_stages=1)):
        with pytest.raises(srm.SrmError) as ei:
            m.set_plan(**bad)
        assert ei.value.status == srm.SRM_ERR_ARG, bad
    # the 16 KB-slot forms need one CTA per tile (T <= 512); this case has T = 1000
    with pytest.raises(srm.SrmError) as ei:
        m.set_plan(single_pass=1, f_slots=9, f_first_stages=6)
    assert ei.value.status == srm.SRM_ERR_UNSUPPORTED


def test_pipelining_plans_are_bitwise_identical():
    # stages, Gram buffers, E[S] residency, prefetch, L2 hints and the
    # single pass's ring split change when bytes arrive, not the order of any sum
    d = make_inputs(CASE_T500)
    runs = []
    for fields in (dict(m_stages=2, m_gram_bufs=2, m_resident_es=0, m_prefetch=0, m_boxes=1),
                   dict(m_stages=4, m_gram_bufs=1, m_resident_es=1, m_prefetch=8, m_boxes=1),
                   dict(m_stages=6, m_gram_bufs=2, m_resident_es=1, m_prefetch=0, m_boxes=1),
                   dict(m_stages=3, m_gram_bufs=1, m_resident_es=1, m_prefetch=0, m_boxes=2),
                   dict(m_stages=2, m_gram_bufs=1, m_resident_es=0, m_prefetch=0, m_boxes=4)):
        m = _model(d, CASE_T500.k)
        m.set_plan(single_pass=0, **fields)
        runs.append(_results(m, CASE_T500.n_iter))
    # the single pass: prefetch distance and L2 eviction hints
    fused = []
    for fields in (dict(f_prefetch=0, f_l2_hints=0, f_first_stages=2),
                   dict(f_prefetch=2, f_l2_hints=7, f_first_stages=1),
                   dict(f_prefetch=1, f_l2_hints=2, f_first_stages=3),
                   dict(f_prefetch=0, f_l2_hints=7, f_first_stages=4),
                   dict(f_prefetch=0, f_l2_hints=7, f_first_stages=2, f_lead=2),
                   dict(f_prefetch=0, f_l2_hints=7, f_first_stages=5, f_slots=8),
                   dict(f_prefetch=1, f_l2_hints=7, f_first_stages=6, f_slots=9, f_lead=3)):
        m = _model(d, CASE_T500.k)
        m.set_plan(single_pass=1, **fields)
        fused.append(_results(m, CASE_T500.n_iter))
    for group in (runs, fused):
        for r in group[1:]:
            np.testing.assert_array_equal(group[0]["ll"], r["ll"])
            np.testing.assert_array_equal(group[0]["ES"], r["ES"])
            for a, b in zip(group[0]["W"], r["W"]):
                np.testing.assert_array_equal(a, b)


def test_plan_switch_between_iterations():
    # two-pass -> single-pass -> two-pass inside one fit stays on the oracle's path
    d = make_inputs(CASE)
    o = run_oracle(d, 6, final_ll=False)
    m = _model(d, CASE.k, final_ll=False)
    m.set_plan(single_pass=0)
    m.fit_async(2)
    m.set_plan(single_pass=1, f_prefetch=2)
    m.fit_async(2)
    m.set_plan(single_pass=0, e_reserve=8)
    g = _results(m, 2)
    g["ll"] = m.ll()
    err = rel_errors(g, o)
    print({k: f"{v:.2e}" for k, v in err.items()})
    for key, e in err.items():
        assert e <= TOL_BF16, (key, e)


def test_autotune_state_errors():
    import paper_1608_04647_gb300 as srm
    d = make_inputs(CASE_T500)
    m = _model(d, CASE_T500.k)
    m.fit(1)
    with pytest.raises(srm.SrmError) as ei:
        m.autotune(None, iters=2)
    assert ei.value.status == srm.SRM_ERR_STATE
    m.estep()
    with pytest.raises(srm.SrmError) as ei:
        m.set_plan(m_stages=3)
    assert ei.value.status == srm.SRM_ERR_STATE
