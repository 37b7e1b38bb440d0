"""The library's sharded E-step (srm_estep_partial / srm_estep_finish,
Algorithm 1's Reduce between processes) on one GPU: the subjects are split
over two contexts, each driven by shard.fit_sharded from its own host
thread, with an in-process sum of the two contexts' y and sums standing in
for the all-reduce.  The result must match one context over all subjects,
and the FP64 oracle, within the form's bar:
* every context holds the whole log-likelihood trace, E[S] and Sigma_s;
* each context holds W_i and rho_i^2 of its own subjects.
The reduction order differs from one context's, so the comparison is to
rounding, not bitwise.  Calls out of order return SRM_ERR_STATE."""
import threading

import numpy as np
import pytest

from gpu_cases import Case, make_inputs, run_oracle

pytestmark = pytest.mark.gpu
TOL = {"f32": 1e-5, "bf16": 2e-2}


@pytest.fixture(scope="module", autouse=True)
def _build():
    from paper_1608_04647_gb300 import _build as b
    b.build()


class ThreadSum:
    """Sum of one tensor across `n` threads, in place in each (an all-reduce
    among contexts of one process).  Each caller's current CUDA stream is
    synchronised before its tensor is read and after the total is copied in."""

    def __init__(self, n):
        self.n = n
        self.bar = threading.Barrier(n)
        self.slots = {}
        self.total = None

    def __call__(self, rank, t):
        import torch
        torch.cuda.current_stream().synchronize()
        self.slots[rank] = t
        self.bar.wait()
        if rank == 0:
            tot = self.slots[0].clone()
            for r in range(1, self.n):
                tot += self.slots[r]
            torch.cuda.current_stream().synchronize()
            self.total = tot
        self.bar.wait()
        t.copy_(self.total)
        torch.cuda.current_stream().synchronize()
        self.bar.wait()


def _fit_two_shards(d, k, n_iter, store):
    import torch

    import paper_1608_04647_gb300 as srm
    from paper_1608_04647_gb300.shard import fit_sharded, shard_subjects
    X = [torch.from_numpy(x).cuda() for x in d["X"]]
    W0 = [torch.from_numpy(w).cuda() for w in d["W0"]]
    plan = shard_subjects([x.shape[0] for x in X], 2)
    models = [srm.SRM([X[i] for i in p], [W0[i] for i in p], k, store=store, stream=torch.cuda.Stream(),
                      max_iter=n_iter + 4) for p in plan]
    red = ThreadSum(2)
    errors = []

    def run(rank):
        try:
            fit_sharded(models[rank], n_iter, lambda t: red(rank, t))
            models[rank].synchronize()
        except Exception as e:  # reported by the main thread
            errors.append(e)
            red.bar.abort()

    th = [threading.Thread(target=run, args=(r,)) for r in range(2)]
    for t in th:
        t.start()
    for t in th:
        t.join(timeout=300)
    assert not errors, errors
    out = {"plan": plan, "models": models, "ll": [m.ll() for m in models],
           "ES": [m.get_s().cpu().numpy().astype(np.float64) for m in models]}
    out["params"] = [m.params() for m in models]
    W = [None] * len(X)
    rho2 = np.zeros(len(X))
    for m, p, (r, _) in zip(models, plan, out["params"]):
        for j, i in enumerate(p):
            W[i] = m.get_w(j).cpu().numpy().astype(np.float64)
            rho2[i] = r[j]
    out["W"], out["rho2"] = W, rho2
    return out


def _rel(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


@pytest.mark.parametrize("k", [50, 80], ids=["k50", "k80-phi-by-cholesky"])
@pytest.mark.parametrize("store", ["f32", "bf16"])
def test_two_shards_match_one_context_and_oracle(store, k):
    import paper_1608_04647_gb300 as srm
    from gpu_cases import run_gpu
    case = Case("sharded", [2999, 4100, 3333, 2500, 1800], 333, k, 6, seed=31)
    d = make_inputs(case)
    sh = _fit_two_shards(d, case.k, case.n_iter, store)
    one = run_gpu(d, case.k, case.n_iter, store=store, final_ll=False)
    o = run_oracle(d, case.n_iter, final_ll=False)
    assert all(len(p) > 0 for p in sh["plan"])
    errs = {}
    for ref, name in ((one, "one context"), (o, "oracle")):
        e = {"ll": max(_rel(ll, ref["ll"]) for ll in sh["ll"]),
             "ES": max(_rel(es, ref["ES"]) for es in sh["ES"]),
             "Sigma_s": max(_rel(p[1], ref["Sigma_s"]) for p in sh["params"]),
             "W": max(_rel(a, b) for a, b in zip(sh["W"], ref["W"])),
             "rho2": float(np.max(np.abs(sh["rho2"] - ref["rho2"]) / ref["rho2"]))}
        errs[name] = e
        for key, v in e.items():
            assert v <= TOL[store], (name, key, v)
    print(store, {n: {k: f"{v:.1e}" for k, v in e.items()} for n, e in errs.items()})
    # both shards hold the same global quantities
    np.testing.assert_array_equal(sh["ll"][0], sh["ll"][1])
    np.testing.assert_array_equal(sh["params"][0][1], sh["params"][1][1])
    for m in sh["models"]:
        m.close()
    one["model"].close()



def test_sharded_calls_out_of_order():
    import torch

    import paper_1608_04647_gb300 as srm
    case = Case("sharded-order", [700, 900], 64, 8, 1, seed=32)
    d = make_inputs(case)
    m = srm.SRM([torch.from_numpy(x).cuda() for x in d["X"]], [torch.from_numpy(w).cuda() for w in d["W0"]],
                case.k, store="f32")
    y, sums = m.shard_buffers()
    with pytest.raises(srm.SrmError) as e:
        m.estep_finish(y, sums)
    assert e.value.status == srm.SRM_ERR_STATE
    m.estep_partial(y, sums)
    for call in (m.estep, m.mstep, lambda: m.fit(1), lambda: m.estep_partial(y, sums)):
        with pytest.raises(srm.SrmError) as e:
            call()
        assert e.value.status == srm.SRM_ERR_STATE
    # a single context is its own whole: its partial sums are the totals
    m.estep_finish(y, sums)
    m.mstep()
    m.synchronize()
    ref = srm.SRM([torch.from_numpy(x).cuda() for x in d["X"]], [torch.from_numpy(w).cuda() for w in d["W0"]],
                  case.k, store="f32")
    ref.fit(1)
    np.testing.assert_allclose(m.ll(), ref.ll(), rtol=1e-9)
    np.testing.assert_allclose(m.params()[0], ref.params()[0], rtol=1e-6)
    m.close()
    ref.close()
