"""Shared helpers of the GPU parity tests: run the library and the FP64
oracle on the same seeded planted inputs and compare result by result."""
import dataclasses

import numpy as np

import oracle
import synth


@dataclasses.dataclass
class Case:
    name: str
    voxels: list
    T: int
    k: int
    n_iter: int
    seed: int = 0
    rho2_range: tuple = (0.1, 1.0)
    scale: float = 1.0  # multiplies the planted data (large-magnitude Gram matrices)


def make_inputs(case: Case):
    spec = synth.PlantedSpec(case.name, len(case.voxels), ("fixed", 0, 0), case.T, case.k, case.n_iter,
                             case.rho2_range, case.seed)
    d = synth.planted_dataset(spec, voxel_counts=case.voxels, dtype=np.float32)
    if case.scale != 1.0:
        d["X"] = [(x * np.float32(case.scale)).astype(np.float32) for x in d["X"]]
    d["W0"] = [w.astype(np.float32) for w in d["W0"]]
    return d


def run_oracle(d, n_iter, final_ll=True):
    return oracle.fit([x.astype(np.float64) for x in d["X"]], [w.astype(np.float64) for w in d["W0"]], n_iter,
                      final_ll=final_ll)


def run_gpu(d, k, n_iter, store="f32", graph=False, final_ll=True, input_bf16=False, single_pass=False,
            eig_polar=False, plan=None):
    import torch

    import paper_1608_04647_gb300 as srm
    X = [torch.from_numpy(x).cuda() for x in d["X"]]
    if input_bf16:
        X = [x.to(torch.bfloat16) for x in X]
    W0 = [torch.from_numpy(w).cuda() for w in d["W0"]]
    m = srm.SRM(X, W0, k, store=store, graph=graph, final_ll=final_ll, single_pass=single_pass)
    if eig_polar:  # every polar factor through the eigen-decomposition path
        srm.srm_debug_force_eig_polar(m.ctx, True)
    if plan:  # launch-plan fields set before the fit
        m.set_plan(**plan)
    ll = m.fit(n_iter)
    out = {"ll": ll, "W": [m.get_w(i).cpu().numpy().astype(np.float64) for i in range(len(X))],
           "ES": m.get_s().cpu().numpy().astype(np.float64)}
    out["rho2"], out["Sigma_s"] = m.params()
    out["model"] = m
    return out


def rel_errors(g, o):
    """Per-result relative errors (max-norm), as stated for each result."""
    ew = max(np.abs(a - b).max() / np.abs(b).max() for a, b in zip(g["W"], o["W"]))
    es = np.abs(g["ES"] - o["ES"]).max() / np.abs(o["ES"]).max()
    er = np.max(np.abs(g["rho2"] - o["rho2"]) / o["rho2"])
    el = np.max(np.abs(g["ll"] - o["ll"]) / np.abs(o["ll"]))
    esg = np.abs(g["Sigma_s"] - o["Sigma_s"]).max() / np.abs(o["Sigma_s"]).max()
    return {"W": ew, "ES": es, "rho2": er, "ll": el, "Sigma_s": esg}


# Largest log-likelihood decrease accepted per iteration, as a fraction of
# |LL|.  EM never decreases the likelihood in exact arithmetic.  The FP32
# form evaluates the quadratic terms of the LL (sum_i ||X^_i||^2 / rho_i^2
# and <y, Phi y>, each at most |LL|) from FP32 sums: 2^-20 |LL| allows a few
# ulps of FP32 on them.  The BF16 form also takes its M-step's polar factor
# from the BF16-rounded A_i, which is not the exact maximiser of the
# Q-function; the loss is second order in that rounding, u_bf16^2 = 2^-18 of
# the quadratic terms, so 2^-16 |LL| allows a factor of 4 on it.
LL_DROP = {"f32": 2.0 ** -20, "bf16": 2.0 ** -16}


def check_ll_trace(g_ll, o_ll, store, rel_inc=2e-2):
    """The GPU's log-likelihood trace against EM's monotonicity and against
    the oracle's per-iteration increments.  Every decrease is reported; none
    may exceed LL_DROP[store] |LL|.  Where the oracle's own increment is
    large against that bound (100 x), the GPU's increment must match it to
    `rel_inc` relative.  Returns the decreases (iteration, nats)."""
    g_ll = np.asarray(g_ll, dtype=np.float64)
    o_ll = np.asarray(o_ll, dtype=np.float64)
    dg, do = np.diff(g_ll), np.diff(o_ll)
    bound = LL_DROP[store] * np.abs(g_ll[1:])
    drops = [(j + 1, float(-x)) for j, x in enumerate(dg) if x < 0]
    if drops:
        print("log-likelihood decreases (iteration, nats):", drops, "bound", bound.max())
    assert np.all(dg >= -bound), (drops, bound)
    big = do > 100 * bound
    assert np.all(np.abs(dg[big] - do[big]) <= rel_inc * do[big]), list(zip(dg[big], do[big]))
    return drops
