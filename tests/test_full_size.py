"""Parity at the full sizes of the benchmarked workloads, in the launch
configuration bench.py times: the batched BF16 form, the autotuned plan and
CUDA-graph iterations.

Whole fits are compared with the oracle in tests/test_config_scale.py: the
greeneyes-like workload in full, and the forrest-like shape on three
subjects.  Here the workloads run at their full sizes: greeneyes-like,
batched (64 subjects), forrest-like (8 x 600000 voxels, T = 3500, k = 100,
34 GB resident) and forrest-1024-like (1024 subjects, 41 GB).  A whole FP64
oracle fit of the larger ones would take many minutes (about a minute per
iteration on 16 host cores for forrest-1024-like) and more host memory than
the box has in FP64.  So each check starts from the GPU's own state after
the workload's fit.  From that state and the same seeded inputs, the oracle
computes outputs it can afford one by one:

* E-step: E[S] on sampled columns.  The reduced E-step acts on each column
  t separately (y_t = sum_i rho_i^-2 W_i^T x^_it, E[s_t] = Phi y_t), so
  oracle.estep on the columns {t} gives exactly those columns of E[S].
* M-step: W_i and rho_i^2 of sampled subjects, from the GPU's E[S] and the
  Sigma_s^new that the oracle forms from it.

Properties that hold at any size are checked too: a log-likelihood that
does not decrease beyond the rounding bound of the BF16 form, orthonormal
W_i, positive rho_i^2, and a symmetric positive definite Sigma_s.  The bar
is the BF16 form's 2e-2 relative (max-norm): the oracle consumes the
unrounded FP32 input.  The sample means of the columns are prepared with
PyTorch on the device (input preparation, not the library).  The oracle
does the E-step and M-step arithmetic.  The number of subjects whose polar
factor failed its Newton-Schulz certificate in the last M-step is
printed."""
from collections.abc import Sequence

import numpy as np
import pytest

from gpu_cases import LL_DROP

pytestmark = pytest.mark.gpu
TOL_BF16 = 2e-2


class _Lazy(Sequence):
    """A sequence whose items are fetched when the oracle reads them, so that
    a thousand subjects never sit on the host at once."""

    def __init__(self, n, fetch):
        self.n, self.fetch = n, fetch

    def __len__(self):
        return self.n

    def __getitem__(self, i):
        if i < 0 or i >= self.n:
            raise IndexError(i)
        return self.fetch(i)


@pytest.fixture(scope="module", autouse=True)
def _build():
    from paper_1608_04647_gb300 import _build as b
    b.build()


def _rel(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


# greeneyes-like (16 subjects, T = 1000), batched (64 subjects of
# 10,000-200,000 voxels), forrest-like (T = 3500, k = 100, 34 GB resident) and
# forrest-1024-like (1024 subjects, T = 500, 41 GB resident)
@pytest.mark.parametrize("config", [1, 2, 3, 4])
def test_full_size_sampled_parity(config):
    import torch

    import oracle
    import paper_1608_04647_gb300 as srm
    import synth
    from synth.planted_torch import planted_dataset_torch

    spec = synth.config_spec(config)
    vox = synth.draw_voxel_counts(spec)
    N, T, k = len(vox), spec.T, spec.k
    d = planted_dataset_torch(spec, vox, device="cuda")
    m = srm.SRM(d["X"], d["W0"], k, store="bf16", graph=True, max_iter=spec.n_iter + 16)
    plan, _, _ = m.autotune(None, iters=2)
    ll = m.fit(spec.n_iter)
    rho2, sig = m.params()
    print(spec.name, plan)

    sweeps = srm.srm_debug_eig_sweeps(m.ctx, N + 1)[:N]
    print("polar factors of the last M-step: %d certified Newton-Schulz, %d eigen-decomposition fallbacks"
          % (int(np.sum(sweeps < 256)), int(np.sum(sweeps >= 256))))

    # properties at any size
    assert np.all(np.isfinite(ll)) and np.all(np.diff(ll) >= -LL_DROP["bf16"] * np.abs(ll[1:])), ll
    assert np.all(rho2 > 0)
    np.testing.assert_allclose(sig, sig.T, rtol=0, atol=1e-12 * np.abs(sig).max())
    assert np.linalg.eigvalsh(sig).min() > 0

    # one more E-step on the GPU; the oracle's E-step on sampled columns
    cols = [0, T // 3, T - 1]

    def xcols(i):
        x = d["X"][i]
        mu = x.double().mean(dim=1, keepdim=True)
        return (x[:, cols].double() - mu).cpu().numpy()

    def wfetch(i):
        return m.get_w(i).double().cpu().numpy()

    est = oracle.estep(_Lazy(N, xcols), _Lazy(N, wfetch), rho2, sig)
    m.estep()
    es_gpu = m.get_s().double().cpu().numpy()
    err_es = float(np.abs(es_gpu[:, cols] - est["ES"]).max() / np.abs(es_gpu).max())

    # the M-step on the GPU; the oracle's M-step for sampled subjects from
    # the GPU's E[S] (all columns) and the Sigma_s^new it implies
    sub = sorted({0, N // 2, N - 1})
    sig_new = oracle.sigma_update({"ES": es_gpu, "Phi": est["Phi"]}, T)
    w_o, r_o = [], []
    for i in sub:  # one subject at a time: a forrest-like subject is 17 GB in FP64
        x_i, _, s_i = oracle.center(d["X"][i].cpu().numpy())
        w, r = oracle.mstep([x_i], [s_i], es_gpu, sig_new)
        w_o.append(w[0])
        r_o.append(r[0])
        del x_i
    m.mstep()
    rho2_new, sig_gpu = m.params()
    err_w = max(_rel(m.get_w(i).double().cpu().numpy(), w_o[j]) for j, i in enumerate(sub))
    err_r = max(abs(rho2_new[i] - r_o[j]) / r_o[j] for j, i in enumerate(sub))
    err_s = _rel(sig_gpu, sig_new)
    print({"E[S] columns": f"{err_es:.2e}", "W": f"{err_w:.2e}", "rho2": f"{err_r:.2e}",
           "Sigma_s": f"{err_s:.2e}"})
    assert err_es <= TOL_BF16
    assert err_w <= TOL_BF16
    assert err_r <= TOL_BF16
    assert err_s <= TOL_BF16
    for i in sub:
        w = m.get_w(i).double().cpu().numpy()
        np.testing.assert_allclose(w.T @ w, np.eye(k), atol=1e-3)
    m.close()
    del d
    torch.cuda.empty_cache()
