"""srm_init with SRM_HOST_INPUT: the subjects' data stay in host memory and
the library streams them through two device staging buffers (copies of
consecutive subjects on two streams, each subject centred once its copy has
landed).  The staging changes no arithmetic, so a fit from host buffers,
pageable or pinned, must equal the fit from the same data on the device bit
for bit: the log-likelihood trace, E[S], rho^2, Sigma_s and every W_i.
Cases: one subject (one staging buffer) and five subjects of uneven size (the
two buffers alternate, each reused after the centring that read it), in both
storage forms."""
import numpy as np
import pytest

from gpu_cases import Case, make_inputs

pytestmark = pytest.mark.gpu

CASES = [
    Case("one-subject", [1777], 150, 12, 3, seed=71),
    Case("five-uneven", [900, 2311, 640, 1500, 1201], 200, 20, 3, seed=72),
]


@pytest.fixture(scope="module", autouse=True)
def _build():
    from paper_1608_04647_gb300 import _build as b
    b.build()


def _fit(X, W0, k, n_iter, store, host):
    import paper_1608_04647_gb300 as srm
    m = srm.SRM(X, W0, k, store=store, host_input=host, final_ll=True)
    ll = m.fit(n_iter)
    out = {"ll": np.asarray(ll), "ES": m.get_s().cpu().numpy(),
           "W": [m.get_w(i).cpu().numpy() for i in range(len(X))]}
    out["rho2"], out["Sigma_s"] = m.params()
    m.close()
    return out


@pytest.mark.parametrize("store", ["f32", "bf16"])
@pytest.mark.parametrize("case", CASES, ids=lambda c: c.name)
def test_host_input_equals_device_input(case, store):
    import torch
    d = make_inputs(case)
    W0 = [torch.from_numpy(w).cuda() for w in d["W0"]]
    dev = _fit([torch.from_numpy(x).cuda() for x in d["X"]], W0, case.k, case.n_iter, store, False)
    for memory in ("pageable", "pinned"):
        Xh = [torch.from_numpy(x).contiguous() for x in d["X"]]
        if memory == "pinned":
            Xh = [x.pin_memory() for x in Xh]
        host = _fit(Xh, W0, case.k, case.n_iter, store, True)
        for key in ("ll", "ES", "rho2", "Sigma_s"):
            np.testing.assert_array_equal(np.asarray(host[key]), np.asarray(dev[key]), err_msg=f"{memory} {key}")
        for i, (a, b) in enumerate(zip(host["W"], dev["W"])):
            np.testing.assert_array_equal(a, b, err_msg=f"{memory} W_{i}")
