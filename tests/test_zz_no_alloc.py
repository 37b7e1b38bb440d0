"""srm_transform_noalloc is the transform for callers that must not allocate
device memory: latency-bound loops, where an allocation would synchronise the
device, and hosts whose device memory belongs to a pool.  These tests check
three things.  It gives the result of srm_transform on two calls in a row, for
the plain FP32 and the batched BF16 forms.  Those calls leave the device's
free memory unchanged.  Oversized requests are refused before anything runs.

The file name sorts last, so pytest collects it after every other test.  That
is its only ordering need: if it fails under ``-x``, every other test has
already run.  It depends on no other test and passes when run alone."""
import numpy as np
import pytest

from gpu_cases import Case, make_inputs

pytestmark = pytest.mark.gpu
TOL = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _build():
    from paper_1608_04647_gb300 import _build as b
    b.build()


@pytest.mark.parametrize("store", ["f32", "bf16"])
def test_noalloc_transform_matches_transform(store):
    import torch

    import paper_1608_04647_gb300 as srm
    case = Case("noalloc", [2999, 4100, 1500], 333, 50, 3, seed=1)
    d = make_inputs(case)
    X = [torch.from_numpy(x).cuda() for x in d["X"]]
    W0 = [torch.from_numpy(w).cuda() for w in d["W0"]]
    m = srm.SRM(X, W0, case.k, store=store)
    m.fit(case.n_iter)
    rng = np.random.default_rng(11)
    for i in range(len(X)):
        Xn = torch.from_numpy((rng.standard_normal((case.voxels[i], 97)) + 1.5).astype(np.float32)).cuda()
        ref = m.transform(i, Xn)
        outs = [torch.full_like(ref, float("nan")) for _ in range(2)]
        for j, S in enumerate(outs):  # two calls in a row share the fixed scratch array
            torch.cuda.synchronize()
            before = torch.cuda.mem_get_info()[0]
            srm.srm_transform_noalloc(m.ctx, i, Xn.data_ptr(), int(Xn.shape[1]), S.data_ptr())
            m.synchronize()
            after = torch.cuda.mem_get_info()[0]
            # the very first call may load the kernels (lazy module loading can
            # take device memory for code); every later call must leave the
            # device's free memory exactly as it was
            if i > 0 or j > 0:
                assert after == before, (before, after)
            err = ((S - ref).abs().max() / ref.abs().max()).item()
            assert err <= TOL, err
    m.close()


def test_noalloc_rejects_oversized_request():
    import torch

    import paper_1608_04647_gb300 as srm
    case = Case("noalloc-big", [700], 40, 8, 1, seed=2)
    d = make_inputs(case)
    X = [torch.from_numpy(x).cuda() for x in d["X"]]
    W0 = [torch.from_numpy(w).cuda() for w in d["W0"]]
    m = srm.SRM(X, W0, case.k, store="f32")
    dummy = torch.zeros(16, device="cuda")
    with pytest.raises(srm.SrmError) as e:
        srm.srm_transform_noalloc(m.ctx, 0, dummy.data_ptr(), 10_000_000, dummy.data_ptr())
    assert e.value.status == srm.SRM_ERR_ARG
    assert "scratch" in str(e.value)
    m.close()
