"""Tensor-core building blocks on the GPU: TMA 128-byte-swizzled loads,
shared-memory descriptors (K-major and MN-major), tcgen05.mma into TMEM and
TMEM loads, against a plain FP32 matrix product of the same BF16 values."""
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _build():
    from paper_1608_04647_gb300 import _build as b
    b.build()


@pytest.mark.parametrize("mn", [0, 1], ids=["kmajor", "mnmajor"])
@pytest.mark.parametrize("N", [64, 128])
@pytest.mark.parametrize("K", [64, 192, 256])
def test_mma_selftest(mn, N, K):
    import torch

    import paper_1608_04647_gb300 as srm
    g = torch.Generator().manual_seed(100 * mn + N + K)
    if mn == 0:
        A = torch.randn(128, K, generator=g).bfloat16()
        B = torch.randn(N, K, generator=g).bfloat16()
        ref = A.float() @ B.float().T
    else:
        A = torch.randn(K, 128, generator=g).bfloat16()
        B = torch.randn(K, N, generator=g).bfloat16()
        ref = A.float().T @ B.float()
    Ad, Bd = A.cuda(), B.cuda()
    D = torch.full((128, N), float("nan"), device="cuda")
    srm.srm_debug_mma(mn, Ad.data_ptr(), Bd.data_ptr(), D.data_ptr(), N, K)
    err = (D.cpu() - ref).abs().max().item() / ref.abs().max().item()
    assert err < 1e-5, err


def test_bounded_wait_gives_up_and_reports():
    """A wait on an mbarrier that nothing arrives on ends by itself: the
    waiter gives up, raises the abort flag (which stops the other waiting
    warp) and the timeout bit of the status word, and the host reads it.  No
    fault, trap or hang: the device stays usable (an MMA self-test after it
    still computes correctly)."""
    import time

    import torch

    import paper_1608_04647_gb300 as srm
    srm.srm_debug_wait(True)  # both waits satisfied
    t0 = time.perf_counter()
    with pytest.raises(srm.SrmError) as ei:
        srm.srm_debug_wait(False)
    dt = time.perf_counter() - t0
    assert ei.value.status == srm.SRM_ERR_NUMERIC
    assert "bounded wait gave up" in str(ei.value) and "0, 0" in str(ei.value)
    assert dt < 10.0  # the limit is one second of waiting
    g = torch.Generator().manual_seed(7)
    A = torch.randn(128, 64, generator=g).bfloat16()
    B = torch.randn(64, 64, generator=g).bfloat16()
    Ad, Bd = A.cuda(), B.cuda()  # kept alive for the call
    D = torch.full((128, 64), float("nan"), device="cuda")
    srm.srm_debug_mma(0, Ad.data_ptr(), Bd.data_ptr(), D.data_ptr(), 64, 64)
    ref = A.float() @ B.float().T
    assert (D.cpu() - ref).abs().max().item() / ref.abs().max().item() < 1e-5
