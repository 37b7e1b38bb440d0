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
