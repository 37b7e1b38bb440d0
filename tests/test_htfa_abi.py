"""Host-side logic of the HTFA boundary (include/htfa.h), without a GPU:
scratch sizes, argument checks that return SRM_ERR_ARG before any launch,
empty batches that launch nothing, and the Python binding's checks."""
import ctypes

import pytest


@pytest.fixture(scope="module")
def lib():
    from paper_1608_04647_gb300 import _build, load_library
    _build.build()
    return load_library()


SRM_OK, SRM_ERR_ARG = 0, 1
P = ctypes.c_void_p(16)  # a non-null pointer that the checks below never dereference


def test_residual_workspace_holds_the_partials(lib):
    # K <= 128 (tensor cores): four doubles per tile of 128 samples x 64 voxels,
    # then a 16-byte status word; K > 128 (FP32 FMA): one double per tile of
    # 64 samples x 128 voxels, then the same 16 bytes
    assert lib.srm_htfa_residual_workspace(40, 100, 174, 6857) == 40 * 4 * 2 * 108 * 8 + 16
    assert lib.srm_htfa_residual_workspace(1, 100, 2000, 50000) == 4 * 16 * 782 * 8 + 16
    assert lib.srm_htfa_residual_workspace(2, 7, 64, 128) == 2 * 4 * 1 * 2 * 8 + 16
    assert lib.srm_htfa_residual_workspace(2, 150, 64, 128) == 2 * 1 * 1 * 8 + 16
    assert lib.srm_htfa_residual_workspace(0, 7, 64, 128) == 0
    assert lib.srm_htfa_residual_workspace(3, 7, 0, 128) == 0


def test_factors_workspace_holds_the_padded_tables(lib):
    # n (nx + ny + nz) Kp floats, K padded to a multiple of 4
    assert lib.srm_htfa_factors_workspace(40, 100, 61, 73, 61) == 40 * 195 * 100 * 4
    assert lib.srm_htfa_factors_workspace(3, 37, 61, 73, 61) == 3 * 195 * 40 * 4
    assert lib.srm_htfa_factors_workspace(1, 1, 1, 1, 1) == 3 * 4 * 4
    assert lib.srm_htfa_factors_workspace(0, 5, 4, 4, 4) == 0


def _msg(lib):
    return lib.srm_last_error().decode()


@pytest.mark.parametrize("args", [
    (-1, 10, 100), (65536, 10, 100), (1, 0, 100), (1, 10, -1)])
def test_factors_rejects_bad_sizes(lib, args):
    n, K, V = args
    st = lib.srm_htfa_factors(n, K, V, P, 4, 4, 4, P, P, P, P, None, P, 1 << 20, None)
    assert st == SRM_ERR_ARG and "srm_htfa_factors" in _msg(lib)


@pytest.mark.parametrize("axes", [(0, 4, 4), (4, 4097, 4), (4, 4, -2)])
def test_factors_rejects_bad_axes(lib, axes):
    st = lib.srm_htfa_factors(1, 3, 10, P, *axes, P, P, P, P, None, P, 1 << 20, None)
    assert st == SRM_ERR_ARG


def test_factors_rejects_null_or_short_scratch(lib):
    need = lib.srm_htfa_factors_workspace(2, 5, 4, 4, 4)
    assert lib.srm_htfa_factors(2, 5, 10, P, 4, 4, 4, P, P, P, P, None, None, need, None) == SRM_ERR_ARG
    assert lib.srm_htfa_factors(2, 5, 10, P, 4, 4, 4, P, P, P, P, None, P, need - 1, None) == SRM_ERR_ARG
    assert "workspace" in _msg(lib)
    assert lib.srm_htfa_factors(2, 5, 10, None, 4, 4, 4, P, P, P, P, None, P, need, None) == SRM_ERR_ARG


def test_empty_batches_launch_nothing(lib):
    # no CUDA call is made for these, so they succeed without a GPU
    assert lib.srm_htfa_factors(0, 5, 10, None, 4, 4, 4, None, None, None, None, None, None, 0, None) == SRM_OK
    assert lib.srm_htfa_factors(3, 5, 0, None, 4, 4, 4, None, None, None, None, None, None, 0, None) == SRM_OK
    assert lib.srm_htfa_residual(0, 5, 10, 10, None, None, None, None, None, 0, None) == SRM_OK
    assert lib.srm_zscore(0, 10, 10, None, None, None) == SRM_OK
    assert lib.srm_zscore(2, 0, 10, None, None, None) == SRM_OK


def test_residual_rejects_bad_arguments(lib):
    assert lib.srm_htfa_residual(-1, 5, 10, 10, P, P, P, P, P, 1 << 20, None) == SRM_ERR_ARG
    assert lib.srm_htfa_residual(1, 0, 10, 10, P, P, P, P, P, 1 << 20, None) == SRM_ERR_ARG
    assert lib.srm_htfa_residual(1, 5, 10, 10, P, P, P, None, P, 1 << 20, None) == SRM_ERR_ARG
    need = lib.srm_htfa_residual_workspace(1, 5, 10, 10)
    assert lib.srm_htfa_residual(1, 5, 10, 10, P, P, P, P, P, need - 1, None) == SRM_ERR_ARG
    assert lib.srm_htfa_residual(1, 5, 10, 10, P, P, P, P, ctypes.c_void_p(20), need, None) == SRM_ERR_ARG
    assert "workspace" in _msg(lib)


def test_zscore_rejects_bad_arguments(lib):
    assert lib.srm_zscore(-1, 10, 10, P, P, None) == SRM_ERR_ARG
    assert lib.srm_zscore(1, 10, 10, None, P, None) == SRM_ERR_ARG


def test_binding_requires_cuda_tensors():
    import torch

    from paper_1608_04647_gb300 import htfa
    X = torch.zeros((4, 5))
    with pytest.raises(ValueError, match="CUDA tensor"):
        htfa.residual(X, torch.zeros((4, 2)), torch.zeros((2, 5)))
    with pytest.raises(ValueError, match="CUDA tensor"):
        htfa.zscore(X)
    with pytest.raises(ValueError, match="CUDA tensor"):
        htfa.GridPositions([torch.zeros(3)] * 3, torch.zeros((5, 3), dtype=torch.int32))
