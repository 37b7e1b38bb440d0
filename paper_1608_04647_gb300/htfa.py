"""Python binding of the HTFA local-step evaluations in libsrm (include/htfa.h).

Argument marshalling only: every step runs in the library's CUDA kernels,
and a missing library raises.  Shapes follow the paper's HTFA notation
(Sec. III-A): X_i is T x V (one sample per row), W_i is T x K, F_i is K x V.
Every function takes one subject (2-D arrays) or a batch of equal-sized
subjects (a leading batch axis).

* ``factors``  -- F_i of Eq. 14 from grid voxel positions, centers, widths;
* ``residual`` -- ||X_i - W_i F_i||_F^2 (Frobenius term of
  eq:htfa_subject_update_rbfs);
* ``zscore``   -- per-voxel standardisation (Sec. IV-A).
"""
from __future__ import annotations

from typing import Optional, Sequence

import torch

from . import SrmError, _check, load_library  # noqa: F401

__all__ = ["GridPositions", "factors", "factors_workspace", "residual", "residual_workspace", "zscore",
           "FLAG_BAD_VOXEL", "FLAG_BAD_WIDTH"]

FLAG_BAD_VOXEL = 1
FLAG_BAD_WIDTH = 2


def _stream(t: torch.Tensor) -> int:
    return torch.cuda.current_stream(t.device).cuda_stream


def _need(t: torch.Tensor, name: str, dtype: torch.dtype, dims: Sequence[int]):
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise ValueError(f"{name} must be {dtype}, got {t.dtype}")
    if t.dim() not in dims:
        raise ValueError(f"{name} must have {' or '.join(map(str, dims))} dimensions, got {t.dim()}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")


class GridPositions:
    """Voxel positions on a grid (Sec. III-C): the distinct coordinates along
    each axis and, per voxel, its index along each axis.

    axes: three 1-D float32 arrays (x, y, z coordinates); vox: int32
    [V, 3] or [n, V, 3] indices into them."""

    def __init__(self, axes: Sequence[torch.Tensor], vox: torch.Tensor):
        if len(axes) != 3:
            raise ValueError("need three axes")
        dev = vox.device
        self.n_axis = tuple(int(a.numel()) for a in axes)
        self.axes = torch.cat([a.reshape(-1).to(device=dev, dtype=torch.float32) for a in axes]).contiguous()
        _need(vox, "vox", torch.int32, (2, 3))
        if vox.shape[-1] != 3:
            raise ValueError("vox must end in an axis of 3 indices")
        self.vox = vox


def factors(grid: GridPositions, mu: torch.Tensor, lam: torch.Tensor, out: Optional[torch.Tensor] = None,
            flag: Optional[torch.Tensor] = None, work: Optional[torch.Tensor] = None) -> torch.Tensor:
    """F (K x V, or n x K x V) with F[k][v] = exp(-||p_v - mu_k||^2 / lambda_k).

    mu: [K, 3] or [n, K, 3]; lam: [K] or [n, K]; flag: optional int32
    device tensor of one element, OR-ed with FLAG_BAD_VOXEL / FLAG_BAD_WIDTH.
    ``work`` (float64 device tensor of ``factors_workspace(...)`` bytes) may
    be given instead of the cached scratch buffer."""
    lib = load_library()
    batched = grid.vox.dim() == 3
    _need(mu, "mu", torch.float32, (3,) if batched else (2,))
    _need(lam, "lam", torch.float32, (2,) if batched else (1,))
    n = grid.vox.shape[0] if batched else 1
    V = grid.vox.shape[-2]
    K = mu.shape[-2]
    if mu.shape[-1] != 3 or tuple(lam.shape) != tuple(mu.shape[:-1]) or (batched and mu.shape[0] != n):
        raise ValueError("mu must be [..., K, 3] and lam [..., K] with the batch of vox")
    shape = (n, K, V) if batched else (K, V)
    if out is None:
        out = torch.empty(shape, device=mu.device, dtype=torch.float32)
    else:
        _need(out, "out", torch.float32, (len(shape),))
        if tuple(out.shape) != shape:
            raise ValueError(f"out must be {shape}")
    fptr = None
    if flag is not None:
        _need(flag, "flag", torch.int32, (0, 1))
        fptr = flag.data_ptr()
    nx, ny, nz = grid.n_axis
    nbytes = lib.srm_htfa_factors_workspace(n, K, nx, ny, nz)
    work = _scratch(work, mu.device, nbytes, "factors")
    _check(lib.srm_htfa_factors(n, K, V, grid.axes.data_ptr(), nx, ny, nz, grid.vox.data_ptr(), mu.data_ptr(),
                                lam.data_ptr(), out.data_ptr(), fptr, work.data_ptr(), work.numel() * 8,
                                _stream(mu)), "srm_htfa_factors")
    return out


def factors_workspace(n: int, K: int, n_axis) -> int:
    """Bytes of scratch ``factors`` needs (n subjects, K factors, axis sizes)."""
    return int(load_library().srm_htfa_factors_workspace(n, K, *n_axis))


_work_cache = {}


def _scratch(work: Optional[torch.Tensor], device: torch.device, nbytes: int, use: str) -> torch.Tensor:
    """The caller's scratch tensor, checked, or a cached one per device and
    use (not safe for concurrent calls on several streams: pass ``work``)."""
    if work is not None:
        if work.dtype != torch.float64 or not work.is_cuda or work.numel() * 8 < nbytes:
            raise ValueError(f"work must be a float64 CUDA tensor of at least {nbytes} bytes")
        return work
    key = (device.type, device.index, use)
    buf = _work_cache.get(key)
    if buf is None or buf.numel() * 8 < nbytes:
        buf = torch.empty(max(1, (nbytes + 7) // 8), device=device, dtype=torch.float64)
        _work_cache[key] = buf
    return buf


def residual(X: torch.Tensor, W: torch.Tensor, F: torch.Tensor, out: Optional[torch.Tensor] = None,
             work: Optional[torch.Tensor] = None) -> torch.Tensor:
    """||X - W F||_F^2 per subject, as a float64 device tensor ([] or [n]).

    X: [T, V] or [n, T, V]; W: [T, K] / [n, T, K]; F: [K, V] / [n, K, V].
    ``work`` (float64 device tensor) may be given to avoid the cached
    scratch buffer; it must hold ``residual_workspace(...)`` bytes."""
    lib = load_library()
    _need(X, "X", torch.float32, (2, 3))
    batched = X.dim() == 3
    _need(W, "W", torch.float32, (X.dim(),))
    _need(F, "F", torch.float32, (X.dim(),))
    n = X.shape[0] if batched else 1
    T, V = X.shape[-2], X.shape[-1]
    K = W.shape[-1]
    if W.shape[-2] != T or tuple(F.shape[-2:]) != (K, V) or (batched and (W.shape[0] != n or F.shape[0] != n)):
        raise ValueError(f"shapes do not chain: X {tuple(X.shape)}, W {tuple(W.shape)}, F {tuple(F.shape)}")
    if out is None:
        out = torch.empty((n,) if batched else (), device=X.device, dtype=torch.float64)
    nbytes = lib.srm_htfa_residual_workspace(n, K, T, V)
    work = _scratch(work, X.device, nbytes, "residual")
    _check(lib.srm_htfa_residual(n, K, T, V, X.data_ptr(), W.data_ptr(), F.data_ptr(), out.data_ptr(),
                                 work.data_ptr(), work.numel() * 8, _stream(X)), "srm_htfa_residual")
    return out


def residual_workspace(n: int, K: int, T: int, V: int) -> int:
    """Bytes of scratch ``residual`` needs for n subjects of T x V."""
    return int(load_library().srm_htfa_residual_workspace(n, K, T, V))


def zscore(X: torch.Tensor, out: Optional[torch.Tensor] = None) -> torch.Tensor:
    """Every column of X ([T, V] or [n, T, V]) standardised over its T
    samples (population variance); constant columns become zeros.  ``out``
    may be X itself."""
    lib = load_library()
    _need(X, "X", torch.float32, (2, 3))
    if out is None:
        out = torch.empty_like(X)
    else:
        _need(out, "out", torch.float32, (X.dim(),))
        if out.shape != X.shape:
            raise ValueError("out must have the shape of X")
    n = X.shape[0] if X.dim() == 3 else 1
    _check(lib.srm_zscore(n, X.shape[-2], X.shape[-1], X.data_ptr(), out.data_ptr(), _stream(X)), "srm_zscore")
    return out

