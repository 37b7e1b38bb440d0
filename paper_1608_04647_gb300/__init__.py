"""GB300 (sm_103a) probabilistic Shared Response Model EM (arXiv 1608.04647).

Thin ctypes binding over ``libsrm.so``, the C-ABI library declared in
``include/srm.h``.  Every step of the EM iteration runs in the library's CUDA
kernels; this module only marshals arguments.  PyTorch is used for device
memory (the caller's tensors) and streams.  There is no CPU fallback: if the
library is missing or its CUDA calls fail, the calls raise.

Low-level functions carry the C names (``srm_init``, ``srm_estep``,
``srm_mstep``, ``srm_fit``, ``srm_transform``, ...); :class:`SRM` wraps a
context for convenience.
"""
from __future__ import annotations

import ctypes
import os
from typing import List, Optional, Sequence

import numpy as np

from . import _build

__all__ = [
    "SRM", "SrmError", "load_library", "srm_config", "SRM_BATCHED", "SRM_GRAPH", "SRM_FINAL_LL",
    "SRM_HOST_INPUT", "SRM_PROFILE", "SRM_SINGLE_PASS", "SRM_F32", "SRM_BF16",
    "srm_init", "srm_estep", "srm_mstep", "srm_fit", "srm_transform", "srm_get_w", "srm_get_s",
    "srm_get_params", "srm_get_ll", "srm_synchronize", "srm_get_state", "srm_set_state",
    "srm_get_kernel_times", "srm_layout", "srm_last_error", "srm_destroy", "srm_debug_mma",
    "srm_transform_noalloc", "srm_debug_eig_sweeps", "srm_debug_force_eig_polar", "srm_debug_wait", "srm_map", "srm_plan", "srm_get_plan", "srm_set_plan",
    "srm_autotune", "srm_estep_partial", "srm_estep_finish",
]

SRM_OK, SRM_ERR_ARG, SRM_ERR_CUDA, SRM_ERR_NOMEM, SRM_ERR_NUMERIC, SRM_ERR_STATE, SRM_ERR_UNSUPPORTED = range(7)
STATUS_NAMES = {0: "SRM_OK", 1: "SRM_ERR_ARG", 2: "SRM_ERR_CUDA", 3: "SRM_ERR_NOMEM", 4: "SRM_ERR_NUMERIC",
                5: "SRM_ERR_STATE", 6: "SRM_ERR_UNSUPPORTED"}
SRM_F32, SRM_BF16 = 0, 1
SRM_BATCHED = 1 << 0
SRM_GRAPH = 1 << 1
SRM_FINAL_LL = 1 << 3
SRM_HOST_INPUT = 1 << 4
SRM_PROFILE = 1 << 5
SRM_SINGLE_PASS = 1 << 6


class SrmError(RuntimeError):
    def __init__(self, status: int, where: str, message: str):
        super().__init__(f"{where}: {STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


class srm_config(ctypes.Structure):
    _fields_ = [
        ("n_subjects", ctypes.c_int32),
        ("voxels", ctypes.POINTER(ctypes.c_int64)),
        ("T", ctypes.c_int32),
        ("k", ctypes.c_int32),
        ("in_dtype", ctypes.c_int),
        ("store_dtype", ctypes.c_int),
        ("flags", ctypes.c_uint32),
        ("max_iter", ctypes.c_int32),
        ("seed", ctypes.c_uint64),
    ]


class srm_plan(ctypes.Structure):
    """Launch plan of the batched form (field meanings in include/srm.h)."""
    _fields_ = [
        ("single_pass", ctypes.c_int32),
        ("e_reserve", ctypes.c_int32),
        ("m_stages", ctypes.c_int32),
        ("m_gram_bufs", ctypes.c_int32),
        ("m_resident_es", ctypes.c_int32),
        ("m_prefetch", ctypes.c_int32),
        ("f_prefetch", ctypes.c_int32),
        ("f_l2_hints", ctypes.c_int32),
        ("f_first_stages", ctypes.c_int32),
        ("f_reserve", ctypes.c_int32),
        ("m_boxes", ctypes.c_int32),
        ("f_lead", ctypes.c_int32),
        ("f_slots", ctypes.c_int32),
    ]

    def as_dict(self) -> dict:
        return {n: int(getattr(self, n)) for n, _ in self._fields_}


_lib = None
_P = ctypes.c_void_p


def load_library(path: Optional[str] = None):
    """Load libsrm.so (built in-tree by ``_build.build()``); raises if absent."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or _build.LIB
    if not os.path.exists(path):
        raise RuntimeError(f"libsrm.so not found at {path}; build it with paper_1608_04647_gb300._build.build()")
    lib = ctypes.CDLL(path)
    st = ctypes.c_int
    sig = {
        "srm_init": (st, [ctypes.POINTER(srm_config), ctypes.POINTER(_P), ctypes.POINTER(_P), _P,
                          ctypes.POINTER(_P)]),
        "srm_estep": (st, [_P]),
        "srm_mstep": (st, [_P]),
        "srm_estep_partial": (st, [_P, _P, _P]),
        "srm_estep_finish": (st, [_P, _P, _P]),
        "srm_fit": (st, [_P, ctypes.c_int32, ctypes.POINTER(ctypes.c_double)]),
        "srm_transform": (st, [_P, ctypes.c_int32, _P, ctypes.c_int32, _P]),
        "srm_get_w": (st, [_P, ctypes.c_int32, _P]),
        "srm_get_s": (st, [_P, _P]),
        "srm_get_params": (st, [_P, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]),
        "srm_get_ll": (st, [_P, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int32)]),
        "srm_synchronize": (st, [_P]),
        "srm_get_state": (st, [_P, _P, ctypes.POINTER(ctypes.c_size_t)]),
        "srm_set_state": (st, [_P, _P, ctypes.c_size_t]),
        "srm_get_kernel_times": (st, [_P, ctypes.POINTER(ctypes.c_char_p), ctypes.POINTER(ctypes.c_int64),
                                      ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int32),
                                      ctypes.c_int32]),
        "srm_layout": (st, [_P, ctypes.POINTER(ctypes.c_int64), ctypes.c_int32]),
        "srm_last_error": (ctypes.c_char_p, []),
        "srm_debug_mma": (st, [ctypes.c_int32, _P, _P, _P, ctypes.c_int32, ctypes.c_int32]),
        "srm_transform_noalloc": (st, [_P, ctypes.c_int32, _P, ctypes.c_int32, _P]),
        "srm_map": (st, [_P, ctypes.c_int32, ctypes.c_int32, _P, ctypes.c_int32, _P]),
        "srm_debug_eig_sweeps": (st, [_P, ctypes.POINTER(ctypes.c_int32), ctypes.c_int32]),
        "srm_debug_force_eig_polar": (st, [_P, ctypes.c_int32]),
        "srm_debug_wait": (st, [ctypes.c_int32]),
        "srm_get_plan": (st, [_P, ctypes.POINTER(srm_plan)]),
        "srm_set_plan": (st, [_P, ctypes.POINTER(srm_plan)]),
        "srm_autotune": (st, [_P, ctypes.c_char_p, ctypes.c_int32, ctypes.POINTER(srm_plan),
                              ctypes.POINTER(ctypes.c_double), ctypes.c_char_p, ctypes.c_size_t]),
        "srm_destroy": (None, [_P]),
        "srm_htfa_factors_workspace": (ctypes.c_size_t, [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                                         ctypes.c_int32, ctypes.c_int32]),
        "srm_htfa_factors": (st, [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, _P, ctypes.c_int32,
                                  ctypes.c_int32, ctypes.c_int32, _P, _P, _P, _P, _P, _P, ctypes.c_size_t, _P]),
        "srm_htfa_residual_workspace": (ctypes.c_size_t, [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                                          ctypes.c_int32]),
        "srm_htfa_residual": (st, [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, _P, _P, _P,
                                   _P, _P, ctypes.c_size_t, _P]),
        "srm_zscore": (st, [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, _P, _P, _P]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def srm_last_error() -> str:
    return load_library().srm_last_error().decode()


def _check(status: int, where: str):
    if status != SRM_OK:
        raise SrmError(status, where, srm_last_error())


# ---------------------------------------------------------------- C names
def srm_init(cfg: srm_config, X_ptrs: Sequence[int], W0_ptrs: Optional[Sequence[int]], stream: int = 0) -> int:
    """W0_ptrs None: the library draws a seeded random orthogonal W^0 (cfg.seed; include/srm.h)."""
    lib = load_library()
    n = len(X_ptrs)
    xa = (_P * n)(*X_ptrs)
    wa = (_P * n)(*W0_ptrs) if W0_ptrs is not None else None
    out = _P()
    _check(lib.srm_init(ctypes.byref(cfg), xa, wa, _P(stream or None), ctypes.byref(out)), "srm_init")
    return out.value


def srm_estep(ctx: int):
    _check(load_library().srm_estep(_P(ctx)), "srm_estep")


def srm_mstep(ctx: int):
    _check(load_library().srm_mstep(_P(ctx)), "srm_mstep")


def srm_estep_partial(ctx: int, y_ptr: int, sums_ptr: int):
    """This context's share of a sharded E-step (include/srm.h): y (k x T
    FP64) and the four sums over its subjects, both device buffers."""
    _check(load_library().srm_estep_partial(_P(ctx), _P(y_ptr), _P(sums_ptr)), "srm_estep_partial")


def srm_estep_finish(ctx: int, y_ptr: int, sums_ptr: int):
    """The rest of a sharded E-step from y and the sums totalled over all
    contexts (device buffers)."""
    _check(load_library().srm_estep_finish(_P(ctx), _P(y_ptr), _P(sums_ptr)), "srm_estep_finish")


def srm_fit(ctx: int, n_iter: int, n_out: int) -> np.ndarray:
    ll = np.zeros(max(n_out, 1), dtype=np.float64)
    _check(load_library().srm_fit(_P(ctx), n_iter, ll.ctypes.data_as(ctypes.POINTER(ctypes.c_double))), "srm_fit")
    return ll[:n_out]


def srm_fit_async(ctx: int, n_iter: int):
    _check(load_library().srm_fit(_P(ctx), n_iter, None), "srm_fit")


def srm_transform(ctx: int, subject: int, X_new_ptr: int, T_new: int, S_out_ptr: int):
    _check(load_library().srm_transform(_P(ctx), subject, _P(X_new_ptr), T_new, _P(S_out_ptr)), "srm_transform")


def srm_transform_noalloc(ctx: int, subject: int, X_new_ptr: int, T_new: int, S_out_ptr: int):
    """srm_transform for callers that must not allocate device memory: scratch
    comes from a fixed 16 MiB device array inside the library (see srm.h)."""
    _check(load_library().srm_transform_noalloc(_P(ctx), subject, _P(X_new_ptr), T_new, _P(S_out_ptr)),
           "srm_transform_noalloc")


def srm_map(ctx: int, src: int, dst: int, X_new_ptr: int, T_new: int, Y_out_ptr: int):
    _check(load_library().srm_map(_P(ctx), src, dst, _P(X_new_ptr), T_new, _P(Y_out_ptr)), "srm_map")


def srm_get_w(ctx: int, subject: int, W_ptr: int):
    _check(load_library().srm_get_w(_P(ctx), subject, _P(W_ptr)), "srm_get_w")


def srm_get_s(ctx: int, S_ptr: int):
    _check(load_library().srm_get_s(_P(ctx), _P(S_ptr)), "srm_get_s")


def srm_get_params(ctx: int, N: int, k: int):
    rho2 = np.zeros(N)
    sig = np.zeros((k, k))
    _check(load_library().srm_get_params(_P(ctx), rho2.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                         sig.ctypes.data_as(ctypes.POINTER(ctypes.c_double))), "srm_get_params")
    return rho2, sig


def srm_get_ll(ctx: int) -> np.ndarray:
    lib = load_library()
    n = ctypes.c_int32(0)
    _check(lib.srm_get_ll(_P(ctx), None, ctypes.byref(n)), "srm_get_ll")
    out = np.zeros(max(n.value, 1))
    m = ctypes.c_int32(n.value)
    _check(lib.srm_get_ll(_P(ctx), out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), ctypes.byref(m)),
           "srm_get_ll")
    return out[: n.value]


def srm_synchronize(ctx: int):
    _check(load_library().srm_synchronize(_P(ctx)), "srm_synchronize")


def srm_get_state(ctx: int) -> bytes:
    lib = load_library()
    nb = ctypes.c_size_t(0)
    _check(lib.srm_get_state(_P(ctx), None, ctypes.byref(nb)), "srm_get_state")
    buf = ctypes.create_string_buffer(nb.value)
    _check(lib.srm_get_state(_P(ctx), ctypes.cast(buf, _P), ctypes.byref(nb)), "srm_get_state")
    return buf.raw[: nb.value]


def srm_set_state(ctx: int, state: bytes):
    buf = ctypes.create_string_buffer(state, len(state))
    _check(load_library().srm_set_state(_P(ctx), ctypes.cast(buf, _P), len(state)), "srm_set_state")


def srm_get_kernel_times(ctx: int, reset: bool = False) -> dict:
    lib = load_library()
    n = ctypes.c_int32(64)
    names = (ctypes.c_char_p * 64)()
    launches = (ctypes.c_int64 * 64)()
    ms = (ctypes.c_double * 64)()
    _check(lib.srm_get_kernel_times(_P(ctx), names, launches, ms, ctypes.byref(n), int(reset)),
           "srm_get_kernel_times")
    return {names[j].decode(): (int(launches[j]), float(ms[j])) for j in range(n.value)}


def srm_layout(ctx: int) -> dict:
    out = (ctypes.c_int64 * 6)()
    _check(load_library().srm_layout(_P(ctx), out, 6), "srm_layout")
    keys = ["ldT", "kld", "rows_padded", "xhat_bytes", "a_bytes", "single_pass"]
    return dict(zip(keys, [int(x) for x in out]))


def srm_debug_mma(mn_major: int, A_ptr: int, B_ptr: int, D_ptr: int, N: int, K: int):
    """Self-test of the tensor-core building blocks (include/srm_debug.h)."""
    _check(load_library().srm_debug_mma(int(mn_major), _P(A_ptr), _P(B_ptr), _P(D_ptr), N, K), "srm_debug_mma")


def srm_debug_wait(arrive: bool):
    """The bounded wait of the tensor-core kernels on one CTA (include/srm_debug.h):
    raises SrmError(SRM_ERR_NUMERIC) when nothing arrives and the wait gives up."""
    _check(load_library().srm_debug_wait(1 if arrive else 0), "srm_debug_wait")


def srm_debug_eig_sweeps(ctx: int, n: int) -> np.ndarray:
    """Jacobi sweeps of the last M-step per matrix (subjects, then Sigma_s)."""
    out = np.zeros(n, dtype=np.int32)
    _check(load_library().srm_debug_eig_sweeps(_P(ctx), out.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), n),
           "srm_debug_eig_sweeps")
    return out


def srm_debug_force_eig_polar(ctx: int, on: bool) -> None:
    """Route every later polar factor through the eigen-decomposition path."""
    _check(load_library().srm_debug_force_eig_polar(_P(ctx), int(bool(on))), "srm_debug_force_eig_polar")


def srm_get_plan(ctx: int) -> srm_plan:
    p = srm_plan()
    _check(load_library().srm_get_plan(_P(ctx), ctypes.byref(p)), "srm_get_plan")
    return p


def srm_set_plan(ctx: int, plan: srm_plan):
    _check(load_library().srm_set_plan(_P(ctx), ctypes.byref(plan)), "srm_set_plan")


def srm_autotune(ctx: int, cache_path: Optional[str] = None, iters: int = 8):
    """Returns (chosen srm_plan, ms per EM iteration, text report of every timing)."""
    p = srm_plan()
    ms = ctypes.c_double(0)
    rep = ctypes.create_string_buffer(1 << 16)
    _check(load_library().srm_autotune(_P(ctx), cache_path.encode() if cache_path else None, int(iters),
                                       ctypes.byref(p), ctypes.byref(ms), rep, len(rep)), "srm_autotune")
    return p, float(ms.value), rep.value.decode()


def srm_destroy(ctx: int):
    load_library().srm_destroy(_P(ctx))


# ---------------------------------------------------------------- wrapper
def _check_buffers(m, y, sums):
    import torch
    if not (y.is_cuda and sums.is_cuda and y.dtype == torch.float64 and sums.dtype == torch.float64
            and y.is_contiguous() and tuple(y.shape) == (m.k, m.T) and sums.numel() >= 4):
        raise ValueError("sharded E-step buffers: y must be a contiguous CUDA float64 (k, T) tensor and sums a "
                         "CUDA float64 tensor of 4")


class SRM:
    """One pSRM context on the current CUDA device.

    X:   list of N subject matrices (v_i x T, row-major): torch CUDA tensors
         (float32 or bfloat16), or with ``host_input=True`` contiguous CPU
         tensors / NumPy arrays (pinned memory recommended).
    W0:  list of N torch CUDA float32 tensors (v_i x k) with orthonormal columns,
         or None: the library draws Algorithm 1's random orthogonal W^0 from
         `seed` (Philox4x64-10 normals, Q of their QR; see include/srm.h).
    store: "bf16" -> batched tensor-core form; "f32" -> plain per-subject form.
    single_pass: with store="bf16", k <= 64 and T <= 1024, stream X^ once per
         EM iteration (SRM_SINGLE_PASS); ignored elsewhere (see layout()).
    """

    def __init__(self, X: Sequence, W0: Sequence, k: int, store: str = "bf16", graph: bool = False,
                 final_ll: bool = False, profile: bool = False, host_input: bool = False,
                 max_iter: int = 1024, stream=None, single_pass: bool = False, seed: int = 0):
        import torch

        self.N = len(X)
        self.k = int(k)
        self.T = int(X[0].shape[1])
        self.voxels = [int(x.shape[0]) for x in X]
        self._vox = (ctypes.c_int64 * self.N)(*self.voxels)
        xdt = X[0].dtype
        in_dtype = SRM_BF16 if xdt in (torch.bfloat16,) else SRM_F32
        if host_input and isinstance(X[0], np.ndarray):
            in_dtype = SRM_F32
        flags = 0
        if store == "bf16":
            flags |= SRM_BATCHED
        if graph:
            flags |= SRM_GRAPH
        if final_ll:
            flags |= SRM_FINAL_LL
        if profile:
            flags |= SRM_PROFILE
        if host_input:
            flags |= SRM_HOST_INPUT
        if single_pass:
            flags |= SRM_SINGLE_PASS
        self.final_ll = final_ll
        self.cfg = srm_config(self.N, ctypes.cast(self._vox, ctypes.POINTER(ctypes.c_int64)), self.T, self.k,
                              in_dtype, SRM_BF16 if store == "bf16" else SRM_F32, flags, max_iter, int(seed))
        if host_input:
            xp = [x.ctypes.data if isinstance(x, np.ndarray) else x.data_ptr() for x in X]
        else:
            xp = [x.data_ptr() for x in X]
        wp = [w.data_ptr() for w in W0] if W0 is not None else None
        self._stream = stream
        s = stream.cuda_stream if stream is not None else 0
        self.ctx = srm_init(self.cfg, xp, wp, s)

    def estep(self):
        srm_estep(self.ctx)

    def mstep(self):
        srm_mstep(self.ctx)

    def shard_buffers(self):
        """Device buffers for a sharded E-step: y (k x T) and the 4 sums, FP64."""
        import torch
        return (torch.empty((self.k, self.T), dtype=torch.float64, device="cuda"),
                torch.empty(4, dtype=torch.float64, device="cuda"))

    def estep_partial(self, y, sums):
        """This context's share of a sharded E-step into the device tensors
        y (k x T) and sums (4), FP64 (see include/srm.h)."""
        _check_buffers(self, y, sums)
        srm_estep_partial(self.ctx, y.data_ptr(), sums.data_ptr())

    def estep_finish(self, y, sums):
        """Finish a sharded E-step from y and sums totalled over all contexts."""
        _check_buffers(self, y, sums)
        srm_estep_finish(self.ctx, y.data_ptr(), sums.data_ptr())

    def fit(self, n_iter: int) -> np.ndarray:
        return srm_fit(self.ctx, n_iter, n_iter + (1 if self.final_ll else 0))

    def fit_async(self, n_iter: int):
        srm_fit_async(self.ctx, n_iter)

    def synchronize(self):
        srm_synchronize(self.ctx)

    def get_w(self, i: int):
        import torch
        W = torch.empty((self.voxels[i], self.k), dtype=torch.float32, device="cuda")
        srm_get_w(self.ctx, i, W.data_ptr())
        self.synchronize()
        return W

    def get_s(self):
        import torch
        S = torch.empty((self.k, self.T), dtype=torch.float32, device="cuda")
        srm_get_s(self.ctx, S.data_ptr())
        self.synchronize()
        return S

    def params(self):
        return srm_get_params(self.ctx, self.N, self.k)

    def ll(self) -> np.ndarray:
        return srm_get_ll(self.ctx)

    def transform(self, i: int, X_new):
        import torch
        S = torch.empty((self.k, int(X_new.shape[1])), dtype=torch.float32, device="cuda")
        srm_transform(self.ctx, i, X_new.data_ptr(), int(X_new.shape[1]), S.data_ptr())
        self.synchronize()
        return S

    def map(self, i: int, j: int, X_new):
        """Subject i's new data in subject j's voxel space: W_j W_i^T (x - mean)."""
        import torch
        Y = torch.empty((self.voxels[j], int(X_new.shape[1])), dtype=torch.float32, device="cuda")
        srm_map(self.ctx, i, j, X_new.data_ptr(), int(X_new.shape[1]), Y.data_ptr())
        self.synchronize()
        return Y

    def state(self) -> bytes:
        return srm_get_state(self.ctx)

    def set_state(self, b: bytes):
        srm_set_state(self.ctx, b)

    def kernel_times(self, reset: bool = False) -> dict:
        return srm_get_kernel_times(self.ctx, reset)

    def layout(self) -> dict:
        return srm_layout(self.ctx)

    def plan(self) -> dict:
        return srm_get_plan(self.ctx).as_dict()

    def set_plan(self, **fields):
        p = srm_get_plan(self.ctx)
        for n, v in fields.items():
            setattr(p, n, int(v))
        srm_set_plan(self.ctx, p)

    def autotune(self, cache_path: Optional[str] = None, iters: int = 8):
        """Time candidate launch plans and keep the fastest (srm_autotune);
        returns (plan dict, ms per EM iteration, report text)."""
        p, ms, rep = srm_autotune(self.ctx, cache_path, iters)
        return p.as_dict(), ms, rep

    def close(self):
        if getattr(self, "ctx", None):
            srm_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
