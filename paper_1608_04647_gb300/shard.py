"""Subject sharding for a multi-GPU run of the EM iteration (host logic).

Algorithm 1 (D-SRM) distributes subjects over processes; its only exchange
per iteration is the reduction of the k x T matrix y = sum_i rho_i^-2
W_i^T X_i together with N scalars (rho_i^2 and the likelihood terms), after
which every process can form Phi, E[S] and Sigma_s itself.  This module
assigns subjects to ranks so that every rank streams about the same number
of bytes (v_i x T elements), largest subjects first onto the least-loaded
rank; ties go to the lowest rank, so every process computes the same plan.
"""
from __future__ import annotations

import heapq
from typing import List, Sequence


def shard_subjects(voxels: Sequence[int], world: int) -> List[List[int]]:
    """Subject indices per rank (each list in increasing subject order)."""
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(voxels)), key=lambda i: (-int(voxels[i]), i))
    heap = [(0, r) for r in range(world)]
    heapq.heapify(heap)
    out: List[List[int]] = [[] for _ in range(world)]
    for i in order:
        load, r = heapq.heappop(heap)
        out[r].append(i)
        heapq.heappush(heap, (load + int(voxels[i]), r))
    return [sorted(x) for x in out]


def imbalance(voxels: Sequence[int], plan: List[List[int]]) -> float:
    """max rank load / mean rank load (1.0 = perfectly balanced)."""
    loads = [sum(int(voxels[i]) for i in p) for p in plan]
    mean = sum(loads) / len(loads)
    return max(loads) / mean if mean > 0 else 1.0


def fit_sharded(model, n_iter: int, all_reduce) -> None:
    """Algorithm 1 (D-SRM) with this process's subjects in `model`: per
    iteration, this process's share of the E-step (``estep_partial``: y and
    the four sums over its subjects), one sum over all processes of each
    (``all_reduce``, in place: the paper's Reduce, which every process
    receives, so no Bcast follows), the rest of the E-step from the totals
    (``estep_finish``) and the M-step of its own subjects (``mstep``).

    ``model`` is an :class:`~paper_1608_04647_gb300.SRM` context over this
    process's subjects, or any object with the same members (``shard_buffers``,
    ``estep_partial``, ``estep_finish``, ``mstep``).  For a context the
    reduction is ordered after the E-pass on the context's stream: the
    context's stream is made current for ``all_reduce`` (NCCL's
    ``torch.distributed.all_reduce`` waits for that stream), and a context on
    a library-owned stream is synchronised first."""
    y, sums = model.shard_buffers()
    stream = getattr(model, "_stream", None)
    on_gpu = getattr(y, "is_cuda", False)
    for _ in range(n_iter):
        model.estep_partial(y, sums)
        if on_gpu and stream is not None:
            import torch
            with torch.cuda.stream(stream):
                all_reduce(y)
                all_reduce(sums)
        elif on_gpu:
            import torch
            model.synchronize()
            all_reduce(y)
            all_reduce(sums)
            torch.cuda.current_stream().synchronize()
        else:
            all_reduce(y)
            all_reduce(sums)
        model.estep_finish(y, sums)
        model.mstep()
