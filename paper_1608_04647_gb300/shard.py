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
