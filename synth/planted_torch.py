"""Device-side planted-data generator (PyTorch), for workloads too large to
draw on the host: same generative model and distributions as
``synth.planted`` (Sec. II-A, Eq. 1), drawn with torch's CUDA generator.
The values differ from the NumPy generator's (different random streams);
tests that compare against the oracle use the NumPy generator.
Nothing here computes an EM quantity."""
from __future__ import annotations

import math
from typing import List, Optional, Sequence

import numpy as np
import torch

from .planted import PlantedSpec, draw_voxel_counts, planted_rho2


def _orthonormal(v: int, k: int, gen: torch.Generator, device) -> torch.Tensor:
    """Q of the QR factorisation of a Gaussian v x k matrix with diag(R) > 0,
    computed as Cholesky-QR applied twice (the large products on the device,
    the k x k Cholesky factor on the host), so that no device linear-algebra
    library is needed."""
    q = torch.randn(v, k, generator=gen, device=device, dtype=torch.float32)
    for _ in range(2):
        g = (q.T.double() @ q.double()).cpu().numpy()
        r = np.linalg.cholesky(g).T  # upper, positive diagonal
        rinv = torch.from_numpy(np.linalg.inv(r)).to(device)
        q = (q.double() @ rinv).float()
    return q.contiguous()


def planted_dataset_torch(spec: PlantedSpec, voxel_counts: Optional[Sequence[int]] = None, device="cuda",
                          dtype=torch.float32, seed_offset: int = 0, keep_truth: bool = False,
                          subjects: Optional[Sequence[int]] = None):
    """X_i (v_i x T, `dtype`) and W0_i (v_i x k, float32) on `device`.

    Each subject is drawn from its own generator (seeded by the workload's
    seed, `seed_offset` and the subject's index) and S from another, so a
    process that holds only some subjects (`subjects`: their indices, in
    order) draws exactly those subjects of the whole workload."""
    vs = list(voxel_counts) if voxel_counts is not None else draw_voxel_counts(spec)
    idx = list(range(len(vs))) if subjects is None else [int(i) for i in subjects]
    base = 1_000_003 * (spec.seed + 1) + 7_919 * seed_offset
    gen = torch.Generator(device=device)
    gen.manual_seed(base)
    sd = torch.sqrt(torch.linspace(2.0, 0.5, spec.k, device=device))
    S = sd[:, None] * torch.randn(spec.k, spec.T, generator=gen, device=device)
    rho2_all = planted_rho2(spec)
    X: List[torch.Tensor] = []
    W0: List[torch.Tensor] = []
    Wt: List[torch.Tensor] = []
    for i in idx:
        v = vs[i]
        gen.manual_seed(base + 104_729 * (i + 1))
        W = _orthonormal(v, spec.k, gen, device)
        x = W @ S
        x += torch.randn(v, 1, generator=gen, device=device)
        x += math.sqrt(float(rho2_all[i])) * torch.randn(v, spec.T, generator=gen, device=device)
        X.append(x.to(dtype) if dtype != torch.float32 else x)
        if keep_truth:
            Wt.append(W)
        del W
        W0.append(_orthonormal(v, spec.k, gen, device))
    out = {"X": X, "W0": W0, "voxel_counts": [vs[i] for i in idx], "S_true": S,
           "rho2_true": torch.tensor(rho2_all[idx], device=device, dtype=torch.float32), "subjects": idx}
    if keep_truth:
        out["W_true"] = Wt
    return out
