"""Seeded synthetic inputs for the HTFA local-step evaluations.

Shapes stand in for the paper's HTFA workloads (Sec. III, Sec. V):

* greeneyes-subsampled-like: 40 subjects of the greeneyes shape (42,855
  voxels, 475 TRs, Sec. V-B table) after the local step's random
  subsampling with replacement (Sec. V-A): per subject
  round((0.25 V + 3000) / 2) = 6,857 voxels and round((0.1 T + 300) / 2) =
  174 TRs; K = 100 factors (the K of the paper's Jacobian-size example);
* jacobian-example-like: one subject of V = 50,000 voxels, T = 2,000
  samples and K = 100 factors (the example of Sec. III-B);
* small cases that span several tiles with ragged edges, for parity.

Voxels lie on a 3 mm grid of 61 x 73 x 61 positions (the grid of a 3 mm
standard brain).  The brain is an ellipsoid in that grid whose semi-axes
are chosen to hold about as many voxels as the workload needs.  Centers are
drawn at random voxels plus a uniform offset of at most half a voxel.
Widths are drawn uniformly in [0.04 D, 1.8 D], with D the brain's diameter
in mm: the bounds of the constrained solver (Sec. III-C), read as bounds on
lambda itself.  Weights are standard normal and the noise is Gaussian.

Nothing here evaluates a factor, a residual or a z-score: the tests build
X = W F + noise with the oracle's F.
"""
from __future__ import annotations

import dataclasses
from typing import Dict, Tuple

import numpy as np

GRID = (61, 73, 61)
VOXEL_MM = 3.0


@dataclasses.dataclass(frozen=True)
class HtfaSpec:
    name: str
    n_subjects: int
    V: int          # voxels per subject (after subsampling)
    T: int          # samples per subject (after subsampling)
    K: int
    brain_voxels: int
    seed: int = 0
    with_replacement: bool = True  # the local step's subsample (Sec. V-A); else distinct voxels


def subsample_counts(V: int, T: int) -> Tuple[int, int]:
    """Sizes of the local step's random subsample (Sec. V-A): the mean of a
    percentage of the data (25 % of the voxels, 10 % of the TRs) and a cap
    (3000 voxels, 300 TRs)."""
    return int(round((0.25 * V + 3000) / 2)), int(round((0.1 * T + 300) / 2))


_GV, _GT = subsample_counts(42855, 475)

HTFA_CONFIGS: Dict[str, HtfaSpec] = {
    "greeneyes-subsampled-like": HtfaSpec("greeneyes-subsampled-like", 40, _GV, _GT, 100, 42855, 11),
    "jacobian-example-like": HtfaSpec("jacobian-example-like", 1, 50000, 2000, 100, 50000, 12, False),
    "ragged-small": HtfaSpec("ragged-small", 3, 700, 150, 37, 4000, 13),
}


def brain_mask(n_voxels: int) -> np.ndarray:
    """Grid indices (M x 3, int32, M >= n_voxels) of an ellipsoid centred in
    the grid, scaled until it holds at least n_voxels positions."""
    g = np.stack(np.meshgrid(*[np.arange(s) for s in GRID], indexing="ij"), axis=-1).reshape(-1, 3)
    c = (np.array(GRID) - 1) / 2.0
    shape = np.array([0.80, 1.00, 0.72])
    lo, hi = 1.0, float(max(GRID))
    for _ in range(60):
        r = 0.5 * (lo + hi)
        inside = np.sum(((g - c) / (r * shape)) ** 2, axis=1) <= 1.0
        if inside.sum() >= n_voxels:
            hi = r
        else:
            lo = r
    inside = np.sum(((g - c) / (hi * shape)) ** 2, axis=1) <= 1.0
    return g[inside].astype(np.int32)


def grid_axes() -> Tuple[np.ndarray, np.ndarray, np.ndarray]:
    """Coordinates (mm, float32) of the grid positions along x, y, z."""
    return tuple((np.arange(s, dtype=np.float64) * VOXEL_MM - 0.5 * (s - 1) * VOXEL_MM).astype(np.float32)
                 for s in GRID)


def draw(spec: HtfaSpec, noise: float = 0.5) -> Dict[str, np.ndarray]:
    """axes (3 arrays), vox [n, V, 3] int32, positions [n, V, 3] float32 (the
    voxels' coordinates, read off the axes), mu [n, K, 3], lam [n, K],
    W [n, T, K] and E [n, T, V] (noise of standard deviation ``noise``),
    all float32."""
    rng = np.random.default_rng(np.random.SeedSequence(spec.seed))
    mask = brain_mask(spec.brain_voxels)
    axes = grid_axes()
    ext = np.array([(axes[a][mask[:, a]].max() - axes[a][mask[:, a]].min()) for a in range(3)])
    diam = float(ext.max())
    n, V, T, K = spec.n_subjects, spec.V, spec.T, spec.K
    vox = np.empty((n, V, 3), np.int32)
    pos = np.empty((n, V, 3), np.float32)
    mu = np.empty((n, K, 3), np.float32)
    for i in range(n):
        if spec.with_replacement:
            pick = rng.integers(0, len(mask), size=V)
        else:
            pick = np.sort(rng.choice(len(mask), size=V, replace=False))
        vox[i] = mask[pick]
        pos[i] = np.stack([axes[a][vox[i, :, a]] for a in range(3)], axis=1)
        cen = mask[rng.integers(0, len(mask), size=K)]
        mu[i] = np.stack([axes[a][cen[:, a]] for a in range(3)], axis=1) + \
            rng.uniform(-0.5 * VOXEL_MM, 0.5 * VOXEL_MM, size=(K, 3))
    lam = rng.uniform(0.04 * diam, 1.8 * diam, size=(n, K)).astype(np.float32)
    W = rng.standard_normal((n, T, K), dtype=np.float32)
    E = (noise * rng.standard_normal((n, T, V), dtype=np.float32)).astype(np.float32)
    return {"axes": axes, "vox": vox, "positions": pos, "mu": mu.astype(np.float32), "lam": lam, "W": W, "E": E,
            "diameter": diam}
