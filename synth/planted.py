"""Planted-data generator for the probabilistic Shared Response Model.

The generative model is the one of Sec. II-A (Eq. 1): every subject i sees
the same shared response ``s_t ~ N(0, Sigma_s)`` through its own orthonormal
mapping ``W_i`` (v_i x k), plus a per-voxel mean ``mu_i`` and isotropic noise
of variance ``rho_i^2``:

    x_it = W_i s_t + mu_i + eps_it,   eps_it ~ N(0, rho_i^2 I),  W_i^T W_i = I.

The paper's datasets (raider, greeneyes, forrest, Sec. V-B) are not
available; the shapes below stand in for them:

* small raider-like correctness case (4 subjects x 2000 voxels, 300 TRs);
* greeneyes-like voxel counts (U[20000, 60000]) with T = 1000 or T = 500;
* forrest-like high resolution (600000 voxels, 3500 TRs, Sec. V-B Tab. I);
* forrest-1024-like subject count (1024 subjects, Sec. V-C).

Random draws use NumPy's ``default_rng`` with one child stream per subject
spawned from ``SeedSequence(seed)``, so any one subject can be regenerated
alone.  Nothing in this module computes an EM quantity.
"""
from __future__ import annotations

import dataclasses
from typing import List, Optional, Sequence, Tuple

import numpy as np


@dataclasses.dataclass(frozen=True)
class PlantedSpec:
    """Shape and distribution of one synthetic workload."""

    name: str
    n_subjects: int
    voxels: Tuple[str, float, float]  # ("fixed", v, v) | ("uniform", lo, hi) | ("loguniform", lo, hi)
    T: int
    k: int
    n_iter: int
    rho2_range: Tuple[float, float] = (0.1, 1.0)
    seed: int = 0


# The five workloads (index = seed).  Voxel counts are drawn per subject.
CONFIGS: List[PlantedSpec] = [
    PlantedSpec("raider-like N=4 v=2000 T=300 k=10", 4, ("fixed", 2000, 2000), 300, 10, 10, (0.1, 1.0), 0),
    PlantedSpec("greeneyes-like N=16 v~U[2e4,6e4] T=1000 k=50", 16, ("uniform", 20000, 60000), 1000, 50, 20, (0.1, 1.0), 1),
    PlantedSpec("batched N=64 v~logU[1e4,2e5] T=1000 k=50", 64, ("loguniform", 10000, 200000), 1000, 50, 10, (0.1, 1.0), 2),
    PlantedSpec("forrest-like N=8 v=600000 T=3500 k=100", 8, ("fixed", 600000, 600000), 3500, 100, 10, (0.5, 2.0), 3),
    PlantedSpec("forrest-1024-like N=1024 v~U[2e4,6e4] T=500 k=50", 1024, ("uniform", 20000, 60000), 500, 50, 10, (0.1, 1.0), 4),
]


def config_spec(index: int) -> PlantedSpec:
    return CONFIGS[index]


def _rng(seed: int, *path: int) -> np.random.Generator:
    """Child generator for a (seed, path...) address; independent streams."""
    ss = np.random.SeedSequence(entropy=seed, spawn_key=tuple(int(p) for p in path))
    return np.random.default_rng(ss)


def draw_voxel_counts(spec: PlantedSpec) -> List[int]:
    """Per-subject voxel counts v_i (uneven where the spec says so)."""
    kind, lo, hi = spec.voxels
    rng = _rng(spec.seed, 0)
    if kind == "fixed":
        return [int(lo)] * spec.n_subjects
    if kind == "uniform":
        return [int(x) for x in rng.integers(int(lo), int(hi) + 1, size=spec.n_subjects)]
    if kind == "loguniform":
        u = rng.uniform(np.log(lo), np.log(hi), size=spec.n_subjects)
        return [int(round(x)) for x in np.exp(u)]
    raise ValueError(kind)


def random_orthonormal(rng: np.random.Generator, v: int, k: int) -> np.ndarray:
    """A v x k matrix with orthonormal columns: Q of the QR factorisation of a
    standard Gaussian matrix, with column signs chosen so that diag(R) > 0.
    (Alg. 1 initialises W_i 'to a random orthogonal matrix' without naming the
    distribution; this is the Haar-distributed choice.)"""
    g = rng.standard_normal((v, k))
    q, r = np.linalg.qr(g)
    s = np.sign(np.diag(r))
    s[s == 0] = 1.0
    return q * s[None, :]


def shared_response(spec: PlantedSpec, T: Optional[int] = None) -> np.ndarray:
    """S (k x T) with rows drawn from N(0, diag(linspace(2, 0.5, k)))."""
    T = spec.T if T is None else T
    rng = _rng(spec.seed, 1)
    sd = np.sqrt(np.linspace(2.0, 0.5, spec.k))
    return sd[:, None] * rng.standard_normal((spec.k, T))


def planted_rho2(spec: PlantedSpec) -> np.ndarray:
    rng = _rng(spec.seed, 2)
    lo, hi = spec.rho2_range
    return rng.uniform(lo, hi, size=spec.n_subjects)


def planted_subject(spec: PlantedSpec, i: int, v: int, S: np.ndarray, rho2_i: float,
                    dtype=np.float64) -> Tuple[np.ndarray, np.ndarray]:
    """Subject i's raw data X_i (v x T) and its true mapping W_i (v x k)."""
    rng = _rng(spec.seed, 3, i)
    W = random_orthonormal(rng, v, spec.k)
    mu = rng.standard_normal(v)
    noise = rng.standard_normal((v, S.shape[1]))
    X = W @ S + mu[:, None] + np.sqrt(rho2_i) * noise
    return X.astype(dtype, copy=False), W


def initial_mappings(seed: int, voxel_counts: Sequence[int], k: int) -> List[np.ndarray]:
    """Random orthonormal starting mappings W_i^0 (Alg. 1 initialisation),
    drawn from a stream separate from the planted truth."""
    return [random_orthonormal(_rng(seed, 4, i), int(v), k) for i, v in enumerate(voxel_counts)]


def planted_dataset(spec: PlantedSpec, voxel_counts: Optional[Sequence[int]] = None,
                    T: Optional[int] = None, dtype=np.float64):
    """Whole planted dataset on the host.

    Returns a dict with X (list of v_i x T), W_true, S_true (k x T),
    rho2_true (N,), W0 (list of v_i x k), voxel_counts.
    """
    vs = list(voxel_counts) if voxel_counts is not None else draw_voxel_counts(spec)
    S = shared_response(spec, T)
    rho2 = planted_rho2(spec)
    if len(rho2) < len(vs):
        raise ValueError("more voxel counts than subjects")
    X, Wt = [], []
    for i, v in enumerate(vs):
        x, w = planted_subject(spec, i, v, S, float(rho2[i]), dtype)
        X.append(x)
        Wt.append(w)
    W0 = initial_mappings(spec.seed, vs, spec.k)
    return {"X": X, "W_true": Wt, "S_true": S, "rho2_true": rho2[: len(vs)],
            "W0": W0, "voxel_counts": vs}
