"""Plain, slow, FP64 NumPy oracle of the HTFA local-step evaluations.

TEST INFRASTRUCTURE ONLY: used by ``tests/`` and the CPU-baseline leg of
``bench.py``; never by the library.  It shares no code with the CUDA path.

It follows the paper (Anderson et al., arXiv 1608.04647), Sec. III and the
list of native extension modules in Sec. IV-A:

* model (Sec. III-A, eq:htfa_factor_analysis): X_i = W_i F_i + E_i with
  X_i (T_i x V_i, one fMRI sample per row), W_i (T_i x K), F_i (K x V_i);
* factor matrix (Eq. 14, eq:htfa_factor): row k of F_i is the radial basis
  function exp(-||p - mu_{i,k}||^2 / lambda_{i,k}) evaluated at every voxel
  position p in R^3;
* residual: the Frobenius term ||X_i - W_i F_i||_F^2 of the local objective
  (eq:htfa_subject_update_rbfs), the quantity the NLLS solver evaluates for
  every trial of the centers and widths (Sec. III-B);
* z-score: the data standardisation of Sec. IV-A, applied per voxel over its
  T samples (a column of X_i).

Readings where the paper is silent (each listed with its reason in the
design notes of the repository):

* voxel positions lie on a grid: the coordinate of voxel v along each axis
  is one of that axis's n_x (n_y, n_z) distinct values (Sec. III-C: the
  number of distinct coordinates per axis is far below V_i).  The oracle
  takes the positions as a V x 3 array and does not use the grid;
* the z-score divides by the population standard deviation (divisor T) and
  maps a constant voxel to zeros.

Everything is float64.
"""
from __future__ import annotations

import numpy as np


def rbf_factors(positions, mu, lam):
    """F (K x V) with F[k, v] = exp(-||p_v - mu_k||^2 / lambda_k) (Eq. 14).

    positions: V x 3 voxel coordinates; mu: K x 3 centers; lam: K widths
    (lambda_k > 0).  The squared distance is summed over the three axes."""
    p = np.asarray(positions, dtype=np.float64)
    mu = np.asarray(mu, dtype=np.float64)
    lam = np.asarray(lam, dtype=np.float64)
    if np.any(~(lam > 0)):
        raise ValueError("widths must be positive")
    diff = p[None, :, :] - mu[:, None, :]          # K x V x 3
    dist2 = np.sum(diff * diff, axis=2)            # K x V
    return np.exp(-dist2 / lam[:, None])


def residual(X, W, F):
    """||X - W F||_F^2 (the Frobenius term of eq:htfa_subject_update_rbfs).

    X: T x V, W: T x K, F: K x V."""
    X = np.asarray(X, dtype=np.float64)
    R = X - np.asarray(W, dtype=np.float64) @ np.asarray(F, dtype=np.float64)
    return float(np.sum(R * R))


def residual_batch(X, W, F):
    """Residual of every subject of a batch (leading axis = subject)."""
    return np.array([residual(x, w, f) for x, w, f in zip(X, W, F)])


def zscore(X):
    """Each column of X (T x V; one voxel's samples) standardised to mean 0
    and unit population variance (Sec. IV-A, data standardisation).  A
    constant column becomes zeros."""
    X = np.asarray(X, dtype=np.float64)
    mean = X.mean(axis=0, keepdims=True)
    dev = X - mean
    std = np.sqrt((dev * dev).mean(axis=0, keepdims=True))
    out = np.zeros_like(X)
    varying = np.any(X != X[:1], axis=0)   # a column of equal values stays zero
    out[:, varying] = dev[:, varying] / std[:, varying]
    return out
