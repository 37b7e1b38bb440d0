"""Plain, slow, FP64 NumPy oracle of the probabilistic SRM EM iteration.

TEST INFRASTRUCTURE ONLY: used by ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py``; never by the library.  It shares no
code with the CUDA path.

It follows the paper (Anderson et al., "Enabling Factor Analysis on
Thousand-Subject Neuroimaging Datasets", arXiv 1608.04647), Sec. II:

* model (Sec. II-A, Eq. 1): x_it = W_i s_t + mu_i + eps_it, W_i^T W_i = I,
  s_t ~ N(0, Sigma_s), eps_it ~ N(0, rho_i^2 I);
* E-step in the reduced form of Sec. II-C/II-D: eq:srm_inversion_opt,
  eq:srm_wt_psi_w (rho_0 = sum_i rho_i^-2) and eq:srm_mean_distributed;
* M-step: eq:srm_variance_update_optimized for Sigma_s, eq:srm_mapping_update
  for W_i (polar factor, here through an SVD of A_i) and eq:srm_rho_update
  for rho_i^2;
* loop order of Algorithm 1 (D-SRM): E-step reduction, E[S] on the master,
  Sigma_s and its trace, then W_i and rho_i^2 per subject.

Readings where the paper is silent or garbled (each one is listed with its
reason in the design notes of the repository):

* rho update (eq:srm_rho_update is garbled): rho_i^2 = (||X_i||_F^2
  - 2 tr(W_i^T A_i) + T tr Sigma_s^new) / (T v_i), the exact maximiser of the
  expected complete-data log-likelihood; V there is v_i.
* the 1/2 in A_i (eq:srm_mapping_update) is dropped: the polar factor is
  scale-free and the cross term of the rho update needs sum_t x_it E[s_t]^T.
* Sigma_s^0 = I_k (Algorithm 1 initialises only W_i and rho_i^2).
* log-likelihood (not in the paper): the Gaussian marginal likelihood of
  the demeaned data under N(0, W Sigma_s W^T + Psi), reduced with the
  Woodbury identity, the determinant lemma and eq:srm_wt_psi_w.
* stopping rule (not stated): a fixed number of iterations.

Everything is float64.  Subjects are processed one at a time.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Sequence

import numpy as np


# ---------------------------------------------------------------- centring
def center(X: np.ndarray):
    """Demean one subject over time (Algorithm 1 initialisation; Sec. II-B):
    mu_i = (1/T) sum_t x_it,  x^_it = x_it - mu_i.  Returns (X^, mu, ||X^||_F^2)."""
    X = np.asarray(X, dtype=np.float64)
    mu = X.mean(axis=1)
    Xh = X - mu[:, None]
    return Xh, mu, float(np.sum(Xh * Xh))


# ---------------------------------------------------------------- E-step
def estep(Xhat: Sequence[np.ndarray], W: Sequence[np.ndarray], rho2: np.ndarray,
          Sigma_s: np.ndarray):
    """Reduced E-step (Sec. II-C/II-D).

    y = sum_i rho_i^-2 W_i^T x^_i                          (the reduction, Alg. 1)
    rho_0 = sum_i rho_i^-2                                  (eq:srm_wt_psi_w)
    Phi = (Sigma_s^-1 + rho_0 I)^-1                         (eq:srm_inversion_opt)
    E[S] = Sigma_s^T [I - rho_0 Phi] y                      (eq:srm_mean_distributed)

    Returns a dict with y (k x T), rho0, Phi (k x k), ES (k x T).
    """
    rho2 = np.asarray(rho2, dtype=np.float64)
    k = Sigma_s.shape[0]
    T = Xhat[0].shape[1]
    y = np.zeros((k, T))
    for i in range(len(Xhat)):
        y += (1.0 / rho2[i]) * (W[i].T @ Xhat[i])
    rho0 = float(np.sum(1.0 / rho2))
    I = np.eye(k)
    Phi = np.linalg.inv(np.linalg.inv(Sigma_s) + rho0 * I)
    ES = Sigma_s.T @ (I - rho0 * Phi) @ y
    return {"y": y, "rho0": rho0, "Phi": Phi, "ES": ES}


def estep_dense(Xhat: Sequence[np.ndarray], W: Sequence[np.ndarray], rho2: np.ndarray,
                Sigma_s: np.ndarray):
    """Original (un-reduced) E-step, eq:srm_mean and eq:srm_var, with the
    V x V matrix W Sigma_s W^T + Psi formed and inverted.  Tiny inputs only.

    Returns ES (k x T), the stack E[s_t s_t^T] (T x k x k) and its mean.
    """
    Wst = np.vstack(W)
    Xst = np.vstack(Xhat)
    psi = np.concatenate([np.full(w.shape[0], r) for w, r in zip(W, rho2)])
    C = Wst @ Sigma_s @ Wst.T + np.diag(psi)
    Ci = np.linalg.inv(C)
    G = Sigma_s.T @ Wst.T @ Ci                       # k x V
    ES = G @ Xst
    post_var = Sigma_s - Sigma_s.T @ Wst.T @ Ci @ Wst @ Sigma_s
    T = Xst.shape[1]
    Ess = np.stack([post_var + np.outer(ES[:, t], ES[:, t]) for t in range(T)])
    return {"ES": ES, "Ess": Ess, "Ess_mean": Ess.mean(axis=0), "post_var": post_var}


def loglik(est: dict, sqnorms: Sequence[float], voxel_counts: Sequence[int],
           rho2: np.ndarray, Sigma_s: np.ndarray, T: int) -> float:
    """Log-likelihood of the demeaned data at the parameters the E-step used.

    x^_t ~ N(0, C), C = W Sigma_s W^T + Psi.  With Woodbury, the determinant
    lemma and W^T Psi^-1 W = rho_0 I (eq:srm_wt_psi_w):
      ln det C = sum_i v_i ln rho_i^2 + ln det(I + rho_0 Sigma_s)
      x^_t^T C^-1 x^_t = sum_i ||x^_it||^2 / rho_i^2 - y_t^T Phi y_t
    """
    rho2 = np.asarray(rho2, dtype=np.float64)
    k = Sigma_s.shape[0]
    V = float(np.sum(voxel_counts))
    sign, logdet = np.linalg.slogdet(np.eye(k) + est["rho0"] * Sigma_s)
    if sign <= 0:
        raise FloatingPointError("I + rho0 Sigma_s is not positive definite")
    quad = float(np.sum(np.asarray(sqnorms) / rho2)) - float(np.sum(est["y"] * (est["Phi"] @ est["y"])))
    return -0.5 * (T * V * math.log(2.0 * math.pi)
                   + T * float(np.sum(np.asarray(voxel_counts) * np.log(rho2)))
                   + T * logdet + quad)


def loglik_dense(Xhat: Sequence[np.ndarray], W: Sequence[np.ndarray], rho2: np.ndarray,
                 Sigma_s: np.ndarray) -> float:
    """The same log-likelihood from the V x V covariance (tiny inputs only)."""
    Wst = np.vstack(W)
    Xst = np.vstack(Xhat)
    psi = np.concatenate([np.full(w.shape[0], r) for w, r in zip(W, rho2)])
    C = Wst @ Sigma_s @ Wst.T + np.diag(psi)
    sign, logdet = np.linalg.slogdet(C)
    V, T = Xst.shape
    quad = float(np.sum(Xst * np.linalg.solve(C, Xst)))
    return -0.5 * (T * V * math.log(2.0 * math.pi) + T * logdet + quad)


# ---------------------------------------------------------------- M-step
def sigma_update(est: dict, T: int) -> np.ndarray:
    """eq:srm_variance_update_optimized:
    Sigma_s^new = (Sigma_s^-1 + rho_0 I)^-1 + (1/T) sum_t E[s_t] E[s_t]^T."""
    ES = est["ES"]
    return est["Phi"] + (ES @ ES.T) / T


def polar_factor(A: np.ndarray) -> np.ndarray:
    """W = A (A^T A)^-1/2 (eq:srm_mapping_update), computed as U V^T from the
    economy SVD A = U S V^T, the route the paper costs in Sec. V-A."""
    U, _, Vt = np.linalg.svd(A, full_matrices=False)
    return U @ Vt


def mstep(Xhat: Sequence[np.ndarray], sqnorms: Sequence[float], ES: np.ndarray,
          Sigma_new: np.ndarray):
    """Per-subject M-step (Alg. 1, last step of the loop body):
    A_i = sum_t x^_it E[s_t]^T, W_i = polar(A_i) (eq:srm_mapping_update),
    rho_i^2 = (||X^_i||_F^2 - 2 tr(W_i^T A_i) + T tr Sigma_s^new) / (T v_i)
    (eq:srm_rho_update as read above)."""
    T = ES.shape[1]
    trS = float(np.trace(Sigma_new))
    W, rho2 = [], []
    for i in range(len(Xhat)):
        A = Xhat[i] @ ES.T
        Wi = polar_factor(A)
        v = Xhat[i].shape[0]
        r = (sqnorms[i] - 2.0 * float(np.sum(Wi * A)) + T * trS) / (T * v)
        W.append(Wi)
        rho2.append(r)
    return W, np.array(rho2)


# ---------------------------------------------------------------- driver
@dataclasses.dataclass
class State:
    W: List[np.ndarray]
    rho2: np.ndarray
    Sigma_s: np.ndarray
    ES: Optional[np.ndarray] = None
    ll: List[float] = dataclasses.field(default_factory=list)


def fit(X: Sequence[np.ndarray], W0: Sequence[np.ndarray], n_iter: int,
        rho2_0: Optional[np.ndarray] = None, Sigma_0: Optional[np.ndarray] = None,
        final_ll: bool = False, centered: bool = False, callback=None) -> dict:
    """Algorithm 1 (D-SRM) on one machine.

    Initialisation: W_i = W0_i (given), rho_i^2 = 1, Sigma_s = I_k, data
    demeaned over time.  Each iteration: E-step (y, rho_0, Phi, E[S]; the
    log-likelihood of the current parameters is recorded), then Sigma_s and
    its trace, then W_i and rho_i^2.  ``final_ll`` adds the log-likelihood of
    the last parameters (one more E-step, whose E[S] is not kept).
    """
    if centered:
        Xh = [np.asarray(x, dtype=np.float64) for x in X]
        sq = [float(np.sum(x * x)) for x in Xh]
    else:
        Xh, sq = [], []
        for x in X:
            xh, _, s = center(x)
            Xh.append(xh)
            sq.append(s)
    N = len(Xh)
    k = W0[0].shape[1]
    T = Xh[0].shape[1]
    vs = [x.shape[0] for x in Xh]
    st = State(W=[np.asarray(w, dtype=np.float64) for w in W0],
               rho2=np.ones(N) if rho2_0 is None else np.asarray(rho2_0, dtype=np.float64).copy(),
               Sigma_s=np.eye(k) if Sigma_0 is None else np.asarray(Sigma_0, dtype=np.float64).copy())
    for it in range(n_iter):
        est = estep(Xh, st.W, st.rho2, st.Sigma_s)
        st.ll.append(loglik(est, sq, vs, st.rho2, st.Sigma_s, T))
        st.ES = est["ES"]
        st.Sigma_s = sigma_update(est, T)
        st.W, st.rho2 = mstep(Xh, sq, est["ES"], st.Sigma_s)
        if callback is not None:
            callback(it, st)
    if final_ll:
        est = estep(Xh, st.W, st.rho2, st.Sigma_s)
        st.ll.append(loglik(est, sq, vs, st.rho2, st.Sigma_s, T))
    return {"W": st.W, "rho2": st.rho2, "Sigma_s": st.Sigma_s, "ES": st.ES,
            "ll": np.array(st.ll), "sqnorms": np.array(sq)}


def transform(W_i: np.ndarray, X_new: np.ndarray) -> np.ndarray:
    """Map new data of subject i into the shared space: W_i^T (x - mean_t x)
    (the projection of Sec. II-A; new data are demeaned by their own
    temporal mean, as the training data are)."""
    Xh, _, _ = center(X_new)
    return W_i.T @ Xh


def map_subjects(W_i: np.ndarray, W_j: np.ndarray, X_new: np.ndarray) -> np.ndarray:
    """Map new data of subject i into subject j's voxel space through the
    shared space: W_j W_i^T (x - mean_t x) (Sec. II-A, the use the
    orthogonality of the mappings makes simple)."""
    return W_j @ transform(W_i, X_new)


# ---------------------------------------------------------------- special case
def ppca_fixed_point(Xhat: np.ndarray, k: int):
    """N = 1: the model is probabilistic PCA with orthonormal loadings
    (Tipping & Bishop 1999).  Its maximum-likelihood point, from the
    eigen-decomposition of the sample covariance (1/T) X^ X^^T:
    rho^2 = mean of the v-k smallest eigenvalues, span W = top-k
    eigenvectors, eig(Sigma_s) = top-k eigenvalues - rho^2."""
    v, T = Xhat.shape
    lam, U = np.linalg.eigh((Xhat @ Xhat.T) / T)
    lam, U = lam[::-1], U[:, ::-1]
    rho2 = float(np.mean(lam[k:]))
    return {"rho2": rho2, "U": U[:, :k], "sigma_eigs": lam[:k] - rho2, "eigs": lam}
