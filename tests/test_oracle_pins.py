"""Pins of the FP64 oracle against what the paper and the mathematics fix.

None of these tests re-types an oracle formula: each one checks the oracle
against a different route to the same quantity (the dense V x V E-step of
eq:srm_mean / eq:srm_var, the slogdet of the full covariance, an SVD-free
polar factor, brute-force maximisation of the EM objective, the PPCA closed
form, invariances, a hand-derived example).
"""
import math

import numpy as np
import pytest

import oracle
import synth


def _rand_problem(seed, vs=(30, 40, 50), T=25, k=4):
    rng = np.random.default_rng(seed)
    W = [synth.random_orthonormal(rng, v, k) for v in vs]
    rho2 = rng.uniform(0.3, 2.0, size=len(vs))
    B = rng.standard_normal((k, k))
    Sigma = B @ B.T + 0.5 * np.eye(k)
    X = [rng.standard_normal((v, T)) * 1.5 + rng.standard_normal((v, 1)) for v in vs]
    Xh = [oracle.center(x)[0] for x in X]
    return Xh, W, rho2, Sigma


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_reduced_estep_equals_dense(seed):
    """eq:srm_mean_distributed (reduced) == eq:srm_mean (V x V inverse)."""
    Xh, W, rho2, Sigma = _rand_problem(seed)
    red = oracle.estep(Xh, W, rho2, Sigma)
    den = oracle.estep_dense(Xh, W, rho2, Sigma)
    np.testing.assert_allclose(red["ES"], den["ES"], rtol=0, atol=1e-10 * np.abs(den["ES"]).max())
    # eq:srm_inversion_opt: posterior covariance == Phi
    np.testing.assert_allclose(red["Phi"], den["post_var"], rtol=0, atol=1e-10)


@pytest.mark.parametrize("seed", [3, 4])
def test_sigma_update_equals_mean_of_stack(seed):
    """eq:srm_variance_update_optimized == (1/T) sum_t E[s_t s_t^T] of eq:srm_var."""
    Xh, W, rho2, Sigma = _rand_problem(seed)
    T = Xh[0].shape[1]
    red = oracle.estep(Xh, W, rho2, Sigma)
    den = oracle.estep_dense(Xh, W, rho2, Sigma)
    np.testing.assert_allclose(oracle.sigma_update(red, T), den["Ess_mean"], rtol=0, atol=1e-10)
    # the trace identity of Sec. II-D
    assert abs(np.trace(oracle.sigma_update(red, T)) - np.mean([np.trace(m) for m in den["Ess"]])) < 1e-10


@pytest.mark.parametrize("seed", [5, 6])
def test_reduced_loglik_equals_dense(seed):
    Xh, W, rho2, Sigma = _rand_problem(seed)
    T = Xh[0].shape[1]
    red = oracle.estep(Xh, W, rho2, Sigma)
    sq = [float(np.sum(x * x)) for x in Xh]
    vs = [x.shape[0] for x in Xh]
    ll = oracle.loglik(red, sq, vs, rho2, Sigma, T)
    lld = oracle.loglik_dense(Xh, W, rho2, Sigma)
    assert abs(ll - lld) <= 1e-10 * abs(lld)


def test_polar_factor_matches_inverse_sqrt_route():
    """eq:srm_mapping_update: U V^T from the SVD equals A (A^T A)^-1/2 formed
    from an eigen-decomposition, is orthonormal (Sec. II-A) and maximises
    tr(W^T A) over orthonormal W (orthogonal Procrustes)."""
    rng = np.random.default_rng(7)
    A = rng.standard_normal((60, 6)) @ np.diag([5, 4, 3, 2, 1, 0.5])
    W = oracle.polar_factor(A)
    lam, U = np.linalg.eigh(A.T @ A)
    W2 = A @ (U @ np.diag(lam ** -0.5) @ U.T)
    np.testing.assert_allclose(W, W2, atol=1e-12)
    np.testing.assert_allclose(W.T @ W, np.eye(6), atol=1e-12)
    best = np.sum(W * A)
    assert abs(best - np.linalg.svd(A, compute_uv=False).sum()) < 1e-10
    for _ in range(20):
        Q = synth.random_orthonormal(rng, 60, 6)
        assert np.sum(Q * A) <= best + 1e-12


def _expected_complete_ll(Xh_i, W_i, rho2_i, ES, Ess):
    """Subject i's part of the EM Q-function, from the per-t posterior
    moments of the dense E-step:  -(T v/2) ln rho^2 - (1/(2 rho^2)) sum_t
    E||x_t - W s_t||^2, with E||x - W s||^2 = ||x||^2 - 2 x^T W E[s]
    + tr(W^T W E[s s^T])."""
    v, T = Xh_i.shape
    tot = 0.0
    for t in range(T):
        x = Xh_i[:, t]
        tot += x @ x - 2 * x @ (W_i @ ES[:, t]) + np.trace(W_i.T @ W_i @ Ess[t])
    return -0.5 * T * v * math.log(rho2_i) - tot / (2 * rho2_i), tot / (T * v)


@pytest.mark.parametrize("seed", [8, 9])
def test_mstep_maximises_q(seed):
    """eq:srm_mapping_update and eq:srm_rho_update (as read: V -> v_i, the
    cross term inside the 1/(T v_i), no 1/2 in A_i) maximise the expected
    complete-data log-likelihood; brute-force check with the dense E-step's
    per-t moments and perturbed parameters."""
    Xh, W, rho2, Sigma = _rand_problem(seed)
    T = Xh[0].shape[1]
    red = oracle.estep(Xh, W, rho2, Sigma)
    den = oracle.estep_dense(Xh, W, rho2, Sigma)
    Sig_new = oracle.sigma_update(red, T)
    sq = [float(np.sum(x * x)) for x in Xh]
    Wn, rn = oracle.mstep(Xh, sq, red["ES"], Sig_new)
    rng = np.random.default_rng(seed)
    for i in range(len(Xh)):
        q0, rho_direct = _expected_complete_ll(Xh[i], Wn[i], rn[i], den["ES"], den["Ess"])
        # rho^2 from the per-t sum equals the trace-shortcut update
        assert abs(rho_direct - rn[i]) <= 1e-10 * rn[i]
        for f in (0.97, 1.03):
            assert _expected_complete_ll(Xh[i], Wn[i], rn[i] * f, den["ES"], den["Ess"])[0] < q0
        # a rotated or perturbed orthonormal W does worse
        k = Wn[i].shape[1]
        Ksk = rng.standard_normal((k, k)) * 0.05
        Ksk = Ksk - Ksk.T
        lam, U = np.linalg.eigh(1j * Ksk)
        R = np.real(U @ np.diag(np.exp(-1j * lam)) @ U.conj().T)
        Wp = Wn[i] @ R
        assert _expected_complete_ll(Xh[i], Wp, rn[i], den["ES"], den["Ess"])[0] < q0
        Wq = oracle.polar_factor(Wn[i] + 0.01 * rng.standard_normal(Wn[i].shape))
        assert _expected_complete_ll(Xh[i], Wq, rn[i], den["ES"], den["Ess"])[0] < q0
    # Sigma_s update maximises the prior part: -(T/2) ln det S - (1/2) tr(S^-1 sum_t E[ss^T])
    def qs(S):
        return -0.5 * T * np.linalg.slogdet(S)[1] - 0.5 * np.trace(np.linalg.solve(S, den["Ess"].sum(0)))
    base = qs(Sig_new)
    for _ in range(5):
        Dl = rng.standard_normal(Sig_new.shape) * 0.02
        assert qs(Sig_new + Dl @ Dl.T) < base
        assert qs(Sig_new * 1.02) < base


def test_loglik_never_decreases():
    """EM monotonicity, on the raider-like workload and on a random one."""
    d = synth.planted_dataset(synth.config_spec(0))
    r = oracle.fit(d["X"], d["W0"], 10, final_ll=True)
    ll = r["ll"]
    assert np.all(np.diff(ll) >= -1e-12 * np.abs(ll[1:]))
    Xh, W, rho2, Sigma = _rand_problem(11, vs=(20, 35, 27, 41), T=60, k=5)
    r = oracle.fit(Xh, W, 30, centered=True, final_ll=True)
    assert np.all(np.diff(r["ll"]) >= -1e-12 * np.abs(r["ll"][1:]))
    for w in r["W"]:
        np.testing.assert_allclose(w.T @ w, np.eye(w.shape[1]), atol=1e-12)


def test_single_subject_reaches_ppca_fixed_point():
    """N = 1 is PPCA with orthonormal W (Tipping & Bishop 1999): the EM fixed
    point has rho^2 = mean of the v-k smallest covariance eigenvalues,
    span W = leading eigenvectors, eig(Sigma_s) = leading eigenvalues - rho^2."""
    rng = np.random.default_rng(12)
    v, T, k = 30, 400, 3
    Wt = synth.random_orthonormal(rng, v, k)
    S = np.diag([3.0, 2.0, 1.2]) @ rng.standard_normal((k, T))
    X = Wt @ S + 0.3 * rng.standard_normal((v, T)) + rng.standard_normal((v, 1))
    W0 = synth.random_orthonormal(rng, v, k)
    r = oracle.fit([X], [W0], 500)
    Xh = oracle.center(X)[0]
    cf = oracle.ppca_fixed_point(Xh, k)
    assert abs(r["rho2"][0] - cf["rho2"]) <= 1e-6 * cf["rho2"]
    sig_eigs = np.sort(np.linalg.eigvalsh(r["Sigma_s"]))[::-1]
    np.testing.assert_allclose(sig_eigs, cf["sigma_eigs"], rtol=1e-6)
    P1 = r["W"][0] @ r["W"][0].T
    P2 = cf["U"] @ cf["U"].T
    assert np.abs(P1 - P2).max() < 1e-6


def test_invariances():
    """Subject permutation, data scaling (with scaled start values) and a
    rotation of the starting mappings leave the fit unchanged up to the
    model's symmetries (Sec. II-A)."""
    Xh, W, rho2, Sigma = _rand_problem(13, vs=(25, 31, 40), T=50, k=3)
    base = oracle.fit(Xh, W, 6, centered=True)
    perm = [2, 0, 1]
    p = oracle.fit([Xh[i] for i in perm], [W[i] for i in perm], 6, centered=True)
    np.testing.assert_allclose(p["ll"], base["ll"], rtol=1e-12)
    np.testing.assert_allclose(p["rho2"], base["rho2"][perm], rtol=1e-10)
    np.testing.assert_allclose(p["ES"], base["ES"], atol=1e-10)
    c = 3.0
    s = oracle.fit([c * x for x in Xh], W, 6, centered=True,
                   rho2_0=np.full(3, c * c), Sigma_0=c * c * np.eye(3))
    np.testing.assert_allclose(s["rho2"], c * c * base["rho2"], rtol=1e-10)
    np.testing.assert_allclose(s["Sigma_s"], c * c * base["Sigma_s"], rtol=1e-9, atol=1e-12)
    np.testing.assert_allclose(s["ES"], c * base["ES"], rtol=1e-9, atol=1e-10)
    for a, b in zip(s["W"], base["W"]):
        np.testing.assert_allclose(a, b, atol=1e-10)
    R = synth.random_orthonormal(np.random.default_rng(14), 3, 3)
    rr = oracle.fit(Xh, [w @ R for w in W], 6, centered=True)
    np.testing.assert_allclose(rr["ll"], base["ll"], rtol=1e-11)
    np.testing.assert_allclose(rr["ES"], R.T @ base["ES"], atol=1e-9)
    for a, b in zip(rr["W"], base["W"]):
        np.testing.assert_allclose(a, b @ R, atol=1e-9)


def test_planted_recovery_high_snr():
    """High-SNR planted data: each W_i's subspace and S (up to rotation) are
    recovered (max principal-angle sine < 0.1)."""
    from scipy.linalg import orthogonal_procrustes, subspace_angles
    rng = np.random.default_rng(15)
    k, T = 5, 4000
    S = np.diag(np.sqrt(np.linspace(20, 5, k))) @ rng.standard_normal((k, T))
    X, Wt, W0 = [], [], []
    for i in range(3):
        w = synth.random_orthonormal(rng, 200, k)
        X.append(w @ S + rng.standard_normal((200, 1)) + math.sqrt(rng.uniform(0.1, 0.3)) * rng.standard_normal((200, T)))
        Wt.append(w)
        W0.append(synth.random_orthonormal(rng, 200, k))
    r = oracle.fit(X, W0, 40)
    for a, b in zip(r["W"], Wt):
        assert np.sin(subspace_angles(a, b)).max() < 0.1
    Sc = S - S.mean(axis=1, keepdims=True)
    R, _ = orthogonal_procrustes(r["ES"].T, Sc.T)
    err = np.linalg.norm(r["ES"].T @ R - Sc.T) / np.linalg.norm(Sc)
    assert err < 0.1


def test_hand_worked_example():
    """One subject, v = 2, k = 1, T = 2, W = (1, 0)^T, Sigma_s = 1, rho^2 = 1,
    x^ = [[1, -1], [2, -2]] (already demeaned).  By hand:
    rho_0 = 1, Phi = 1/2, y = (1, -1), E[S] = (1/2, -1/2),
    Sigma_s^new = 1/2 + (1/4 + 1/4)/2 = 3/4,
    A = x^ E[S]^T = (1, 2)^T, W^new = (1, 2)/sqrt(5), tr(W^T A) = sqrt(5),
    rho^2 = (10 - 2 sqrt(5) + 2 * 3/4) / 4,
    LL = -1/2 [4 ln 2pi + 0 + 2 ln 2 + 10 - y^T Phi y summed = 1]."""
    Xh = [np.array([[1.0, -1.0], [2.0, -2.0]])]
    W = [np.array([[1.0], [0.0]])]
    est = oracle.estep(Xh, W, np.array([1.0]), np.eye(1))
    assert est["rho0"] == 1.0
    np.testing.assert_allclose(est["Phi"], [[0.5]], atol=1e-15)
    np.testing.assert_allclose(est["ES"], [[0.5, -0.5]], atol=1e-15)
    Sn = oracle.sigma_update(est, 2)
    np.testing.assert_allclose(Sn, [[0.75]], atol=1e-15)
    Wn, rn = oracle.mstep(Xh, [10.0], est["ES"], Sn)
    np.testing.assert_allclose(Wn[0][:, 0], np.array([1.0, 2.0]) / math.sqrt(5), atol=1e-15)
    assert abs(rn[0] - (11.5 - 2 * math.sqrt(5)) / 4) < 1e-14
    ll = oracle.loglik(est, [10.0], [2], np.array([1.0]), np.eye(1), 2)
    assert abs(ll - (-0.5 * (4 * math.log(2 * math.pi) + 2 * math.log(2.0) + 10.0 - 1.0))) < 1e-12


def test_transform_noise_free_closed_form():
    """x_t = W s_t + mu exactly -> W^T (x - mean_t x) = s - mean_t s."""
    rng = np.random.default_rng(16)
    W = synth.random_orthonormal(rng, 50, 4)
    S = rng.standard_normal((4, 33))
    X = W @ S + rng.standard_normal((50, 1))
    np.testing.assert_allclose(oracle.transform(W, X), S - S.mean(axis=1, keepdims=True), atol=1e-12)


def test_map_subjects_closed_form_and_projection():
    """Sec. II-A: x_it = W_i s_t + mu_i exactly -> W_j W_i^T (x - mean_t x) is
    subject j's noise-free data W_j (s - mean_t s); and mapping a subject to
    itself is the orthogonal projection onto span W_i (idempotent, residual
    orthogonal to W_i)."""
    rng = np.random.default_rng(17)
    Wi = synth.random_orthonormal(rng, 60, 5)
    Wj = synth.random_orthonormal(rng, 45, 5)
    S = rng.standard_normal((5, 29))
    X = Wi @ S + rng.standard_normal((60, 1))
    np.testing.assert_allclose(oracle.map_subjects(Wi, Wj, X), Wj @ (S - S.mean(axis=1, keepdims=True)),
                               atol=1e-12)
    Y = rng.standard_normal((60, 29)) + 3.0
    P = oracle.map_subjects(Wi, Wi, Y)
    Yc = Y - Y.mean(axis=1, keepdims=True)
    np.testing.assert_allclose(oracle.map_subjects(Wi, Wi, P), P, atol=1e-12)
    np.testing.assert_allclose(Wi.T @ (Yc - P), np.zeros((5, 29)), atol=1e-12)


def test_oracle_matches_committed_golden():
    """Regression pin: the oracle still reproduces the values its own script
    wrote for the raider-like workload (tests/golden/make_golden.py)."""
    import json
    import os
    with open(os.path.join(os.path.dirname(__file__), "golden", "raider_like_k10.json")) as f:
        g = json.load(f)
    spec = synth.config_spec(0)
    d = synth.planted_dataset(spec, dtype=np.float32)
    np.testing.assert_allclose(d["W0"][0][:4, 0], g["W0_first_col_head"], rtol=1e-12)
    r = oracle.fit([x.astype(np.float64) for x in d["X"]], d["W0"], g["n_iter"], final_ll=True)
    np.testing.assert_allclose(r["ll"], g["ll"], rtol=1e-10)
    np.testing.assert_allclose(r["rho2"], g["rho2"], rtol=1e-9)
    np.testing.assert_allclose(np.trace(r["Sigma_s"]), g["sigma_s_trace"], rtol=1e-9)
