"""Pins for the oracle's GLE propagator and per-mode covariances (closed forms,
limits, invariances, brute force)."""
import numpy as np
import pytest
import scipy.linalg as sla

import fth_synth as syn
from oracle import gle


def test_chol_psd_matches_lapack_on_pd():
    g = np.random.default_rng(0)
    x = g.standard_normal((5, 5))
    a = x @ x.T + 0.1 * np.eye(5)
    assert np.allclose(gle.chol_psd(a), np.linalg.cholesky(a), atol=1e-13)


def test_chol_psd_semidefinite():
    assert np.all(gle.chol_psd(np.zeros((4, 4))) == 0)
    g = np.random.default_rng(1)
    v = g.standard_normal((5, 2))
    a = v @ v.T  # rank 2
    L = gle.chol_psd(a, rel=1e-12)
    assert np.allclose(L @ L.T, a, atol=1e-10)
    assert np.allclose(L, np.tril(L))


def test_propagator_against_eigen_route():
    a, c = syn.random_gle(4, seed=3, rate=2.0)
    dt = 0.05
    T, S = gle.propagator(a, c, dt)
    w, V = np.linalg.eig(a)
    T2 = (V @ np.diag(np.exp(-0.5 * dt * w)) @ np.linalg.inv(V)).real
    assert np.allclose(T, T2, atol=1e-12)
    assert np.allclose(S @ S.T, c - T @ c @ T.T, atol=1e-13)
    assert np.allclose(S, np.tril(S))


def test_white_noise_langevin_closed_forms():
    # s = 0: O(dt/2) is p <- c p + sqrt(1-c^2) sqrt(kT) xi, c = exp(-gamma dt/2).
    # The velocity Verlet map conserves p^2/2 + (w^2/2)(1 - w^2 dt^2/4) q^2, so at the
    # end of a step <p^2> = kT exactly and w^2 <q^2> = kT / (1 - w^2 dt^2/4).
    gamma, kT, dt = 0.7, 1.3, 0.1
    a, c = syn.white_noise_gle(gamma, kT)
    T, S = gle.propagator(a, c, dt)
    assert np.isclose(T[0, 0], np.exp(-gamma * dt / 2), rtol=1e-15)
    assert np.isclose(S[0, 0], np.sqrt(kT * (1 - np.exp(-gamma * dt)))), S
    for w in (0.3, 1.0, 5.0, 12.0):
        C = gle.discrete_cov(w * w, T, S, dt)
        assert np.isclose(C[1, 1], kT, rtol=1e-12)
        assert np.isclose(w * w * C[0, 0], kT / (1 - w * w * dt * dt / 4), rtol=1e-12)


def test_kron_and_lyapunov_solvers_agree():
    a, c = syn.random_gle(4, seed=5, rate=3.0)
    T, S = gle.propagator(a, c, 0.02)
    for lam in (0.5, 4.0, 60.0):
        assert np.allclose(gle.discrete_cov(lam, T, S, 0.02),
                           gle.discrete_cov_kron(lam, T, S, 0.02), rtol=1e-10, atol=1e-12)


def test_canonical_gle_continuous_limit():
    # C_p = kT I satisfies the fluctuation-dissipation theorem: <p^2> = kT and
    # <q^2> = kT / w^2 for every w, whatever the (stable) drift.
    a, _ = syn.random_gle(4, seed=7, rate=2.0)
    sym = 0.5 * (a + a.T)
    a = a + (max(0.0, -np.min(np.linalg.eigvalsh(sym))) + 0.1) * np.eye(5)
    kT = 0.8
    c = kT * np.eye(5)
    for w in (0.5, 2.0, 9.0):
        C, _ = gle.continuous_cov(w * w, a, c)
        assert np.isclose(C[1, 1], kT, rtol=1e-10)
        assert np.isclose(C[0, 0], kT / (w * w), rtol=1e-10)


def test_discrete_converges_to_continuous_at_second_order():
    a, c = syn.random_gle(4, seed=11, rate=1.5)
    lam = 1.7 ** 2
    Cc, _ = gle.continuous_cov(lam, a, c)
    errs = []
    for dt in (0.04, 0.02, 0.01):
        T, S = gle.propagator(a, c, dt)
        errs.append(abs(gle.discrete_cov(lam, T, S, dt)[1, 1] - Cc[1, 1]))
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 3.5 < r1 < 4.5 and 3.5 < r2 < 4.5, errs


def test_time_rescaling_law():
    # A_p -> alpha A_p, C_p -> gamma C_p, lam -> alpha^2 lam, dt -> dt/alpha is the same
    # chain in rescaled time with amplitudes scaled by gamma: p-moment scales by gamma
    # (the scaling rule of the paper, Sec. "The f-thermostat", exact here because dt is
    # rescaled with A_p).
    a, c = syn.random_gle(4, seed=13, rate=1.0)
    dt, alpha, gam = 0.03, 2.5, 0.7
    T, S = gle.propagator(a, c, dt)
    T2, S2 = gle.propagator(alpha * a, gam * c, dt / alpha)
    for lam in (0.4, 3.0, 20.0):
        g1 = gle.discrete_cov(lam, T, S, dt)[1, 1]
        g2 = gle.discrete_cov(alpha * alpha * lam, T2, S2, dt / alpha)[1, 1]
        assert np.isclose(g2, gam * g1, rtol=1e-9)


def _full_chain(M, T, S, dt):
    """Sample-to-sample map of the whole N-dof system, built from M itself:
    state (q, p, s_1, .., s_n), each block of length N."""
    n = M.shape[0]
    ns = T.shape[0]
    d = (ns + 1) * n
    I = np.eye(n)
    O = np.zeros((d, d))
    O[:n, :n] = I
    O[n:, n:] = np.kron(T, I)
    sig = np.zeros((d, ns * n))
    sig[n:, :] = np.kron(S, I)
    B = np.eye(d)
    B[n:2 * n, :n] = -0.5 * dt * M
    A = np.eye(d)
    A[:n, n:2 * n] = dt * I
    V = B @ A @ B
    G = O @ V @ O
    ov = O @ V @ sig
    return G, ov @ ov.T + sig @ sig.T


@pytest.mark.parametrize("n", [3, 4])
def test_brute_force_full_system_equals_mode_composition(n):
    # Eq. 6: the isotropic GLE acts on each normal mode independently, so the
    # stationary <p p^T> of the coupled system is U diag(g(eps)) U^T.
    M, _, _ = syn.dense_spd(n, 1.0, 30.0, seed=17 + n)
    a, c = syn.random_gle(4, seed=19, rate=2.0)
    dt = 0.05
    T, S = gle.propagator(a, c, dt)
    G, Qn = _full_chain(M, T, S, dt)
    d = G.shape[0]
    x = np.linalg.solve(np.eye(d * d) - np.kron(G, G), Qn.reshape(-1)).reshape(d, d)
    pp = x[n:2 * n, n:2 * n]
    qq = x[:n, :n]
    w, U = np.linalg.eigh(M)
    gp = np.array([gle.discrete_cov(l, T, S, dt)[1, 1] for l in w])
    gq = np.array([gle.discrete_cov(l, T, S, dt)[0, 0] for l in w])
    assert np.allclose(pp, (U * gp) @ U.T, atol=1e-12)
    assert np.allclose(qq, (U * gq) @ U.T, atol=1e-12)


def test_transient_recursion_reaches_stationary():
    a, c = syn.random_gle(4, seed=23, rate=3.0)
    T, S = gle.propagator(a, c, 0.05)
    covs = gle.transient_covs(2.0, T, S, 0.05, 4000)
    G, Qn = gle.mode_chain(2.0, T, S, 0.05)
    assert np.allclose(covs[0], Qn)
    assert np.allclose(covs[-1], gle.discrete_cov(2.0, T, S, 0.05), rtol=1e-8, atol=1e-12)


def test_tau_p2_white_noise():
    # s = 0, free particle limit w -> 0 is an OU process in p with rate gamma:
    # c(t) = kT exp(-gamma t), so tau = int c^2 / c(0)^2 = 1/(2 gamma).  For w > 0 the
    # same formula is checked against direct quadrature of c(t)^2.
    gamma = 0.9
    a, c = syn.white_noise_gle(gamma, 1.0)
    assert np.isclose(gle.tau_p2(1e-8, a, c), 1 / (2 * gamma), rtol=1e-6)
    lam = 2.0
    C, A = gle.continuous_cov(lam, a, c)
    w, V = np.linalg.eig(A)
    Vi = np.linalg.inv(V)
    tt = np.linspace(0, 60, 120001)
    ct = np.einsum("j,tj,j->t", V[1, :], np.exp(-np.outer(tt, w)), (Vi @ C)[:, 1]).real
    integral = np.trapezoid(ct ** 2, tt)
    assert np.isclose(gle.tau_p2(lam, a, c), integral / C[1, 1] ** 2, rtol=1e-6)


@pytest.mark.parametrize("burnin,n", [(0, 1), (0, 300), (25, 700), (400, 50)])
def test_transient_mean_closed_form_equals_recursion(burnin, n):
    a, c = syn.random_gle(4, seed=29, rate=2.0)
    T, S = gle.propagator(a, c, 0.05)
    lams = [0.3, 2.0, 35.0]
    for obs in (0, 1):
        fast = gle.mode_response_mean(lams, T, S, 0.05, burnin, n, obs)
        slow = gle.mode_response_mean_recursive(lams, T, S, 0.05, burnin, n, obs)
        assert np.allclose(fast, slow, rtol=1e-9, atol=1e-12)


def test_x2_correlation_time_predicts_the_variance_of_the_mean():
    """The oracle's correlation time of p^2 against the FP64 integrator: for one mode
    (N = 1, M = [lam]) and many independent replicas, the variance over replicas of the
    time average of p^2 (after a burn-in) tends to 2 <p^2>^2 tau / n."""
    from oracle.fth import OracleFTH
    a, c = syn.random_gle(4, seed=21, rate=3.0)
    dt, lam, R = 0.05, 2.0, 2000
    T, S = gle.propagator(a, c, dt)
    tau = gle.x2_correlation_time(lam, T, S, dt)
    g = gle.discrete_cov(lam, T, S, dt)[1, 1]
    assert 1.0 < tau < 500.0
    nburn, n, chunk = int(20 * tau), int(400 * tau), 2000
    o = OracleFTH(M=np.array([[lam]]), a_p=a, c_p=c, dt=dt, replicas=R, seed=5)
    o.run(nburn)
    acc = np.zeros(R)
    done = 0
    while done < n:
        k = min(chunk, n - done)
        x = o.run(k, keep_samples=True)[:, :, 0]
        acc += np.sum(x * x, axis=0)
        done += k
    var = np.var(acc / n, ddof=1)
    want = 2.0 * g * g * tau / n
    # R = 2000 replicas: the sample variance is within ~3 % (1 sigma) of its mean; the
    # finite length adds a relative O(tau / n) = 0.25 % bias
    assert abs(var / want - 1.0) < 0.12, (var, want)


def test_x2_correlation_time_white_noise_limit():
    """s = 0 with a large friction: the O half-steps redraw p almost completely, so
    successive end-of-step samples of p are nearly independent and tau -> 1."""
    a, c = syn.white_noise_gle(2000.0, 1.0)
    T, S = gle.propagator(a, c, 0.01)
    tau = gle.x2_correlation_time(0.5, T, S, 0.01)
    assert 1.0 <= tau < 1.01
