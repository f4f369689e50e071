"""GLE propagator and exact per-mode covariances (oracle; test infrastructure only).

Paper references (Nava, Ceriotti, Dryzun, Parrinello):
  Eq. 2   Markovian GLE in the extended momentum space (p, s_1..s_n), drift A_p and
          diffusion B_p;
  Eq. 4   A_p C_p + C_p A_p^T = B_p B_p^T links the free-particle covariance C_p to B_p;
  Eq. 5   V(q) = q^T M q / 2, so every normal mode is a harmonic oscillator with
          omega^2 = eigenvalue;
  Eq. 6   <p_i p_j> = sum_k U_ik T*(omega_k) U_jk: the isotropic GLE acts on each normal
          mode independently (linearity and Gaussian noise).
The integrator is the modified velocity Verlet scheme the paper cites: per step
O(dt/2) B(dt/2) A(dt) [force] B(dt/2) O(dt/2), where the O half-step is the exact
Ornstein-Uhlenbeck update  p~ <- T p~ + S xi,  T = exp(-A_p dt/2),
S S^T = C_p - T C_p T^T, and samples are taken at the end of each step.

For one normal mode of eigenvalue lam the step is linear in x = (q, p, s_1..s_n):
from one sample point to the next, x' = G x + O V Sig xi_a + Sig xi_b with
O = diag(1, T), Sig = [0; S], V = B A B, B = I - (lam dt/2) e_p e_q^T,
A = I + dt e_q e_p^T and G = O V O.  Its stationary covariance solves the discrete
Lyapunov equation C = G C G^T + Qn with Qn = (O V Sig)(O V Sig)^T + Sig Sig^T; that
C[p,p] (or C[q,q]) is what the simulation converges to, exactly, for the fitted GLE
at this time step.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla

IQ, IP = 0, 1  # positions of q and p in the per-mode state x = (q, p, s...)


def chol_psd(sig: np.ndarray, rel: float = 1e-14) -> np.ndarray:
    """Lower-triangular L with L L^T = sig for symmetric PSD sig.

    Plain Cholesky-Banachiewicz; a pivot at or below rel * max(diag) is taken as an
    exact zero (its column of L is zero), which is the reading used when
    C_p - T C_p T^T is only positive semi-definite (e.g. noise-free directions)."""
    sig = 0.5 * (np.asarray(sig, dtype=np.float64) + np.asarray(sig, dtype=np.float64).T)
    n = sig.shape[0]
    L = np.zeros_like(sig)
    tol = rel * max(float(np.max(np.diag(sig))), 0.0)
    for j in range(n):
        d = sig[j, j] - float(np.dot(L[j, :j], L[j, :j]))
        if d <= tol:
            continue
        L[j, j] = np.sqrt(d)
        for i in range(j + 1, n):
            L[i, j] = (sig[i, j] - float(np.dot(L[i, :j], L[j, :j]))) / L[j, j]
    return L


def joint_noise(T: np.ndarray, S: np.ndarray) -> np.ndarray:
    """Factor L ((ns+1) x (ns+1), lower) of the joint law of the two O half-steps
    around the end-of-step sample (Eq. 2's exact Ornstein-Uhlenbeck half-step, applied
    twice with the sample of p in between).  From a state v the sample is
    (T v)_0 + x and the next state T T v + y with x = e_0^T S xi1, y = T S xi1 + S xi2;
    (x, y) is Gaussian with covariance
        [[C1_00,      (T C1 e_0)^T     ],
         [T C1 e_0,   T C1 T^T + C1    ]],  C1 = S S^T,
    factored by chol_psd (same zero-pivot rule as S)."""
    T = np.asarray(T, dtype=np.float64)
    S = np.asarray(S, dtype=np.float64)
    ns = T.shape[0]
    C1 = S @ S.T
    sig = np.zeros((ns + 1, ns + 1))
    sig[0, 0] = C1[0, 0]
    sig[1:, 0] = sig[0, 1:] = T @ C1[:, 0]
    sig[1:, 1:] = T @ C1 @ T.T + C1
    return chol_psd(sig)


def propagator(a_p: np.ndarray, c_p: np.ndarray, dt: float):
    """(T, S) of the O half-step: T = exp(-A_p dt/2), S = chol(C_p - T C_p T^T)."""
    a_p = np.asarray(a_p, dtype=np.float64)
    c_p = np.asarray(c_p, dtype=np.float64)
    T = sla.expm(-a_p * (0.5 * dt))
    sig = c_p - T @ c_p @ T.T
    return T, chol_psd(sig)


def mode_chain(lam: float, T: np.ndarray, S: np.ndarray, dt: float):
    """(G, Qn) of the sample-to-sample map of one normal mode (see module doc)."""
    ns = T.shape[0]
    d = ns + 1
    O = np.eye(d)
    O[1:, 1:] = T
    sig = np.zeros((d, ns))
    sig[1:, :] = S
    B = np.eye(d)
    B[IP, IQ] = -0.5 * dt * lam
    A = np.eye(d)
    A[IQ, IP] = dt
    V = B @ A @ B
    G = O @ V @ O
    ov = O @ V @ sig
    Qn = ov @ ov.T + sig @ sig.T
    return G, Qn


def discrete_cov(lam: float, T, S, dt) -> np.ndarray:
    """Stationary covariance at the sample point: C = G C G^T + Qn."""
    G, Qn = mode_chain(lam, T, S, dt)
    C = sla.solve_discrete_lyapunov(G, Qn)
    return 0.5 * (C + C.T)


def discrete_cov_kron(lam: float, T, S, dt) -> np.ndarray:
    """Same fixed point by a dense Kronecker solve, (I - G (x) G) vec C = vec Qn."""
    G, Qn = mode_chain(lam, T, S, dt)
    d = G.shape[0]
    c = np.linalg.solve(np.eye(d * d) - np.kron(G, G), Qn.reshape(-1))
    C = c.reshape(d, d)
    return 0.5 * (C + C.T)


def transient_covs(lam: float, T, S, dt, nsamples: int) -> np.ndarray:
    """Covariances of samples 0..nsamples-1 when the run starts from x = 0.

    The first sample follows one full sample-to-sample map from x = 0 (prologue
    O B A, then force, B, O), so C_0 = Qn and C_k = G C_{k-1} G^T + Qn."""
    G, Qn = mode_chain(lam, T, S, dt)
    out = np.empty((nsamples,) + G.shape)
    C = np.zeros_like(G)
    for k in range(nsamples):
        C = G @ C @ G.T + Qn
        out[k] = C
    return out


def mode_response(lams, T, S, dt, observable: int = 0) -> np.ndarray:
    """g(lam): stationary <p^2> (observable 0) or <q^2> (1) of each mode."""
    idx = IP if observable == 0 else IQ
    return np.array([discrete_cov(float(l), T, S, dt)[idx, idx] for l in np.ravel(lams)])


def mode_response_mean(lams, T, S, dt, burnin: int, nsamples: int, observable: int = 0):
    """Exact expected running mean of x^2 over samples burnin..burnin+nsamples-1 from
    the zero initial state, per mode.

    From C_k - C = G (C_{k-1} - C) G^T and C_{-1} = 0: C_k = C - G^{k+1} C G^{k+1 T}, so
    the mean over k = b..b+n-1 is C - (1/n) [G^{b+1} X G^{b+1 T} - G^{b+n+1} X G^{b+n+1 T}]
    with X = sum_j G^j C G^{j T}, the solution of X = G X G^T + C."""
    idx = IP if observable == 0 else IQ
    out = []
    for l in np.ravel(lams):
        G, Qn = mode_chain(float(l), T, S, dt)
        C = sla.solve_discrete_lyapunov(G, Qn)
        X = sla.solve_discrete_lyapunov(G, C)
        Ga = np.linalg.matrix_power(G, burnin + 1)
        Gb = np.linalg.matrix_power(G, burnin + nsamples + 1)
        tail = (Ga @ X @ Ga.T - Gb @ X @ Gb.T) / nsamples
        out.append(float(C[idx, idx] - tail[idx, idx]))
    return np.asarray(out)


def mode_response_mean_recursive(lams, T, S, dt, burnin: int, nsamples: int, observable=0):
    """Same quantity by running the covariance recursion sample by sample."""
    idx = IP if observable == 0 else IQ
    out = []
    for l in np.ravel(lams):
        covs = transient_covs(float(l), T, S, dt, burnin + nsamples)
        out.append(float(np.mean(covs[burnin:, idx, idx])))
    return np.asarray(out)


def x2_correlation_time(lam: float, T, S, dt, observable: int = 0, rel: float = 1e-17,
                        max_lags: int = 10_000_000) -> float:
    """Integrated correlation time, in samples, of x^2 for the sampled observable x of
    one mode (x = p or q): tau = 1 + 2 sum_{l >= 1} corr(x^2(0), x^2(l)).  For the
    Gaussian stationary chain the autocovariance of x^2 at lag l is 2 c(l)^2 with
    c(l) = e_x^T G^l C e_x, so corr = (c(l) / c(0))^2; the lags are summed one by one
    (w_{l+1} = G w_l from w_0 = C e_x) until a term falls below rel.  The variance of the
    mean of x^2 over n samples tends to 2 c(0)^2 tau / n."""
    idx = IP if observable == 0 else IQ
    G, _ = mode_chain(lam, T, S, dt)
    C = discrete_cov(lam, T, S, dt)
    w = C[:, idx].copy()
    c0 = w[idx]
    total = 1.0
    for _ in range(max_lags):
        w = G @ w
        term = (w[idx] / c0) ** 2
        total += 2.0 * term
        if term < rel:
            return float(total)
    raise RuntimeError("correlation sum did not converge")


# ---------------------------------------------------------------- continuous limit
def continuous_cov(lam: float, a_p, c_p) -> np.ndarray:
    """dt -> 0 stationary covariance of (q, p, s): A X + X A^T = D with
    A = [[0, -1, 0], [lam, A_p]] and D = diag(0, A_p C_p + C_p A_p^T) (Eq. 2, Eq. 4)."""
    a_p = np.asarray(a_p, dtype=np.float64)
    c_p = np.asarray(c_p, dtype=np.float64)
    ns = a_p.shape[0]
    d = ns + 1
    A = np.zeros((d, d))
    A[IQ, IP] = -1.0
    A[IP, IQ] = lam
    A[1:, 1:] = a_p
    D = np.zeros((d, d))
    D[1:, 1:] = a_p @ c_p + c_p @ a_p.T
    X = sla.solve_continuous_lyapunov(A, D)
    return 0.5 * (X + X.T), A


def tau_p2(lam: float, a_p, c_p) -> float:
    """Correlation time of p^2 for one mode in the dt -> 0 limit:
    tau = int_0^inf c(t)^2 dt / c(0)^2 with c(t) = [exp(-A t) C]_pp, evaluated as
    X_pp / C_pp^2 where A X + X A^T = C e_p e_p^T C."""
    C, A = continuous_cov(lam, a_p, c_p)
    v = C[:, IP:IP + 1]
    X = sla.solve_continuous_lyapunov(A, v @ v.T)
    return float(X[IP, IP] / C[IP, IP] ** 2)
