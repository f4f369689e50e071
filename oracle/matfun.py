"""Reference matrix functions (oracle; test infrastructure only).

f(M) = U diag(f(eps)) U^T from the eigendecomposition (paper, Introduction, Eq. 1),
and the same construction with the per-mode response g of the discretised GLE in
place of f (Eq. 6 with T*(omega) replaced by the exact discrete <p^2>(omega)).
For lattices too large for a dense eigendecomposition, a Chebyshev expansion of g on
an interval containing the spectrum is applied to unit vectors with sparse
matrix-vector products (Chebyshev approximation of matrix functions, e.g. Higham,
"Functions of Matrices", SIAM 2008, Sec. 4.4).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from . import gle


def f_scalar(kind: str, x, params=()):
    x = np.asarray(x, dtype=np.float64)
    if kind == "inv_sqrt":
        return x ** -0.5
    if kind == "fermi":
        beta, mu = params
        return 0.5 * (1.0 - np.tanh(0.5 * beta * (x - mu)))  # 1/(1+exp(beta(x-mu)))
    if kind == "log":
        return np.log(x)
    if kind == "exp":
        (alpha,) = params
        return np.exp(-alpha * x)
    raise ValueError(kind)


def f_of_matrix(M: np.ndarray, fn) -> np.ndarray:
    w, U = np.linalg.eigh(np.asarray(M, dtype=np.float64))
    return (U * fn(w)[None, :]) @ U.T


def g_of_matrix(M: np.ndarray, T, S, dt, observable: int = 0) -> np.ndarray:
    w, U = np.linalg.eigh(np.asarray(M, dtype=np.float64))
    g = gle.mode_response(w, T, S, dt, observable)
    return (U * g[None, :]) @ U.T


def g_mean_of_matrix(M: np.ndarray, T, S, dt, burnin, nsamples, observable: int = 0):
    """Exact expected estimate after `nsamples` accumulated samples (burn-in skipped),
    from the zero initial state."""
    w, U = np.linalg.eigh(np.asarray(M, dtype=np.float64))
    g = gle.mode_response_mean(w, T, S, dt, burnin, nsamples, observable)
    return (U * g[None, :]) @ U.T


# ---------------------------------------------------------------- Chebyshev route
def gershgorin(rowptr, col, val, n):
    a = sp.csr_matrix((np.asarray(val, np.float64), np.asarray(col), np.asarray(rowptr)),
                      shape=(n, n))
    d = a.diagonal()
    rad = np.asarray(abs(a).sum(axis=1)).ravel() - np.abs(d)
    return float(np.min(d - rad)), float(np.max(d + rad))


def cheb_coeffs(fn, a: float, b: float, degree: int) -> np.ndarray:
    """Chebyshev interpolation coefficients of fn on [a, b] at the Chebyshev nodes."""
    m = degree + 1
    k = np.arange(m)
    theta = np.pi * (k + 0.5) / m
    x = np.cos(theta)
    fx = fn(0.5 * (b - a) * x + 0.5 * (b + a))
    c = np.array([2.0 / m * np.sum(fx * np.cos(j * theta)) for j in range(m)])
    c[0] *= 0.5
    return c


def cheb_apply(rowptr, col, val, n, coeffs, a, b, cols) -> np.ndarray:
    """Columns `cols` of p(M), p the Chebyshev series on [a, b]; returns [n, len(cols)]."""
    A = sp.csr_matrix((np.asarray(val, np.float64), np.asarray(col), np.asarray(rowptr)),
                      shape=(n, n))
    alpha = 2.0 / (b - a)
    beta = -(b + a) / (b - a)
    V0 = np.zeros((n, len(cols)))
    V0[np.asarray(cols), np.arange(len(cols))] = 1.0
    V1 = alpha * (A @ V0) + beta * V0
    out = coeffs[0] * V0 + coeffs[1] * V1
    for c in coeffs[2:]:
        V2 = 2.0 * (alpha * (A @ V1) + beta * V1) - V0
        out += c * V2
        V0, V1 = V1, V2
    return out


def fn_elements_sparse(rowptr, col, val, n, fns, pairs, degree=400, interval=None):
    """Elements p_k(M)_ij for several functions at once by the Chebyshev route (one
    three-term recurrence over the unit vectors e_j, shared by all of them).

    fns: callables on arrays of eigenvalues.  Returns (values [len(fns), len(pairs)],
    tails), tails[k] = sum of |c| over the last 10 % of function k's coefficients."""
    if interval is None:
        a, b = gershgorin(rowptr, col, val, n)
        pad = 1e-3 * (b - a)
        a, b = a - pad, b + pad
    else:
        a, b = interval
    coeffs = [cheb_coeffs(fn, a, b, degree) for fn in fns]
    pairs = np.asarray(pairs, dtype=np.int64).reshape(-1, 2)
    js = np.unique(pairs[:, 1])
    A = sp.csr_matrix((np.asarray(val, np.float64), np.asarray(col), np.asarray(rowptr)),
                      shape=(n, n))
    alpha = 2.0 / (b - a)
    beta = -(b + a) / (b - a)
    V0 = np.zeros((n, len(js)))
    V0[js, np.arange(len(js))] = 1.0
    V1 = alpha * (A @ V0) + beta * V0
    outs = [c[0] * V0 + c[1] * V1 for c in coeffs]
    for k in range(2, degree + 1):
        V2 = 2.0 * (alpha * (A @ V1) + beta * V1) - V0
        for o, c in zip(outs, coeffs):
            o += c[k] * V2
        V0, V1 = V1, V2
    where = {int(j): k for k, j in enumerate(js)}
    vals = np.array([[o[int(i), where[int(j)]] for i, j in pairs] for o in outs])
    tails = [float(np.sum(np.abs(c[int(0.9 * len(c)):]))) for c in coeffs]
    return vals, tails


def g_elements_sparse(rowptr, col, val, n, T, S, dt, pairs, degree=256, observable=0,
                      interval=None):
    """Elements g(M)_ij for the given pairs by the Chebyshev route.

    Returns (values, tail) where tail = sum of |c_k| over the last 10% of the
    coefficients, a bound on the truncation error's order of magnitude."""
    if interval is None:
        a, b = gershgorin(rowptr, col, val, n)
        pad = 1e-3 * (b - a)
        a, b = a - pad, b + pad
    else:
        a, b = interval
    fn = lambda x: gle.mode_response(x, T, S, dt, observable)
    c = cheb_coeffs(fn, a, b, degree)
    pairs = np.asarray(pairs, dtype=np.int64).reshape(-1, 2)
    js = np.unique(pairs[:, 1])
    cols = cheb_apply(rowptr, col, val, n, c, a, b, js)
    where = {int(j): k for k, j in enumerate(js)}
    vals = np.array([cols[int(i), where[int(j)]] for i, j in pairs])
    tail = float(np.sum(np.abs(c[int(0.9 * len(c)):])))
    return vals, tail
