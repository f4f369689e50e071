"""Host-side bookkeeping around a fitted GLE: reusing one fit for other spectra and the
inverse transforms of Sec. "The f-thermostat" (paper's scaling and shift relations).

Scaling and shift: with A_p -> alpha A_p, C_p -> gamma C_p and M -> r M + m I, the
sampled <p p^T> becomes gamma f((r M + m I) / alpha^2) for a GLE fitted to f.  The paper
prints the shift with its sign flipped; affine_map() uses the form derived from
r lo + m = lo' and r hi + m = hi'.

Inverse transforms: ln M = ln(r M) - I ln r (a fit of ln on a range where it is
positive serves any M whose scaled spectrum falls inside it),
exp(-a M) = exp(-a (M + m I)) e^{a m} (a shift makes an indefinite M positive definite),
and for a power law f(x) = x^k, f(M) = f(r M) r^-k (one fit serves every spectrum that a
scaling r moves into its range).
"""
from __future__ import annotations

import numpy as np


def affine_map(spec, target):
    """(r, m) such that r x + m maps [spec[0], spec[1]] onto [target[0], target[1]]."""
    lo, hi = float(spec[0]), float(spec[1])
    tlo, thi = float(target[0]), float(target[1])
    if not hi > lo:
        raise ValueError("empty spectral interval")
    r = (thi - tlo) / (hi - lo)
    m = (tlo * hi - thi * lo) / (hi - lo)
    return r, m


def scale_gle(a_p, c_p, alpha: float = 1.0, gamma: float = 1.0):
    """(alpha A_p, gamma C_p): the same GLE on a frequency axis scaled by alpha, with its
    fluctuations scaled by gamma."""
    return alpha * np.asarray(a_p, dtype=np.float64), gamma * np.asarray(c_p, dtype=np.float64)


def log_from_scaled(values, pairs, r: float):
    """Elements of ln M from elements of ln(r M): the diagonal ones lose ln r."""
    v = np.array(values, dtype=np.float64, copy=True)
    p = np.asarray(pairs).reshape(-1, 2)
    v[p[:, 0] == p[:, 1]] -= np.log(r)
    return v


def log_trace_from_scaled(trace_of_log_rM: float, n: int, r: float) -> float:
    """Tr ln M from Tr ln(r M) for an n x n matrix."""
    return float(trace_of_log_rM) - n * np.log(r)


def exp_from_shifted(values, a: float, m: float):
    """Elements (or the trace) of exp(-a M) from those of exp(-a (M + m I))."""
    return np.asarray(values, dtype=np.float64) * np.exp(a * m)


def power_from_scaled(values, r: float, k: float):
    """Elements of M^k from those of (r M)^k."""
    return np.asarray(values, dtype=np.float64) * float(r) ** (-k)
