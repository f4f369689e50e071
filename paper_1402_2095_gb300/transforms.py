"""Reusing one fitted GLE for other spectra and the inverse transforms of Sec. "The
f-thermostat" (scaling, shift, ln and exp relations), as thin wrappers of the library's
C ABI (fth_spectral_map, fth_gle_scale, fth_untransform, fth_untransform_trace): the
arithmetic is in libfth.so; this module only marshals arguments.

With A_p -> alpha A_p, C_p -> gamma C_p and M -> r M + m I, the sampled <p p^T> becomes
gamma f((r M + m I) / alpha^2) for a GLE fitted to f.  ln M = ln(r M) - I ln r,
exp(-a M) = exp(-a (M + m I)) e^{a m}, and for f(x) = x^k, f(M) = f(r M) r^-k.
"""
from __future__ import annotations

import numpy as np

from .binding import gle_scale, spectral_map, untransform, untransform_trace


def affine_map(spec, target):
    """(r, m) such that r x + m maps [spec[0], spec[1]] onto [target[0], target[1]]."""
    return spectral_map(spec, target)


def scale_gle(a_p, c_p, alpha: float = 1.0, gamma: float = 1.0):
    """(alpha A_p, gamma C_p)."""
    return gle_scale(a_p, c_p, alpha, gamma)


def log_from_scaled(values, pairs, r: float):
    """Elements of ln M from elements of ln(r M) at `pairs`."""
    return untransform("log", (r,), pairs, values)[0]


def log_trace_from_scaled(trace_of_log_rM: float, n: int, r: float) -> float:
    """Tr ln M from Tr ln(r M) for an n x n matrix."""
    return untransform_trace("log", (r,), n, trace_of_log_rM)


def _scaled(kind, params, values):
    v = np.asarray(values, dtype=np.float64)
    if v.ndim == 0:
        return untransform_trace(kind, params, 1, float(v))
    flat = v.reshape(-1)
    off = np.zeros((flat.size, 2), dtype=np.int64)
    off[:, 1] = 1                     # element names do not matter for these two kinds
    return untransform(kind, params, off, flat)[0].reshape(v.shape)


def exp_from_shifted(values, a: float, m: float):
    """Elements (or the trace) of exp(-a M) from those of exp(-a (M + m I))."""
    return _scaled("exp", (a, m), values)


def power_from_scaled(values, r: float, k: float):
    """Elements of M^k from those of (r M)^k."""
    return _scaled("power", (r, k), values)
