"""The stored GLE fits (gle_params.json) against the oracle: each is a valid GLE (drift
with eigenvalues in the right half-plane, C_p symmetric positive definite, diffusion
A_p C_p + C_p A_p^T positive semi-definite, Eq. 4), the fitter's discrete response equals
the oracle's exact per-mode response of the integrator, and the reported fit error is
what that response gives on the fit grid."""
import json

import numpy as np
import pytest

from oracle import gle
from paper_1402_2095_gb300 import fit

with open(fit.PARAMS_FILE) as fh:
    FITS = json.load(fh)


@pytest.mark.parametrize("name", sorted(FITS))
def test_stored_fit_is_valid_and_its_report_is_reproduced(name):
    rep = FITS[name]
    a, c, dt = np.array(rep["a_p"]), np.array(rep["c_p"]), float(rep["dt"])
    lo, hi = rep["lam"]
    ns = rep["s"] + 1
    assert a.shape == c.shape == (ns, ns)
    assert np.min(np.linalg.eigvals(a).real) > 0
    assert np.allclose(c, c.T, rtol=0, atol=1e-12 * np.max(np.abs(c)))
    assert np.min(np.linalg.eigvalsh(c)) > 0
    d = a @ c + c @ a.T
    assert np.min(np.linalg.eigvalsh(0.5 * (d + d.T))) >= -1e-10 * np.max(np.abs(d))
    assert dt == pytest.approx(0.1 / np.sqrt(hi), rel=1e-12)
    lams = np.exp(np.linspace(np.log(lo), np.log(hi), 120))
    T, S = gle.propagator(a, c, dt)
    g = gle.mode_response(lams, T, S, dt)
    assert np.allclose(fit.discrete_response(a, c, dt, lams), g, rtol=1e-9, atol=0)
    f = fit.target(rep["kind"], lams, rep["params"])
    pts = f >= 1e-3 * np.max(f)
    assert np.max(np.abs(g[pts] / f[pts] - 1.0)) == pytest.approx(rep["max_rel_err"], rel=1e-8)
