"""The stored GLE fits (gle_params.json, written by the library's fitter fth_fit_gle)
against the oracle: each is a valid GLE (drift with eigenvalues in the right half-plane,
C_p symmetric positive definite, diffusion A_p C_p + C_p A_p^T positive semi-definite,
Eq. 4), the library's per-mode response equals the oracle's exact response of the
integrator, and the reported fit quality and correlation time are what the oracle's
response gives on the fit grid."""
import json

import numpy as np
import pytest

from oracle import gle, matfun
from paper_1402_2095_gb300 import binding as B
from paper_1402_2095_gb300 import fit

with open(fit.PARAMS_FILE) as fh:
    FITS = json.load(fh)


def test_every_table_entry_is_stored():
    assert set(fit.FITS) <= set(FITS)


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
    npts = rep["grid"]
    lams = np.exp(np.linspace(np.log(lo), np.log(hi), npts))
    T, S = gle.propagator(a, c, dt)
    g = gle.mode_response(lams, T, S, dt)
    gl, tau = B.gle_response(a, c, dt, lams, tau=True)
    # the Stein solve loses digits in proportion to the correlation time
    assert np.allclose(gl, g, rtol=1e-12 * max(1.0, float(np.max(tau))), atol=0)
    f = matfun.f_scalar(rep["kind"], lams, rep["params"])
    pts = f >= 1e-3 * np.max(f)
    rel = np.abs(g[pts] / f[pts] - 1.0)
    assert np.max(rel) == pytest.approx(rep["max_rel_err"], rel=1e-7)
    assert np.sqrt(np.mean(rel ** 2)) == pytest.approx(rep["rms_rel_err"], rel=1e-7)
    assert np.max(np.abs(g - f)) / np.max(f) == pytest.approx(rep["max_abs_err"], rel=1e-7)
    k = int(np.argmax(tau))
    assert tau[k] == pytest.approx(rep["tau_max"], rel=1e-9)
    assert gle.x2_correlation_time(lams[k], T, S, dt) == pytest.approx(rep["tau_max"], rel=1e-6)
