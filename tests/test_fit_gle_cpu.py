"""The library's host fitter and per-mode response (fth_fit_gle, fth_gle_response; FP64,
no GPU) against the oracle: the exact discrete response of the integrator (discrete
Lyapunov solve per mode), the correlation time of the sampled p^2 (direct lag sum,
itself pinned against the FP64 integrator in test_oracle_gle.py), and the fit's own
report recomputed from the oracle's response."""
import numpy as np
import pytest

import fth_synth as syn
from oracle import gle, matfun
from paper_1402_2095_gb300 import binding as B


@pytest.mark.parametrize("s,seed,rate,dt,obs", [(4, 1, 2.0, 0.05, "p"), (4, 2, 30.0, 0.01, "p"),
                                                (2, 3, 1.0, 0.1, "q"), (1, 4, 0.5, 0.2, "p"),
                                                (0, 5, 1.0, 0.05, "q")])
def test_response_and_correlation_time_match_oracle(s, seed, rate, dt, obs):
    a, c = syn.random_gle(s, seed=seed, rate=rate)
    lams = np.array([0.3, 1.0, 4.0, 17.0, 80.0, 0.95 * (2.0 / dt) ** 2])   # up to near dt instability
    g, tau = B.gle_response(a, c, dt, lams, observable=obs, tau=True)
    T, S = gle.propagator(a, c, dt)
    ob = 0 if obs == "p" else 1
    go = gle.mode_response(lams, T, S, dt, observable=ob)
    assert np.allclose(g, go, rtol=1e-9, atol=0)
    to = np.array([gle.x2_correlation_time(l, T, S, dt, observable=ob) for l in lams[:4]])
    assert np.allclose(tau[:4], to, rtol=1e-8, atol=0)


def test_response_rejects_bad_arguments():
    a, c = syn.random_gle(4, seed=1, rate=2.0)
    with pytest.raises(B.FthError):
        B.gle_response(a, c, 0.01, [1.0, -2.0])
    with pytest.raises(B.FthError):
        B.gle_response(a, c, -0.01, [1.0])
    # beyond the velocity Verlet stability limit (lam dt^2 > 4) the chain has no
    # stationary state
    with pytest.raises(B.FthError):
        B.gle_response(a, c, 0.1, [500.0])


def _valid_gle(a, c):
    assert np.min(np.linalg.eigvals(a).real) > 0
    assert np.allclose(c, c.T, rtol=0, atol=1e-12 * np.max(np.abs(c)))
    assert np.min(np.linalg.eigvalsh(c)) > 0
    d = a @ c + c @ a.T
    assert np.min(np.linalg.eigvalsh(0.5 * (d + d.T))) >= -1e-10 * np.max(np.abs(d))


def _report_from_oracle(a, c, dt, kind, params, lo, hi, npts, delta):
    lams = np.exp(np.linspace(np.log(lo), np.log(hi), npts))
    T, S = gle.propagator(a, c, dt)
    g = gle.mode_response(lams, T, S, dt)
    f = matfun.f_scalar(kind, lams, params)
    fit = f >= delta * np.max(f)
    rel = np.abs(g[fit] / f[fit] - 1.0)
    return {"max_rel_err": rel.max(), "rms_rel_err": np.sqrt(np.mean(rel ** 2)),
            "max_abs_err": np.max(np.abs(g - f)) / np.max(f),
            "tau_max": max(gle.x2_correlation_time(l, T, S, dt) for l in lams[::10])}


def test_fit_inv_sqrt_quality_report_and_determinism():
    lo, hi, dt = 1.0, 100.0, 0.01
    kw = dict(starts=2, max_iter=200, npts=60, seed=3)
    a, c, rep = B.fit_gle("inv_sqrt", (), lo, hi, dt, 4, **kw)
    _valid_gle(a, c)
    assert rep["objective"] == "log" and rep["grid"] == 60
    assert rep["max_rel_err"] < 5e-3
    ref = _report_from_oracle(a, c, dt, "inv_sqrt", (), lo, hi, 60, 1e-3)
    for k in ("max_rel_err", "rms_rel_err", "max_abs_err"):
        assert rep[k] == pytest.approx(ref[k], rel=1e-7, abs=1e-12), k
    assert rep["tau_max"] >= ref["tau_max"] * (1 - 1e-8)      # the sampled grid is a subset
    a2, c2, rep2 = B.fit_gle("inv_sqrt", (), lo, hi, dt, 4, **kw)
    assert np.array_equal(a, a2) and np.array_equal(c, c2)


def test_fit_fermi_absolute_objective():
    lo, hi = 0.5, 14.5
    dt = 0.1 / np.sqrt(hi)
    a, c, rep = B.fit_gle("fermi", (2.0, 7.0), lo, hi, dt, 4, starts=2, max_iter=150, npts=60)
    _valid_gle(a, c)
    assert rep["objective"] == "abs"
    ref = _report_from_oracle(a, c, dt, "fermi", (2.0, 7.0), lo, hi, 60, 1e-3)
    assert rep["max_abs_err"] == pytest.approx(ref["max_abs_err"], rel=1e-7)
    assert rep["max_abs_err"] < 0.5           # a short fit: 2 starts, 150 iterations


def test_fit_rejects_bad_input():
    for args in [("log", (), 0.5, 10.0, 0.01, 4),        # ln is not positive on the range
                 ("inv_sqrt", (), 1.0, 100.0, 0.01, 0),  # s out of range
                 ("inv_sqrt", (), 1.0, 100.0, 0.01, 5),
                 ("inv_sqrt", (), 10.0, 1.0, 0.01, 4),   # empty range
                 ("inv_sqrt", (), 1.0, 100.0, -0.01, 4)]:
        with pytest.raises(B.FthError) as ex:
            B.fit_gle(*args, starts=1, max_iter=1)
        assert ex.value.status == 1, args
    with pytest.raises(B.FthError):
        B.fit_gle("inv_sqrt", (), 1.0, 100.0, 0.01, 4, w_tau=-1.0, starts=1, max_iter=1)
