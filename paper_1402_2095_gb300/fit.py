"""The GLE fits the workloads use: their definitions, the stored parameters
(gle_params.json) and their regeneration through the library's FP64 host fitter
(fth_fit_gle in libfth.so, see include/fth.h; the fitting method of Sec. "The
f-thermostat" and the requirements of Sec. "Results and benchmarks").  This module only
marshals arguments and keeps the table; the fit itself runs in the library.

    python -m paper_1402_2095_gb300.fit [names...]     # refit and store (all by default)
"""
from __future__ import annotations

import json
import os

import numpy as np

from . import binding

PARAMS_FILE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "gle_params.json")

# Median eigenvalue of the seeded N = 4096 dense workload (lambda log-uniform in [1, 1e3],
# base seed 1402 + 1): its Fermi function is centred there.
MU_DENSE4096 = 32.31759453882913

# name -> (f, f parameters, lam_min, lam_max, fitter options); dt = 0.1 / sqrt(lam_max).
# Fermi fits use the absolute objective (AUTO), the others the relative (log) one.
FITS = {
    "fermi_b5_dense4096": ("fermi", (5.0, MU_DENSE4096), 1.0, 1000.0,
                           dict(starts=8, max_iter=1500)),
    "inv_sqrt_1_100": ("inv_sqrt", (), 1.0, 100.0, dict(starts=8, max_iter=1500)),
    "fermi_b2_lattice": ("fermi", (2.0, 7.0), 0.5, 14.5, dict(starts=8, max_iter=1500)),
    # request mix of the serving loop: the two functions on both spectral ranges
    "fermi_b2_1_100": ("fermi", (2.0, 10.0), 1.0, 100.0, dict(starts=8, max_iter=1500)),
    "inv_sqrt_lattice": ("inv_sqrt", (), 0.5, 14.5, dict(starts=16, max_iter=3000)),
    # the paper's two benchmark functions: ln on [e, 100 e] (M1 scaled into it, then
    # ln M = ln(rM) - I ln r) and exp(-x/100) on [1, 601] (M2 + 301 I, eigenvalues of M2
    # in (-300, 300); exp(-M2/100) = exp(-(M2 + 301 I)/100) e^3.01)
    "log_e_100e": ("log", (), float(np.e), float(100 * np.e), dict(starts=32, max_iter=3000)),
    "exp_001_1_601": ("exp", (0.01,), 1.0, 601.0, dict(starts=8, max_iter=1500)),
}


def load_gle(name: str):
    """(a_p, c_p, dt, report) of a stored fit."""
    with open(PARAMS_FILE) as fh:
        d = json.load(fh)[name]
    return np.array(d["a_p"]), np.array(d["c_p"]), float(d["dt"]), d


def fit_one(name: str):
    """Run the library's fitter for one table entry: (a_p, c_p, report)."""
    kind, params, lo, hi, opts = FITS[name]
    dt = 0.1 / np.sqrt(hi)
    a, c, rep = binding.fit_gle(kind, params, lo, hi, dt, 4, **opts)
    rep.update({"kind": kind, "params": list(params), "lam": [lo, hi], "dt": float(dt), "s": 4,
                "options": opts})
    return a, c, rep


def write_params(names=None):
    out = {}
    if os.path.exists(PARAMS_FILE):
        with open(PARAMS_FILE) as fh:
            out = json.load(fh)
    for name in FITS:
        if names and name not in names:
            continue
        a, c, rep = fit_one(name)
        rep.update({"a_p": a.tolist(), "c_p": c.tolist()})
        out[name] = rep
        print(name, {k: v for k, v in rep.items() if k not in ("a_p", "c_p")}, flush=True)
        with open(PARAMS_FILE, "w") as fh:       # after every fit
            json.dump(out, fh, indent=1)


if __name__ == "__main__":
    import sys
    write_params(sys.argv[1:] or None)
