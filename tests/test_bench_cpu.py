"""Host-side pieces of bench.py: the roofline arithmetic and the traffic table lookup
(no GPU)."""
import hashlib
import os
import re
import sys

import pytest

ROOT = os.path.abspath(os.path.join(os.path.dirname(__file__), ".."))
sys.path.insert(0, ROOT)
bench = pytest.importorskip("bench")

KNOWN = {"force_tc", "syrk_tc", "gle_dense", "csr_step", "pair_accum", "pool_force", "pool_gle",
         "pool_accum", "fp64_dense"}
WORKLOADS = {"dense4096", "small_fp64", "lattice64", "ragged512", "m1", "m2"}
PRECISIONS = {"fp32", "tf32", "bf16x3", "fp64"}


def test_traffic_table_format():
    lines = open(os.path.join(ROOT, "profiles", "traffic.txt")).read().splitlines()
    rows = [ln.split() for ln in lines if ln.strip() and not ln.startswith("#")]
    assert rows
    for f in rows:
        assert len(f) == 5, f
        kernel, workload, src, digest, nbytes = f
        assert kernel in KNOWN, kernel
        name, precision = workload.split(":")
        assert name in WORKLOADS and precision in PRECISIONS, workload
        assert os.path.exists(os.path.join(ROOT, src)), src
        assert re.fullmatch(r"[0-9a-f]{16}", digest), digest
        assert int(nbytes) > 0


def test_traffic_lookup_follows_the_source_hash(tmp_path, monkeypatch):
    src = tmp_path / "k.cu"
    src.write_text("kernel source v1\n")
    digest = hashlib.sha256(src.read_bytes()).hexdigest()[:16]
    (tmp_path / "profiles").mkdir()
    (tmp_path / "profiles" / "traffic.txt").write_text(
        f"# header\nforce_tc  dense4096:tf32  k.cu  {digest}  12345\n"
        "gle_dense  dense4096:tf32  k.cu  0000000000000000  7\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench._traffic("force_tc", "dense4096:tf32") == 12345
    assert bench._traffic("force_tc", "m2:tf32") is None      # captured on another workload
    assert bench._traffic("force_tc", "dense4096:bf16x3") is None
    assert bench._traffic("gle_dense", "dense4096:tf32") is None   # stale: source changed
    assert bench._traffic("csr_step", "lattice64:fp32") is None    # never captured
    src.write_text("kernel source v2\n")
    assert bench._traffic("force_tc", "dense4096:tf32") is None


class _Wl:
    name = "dense4096"
    precision = "tf32"

    def work(self, cls, info):
        return {"gle_dense": ("hbm", 62.9e6), "force_tc": ("tensor", 8.59e9)}[cls]


def test_roofline_picks_the_dominant_kernel_and_divides_by_its_peak():
    peaks = {"hbm_gbs": 6778.0, "bf16_tflops": 1873.2, "bf16_tflops_sustained": 1678.5}
    # force: 100 launches, 2.5 ms in all (25 us each); GLE: 100 launches, 2.0 ms
    prof = {"force_tc": (2.5, 100), "gle_dense": (2.0, 100)}
    out = bench.roofline(prof, _Wl(), {}, peaks, "measured")
    assert out["kernel"] == "force_tc" and out["bound"] == "tensor"
    achieved = 8.59e9 / 25e-6 / 1e12
    assert out["achieved"] == pytest.approx(achieved)
    assert out["peak"] == pytest.approx(1873.2 * 1.1 / 2.25)
    assert out["frac"] == pytest.approx(achieved / (1873.2 * 1.1 / 2.25))
    assert out["share"] == {"force_tc": pytest.approx(2.5 / 4.5, abs=1e-4),
                            "gle_dense": pytest.approx(2.0 / 4.5, abs=1e-4)}
    prof = {"force_tc": (1.0, 100), "gle_dense": (2.0, 100)}
    out = bench.roofline(prof, _Wl(), {}, peaks, "measured")
    assert out["kernel"] == "gle_dense" and out["bound"] == "hbm"
    assert out["achieved"] == pytest.approx(62.9e6 / 20e-6 / 1e9)
    assert out["frac"] == pytest.approx(out["achieved"] / 6778.0)


def test_sampled_exact_target_agrees_with_the_eigendecomposition():
    """The lattice route (Chebyshev on a sample of elements, taken for orders beyond a
    dense eigendecomposition) against U diag(g) U^T on a lattice small enough for eigh,
    with a burn-in; fed the exact expected values the accuracy report shows zero error."""
    import numpy as np
    import fth_synth as syn
    from oracle import gle

    L = 8
    n = L ** 3
    rowptr, col, val = syn.lattice_csr(L, seed=3)
    val64 = val.astype(np.float32).astype(np.float64)
    a, c = syn.random_gle(4, seed=4, rate=2.0)
    dt = 0.1 / np.sqrt(14.5)

    class _Lattice:
        seed = 5
        n = 10 ** 6                     # takes the sampled route
        csr = (rowptr, col, val.astype(np.float32), 512)
        fit = {"kind": "fermi", "params": [2.0, 7.0]}
        precision = "fp32"
        trace = None

        def __init__(self):
            self.a_p, self.c_p, self.dt = a, c, dt

        def oracle_matrix(self):
            return {"csr": (rowptr, col, val64, n)}

    wl = _Lattice()
    pairs = np.concatenate([syn.diag_pairs(n), syn.lattice_nn_pairs(L)])
    lam, U = np.linalg.eigh(syn.csr_to_dense(rowptr, col, val64, n))
    T, S = gle.propagator(a, c, dt)
    burnin, nacc = 7, 100
    gm = gle.mode_response_mean(lam, T, S, dt, burnin, nacc)
    GMall = np.einsum("kj,kj->k", U[pairs[:, 0]] * gm[None, :], U[pairs[:, 1]])
    pick, G, GM, F, info, modes = bench._exact_values(wl, pairs, burnin, nacc, nsample=8,
                                                      degree=300)
    assert modes is None and len(pick) == 8
    assert info["chebyshev_tail"] < 1e-10
    assert np.allclose(GM, GMall[pick], rtol=1e-9, atol=1e-12)
    acc = {"form": "fp32", "burnin": burnin, "block": 10, "accumulated": nacc, "tau_max": 3.0,
           "snapshot": GMall, "trace": None,
           "runs": {"fp32": {"vals": GMall, "errs": np.full(len(pairs), 1e-3),
                             "ms_per_step": 1.0, "steps": burnin + nacc}}}
    out = bench.exact_target(wl, pairs, acc)
    assert out["fp32"]["rel_err"] < 1e-9
    assert out["fp32"]["sigma_rel"] > 0 and out["fp32"]["steps_to_1e-3"] > burnin


def test_ragged_exact_target_reports_zero_error_for_the_exact_values():
    import numpy as np
    import fth_synth as syn
    from oracle import gle

    a, c = syn.random_gle(4, seed=9, rate=3.0)

    class _Ragged:
        seed, count = 11, 3
        fit = {"kind": "inv_sqrt", "params": []}

        def __init__(self):
            self.a_p, self.c_p, self.dt = a, c, 0.01
            self.mats = [syn.dense_spd(n, 1.0, 100.0, seed=20 + n)[0].astype(np.float32)
                         for n in (40, 64, 100)]
            self.pairs = [np.concatenate([syn.diag_pairs(m.shape[0]), syn.random_pairs(m.shape[0], 8, seed=1)])
                          for m in self.mats]

    wl = _Ragged()
    T, S = gle.propagator(a, c, 0.01)
    read = {}
    for k, m in enumerate(wl.mats):
        lam, U = np.linalg.eigh(m.astype(np.float64))
        gm = gle.mode_response_mean(lam, T, S, 0.01, 0, 300)
        pr = wl.pairs[k]
        v = np.einsum("kj,kj->k", U[pr[:, 0]] * gm[None, :], U[pr[:, 1]])
        read[k] = (v, np.full(len(pr), 1e-3))
    out = bench.exact_target_ragged(wl, read, 0, 300, 0.25, nsample=2)
    assert out["rel_err"] < 1e-12
    assert out["sigma_rel"] > 0 and out["time_to_1e-3_s"] > 0 and out["fit_bias"] > 0


def test_serving_exact_scores_the_exact_values_at_zero():
    import numpy as np
    import fth_synth as syn
    from oracle import gle

    a, c = syn.random_gle(4, seed=12, rate=3.0)

    class _Serving:
        seed = 21

        def __init__(self):
            self.reqs = []
            for n in (50, 80, 120):
                M = syn.dense_spd(n, 1.0, 100.0, seed=n)[0].astype(np.float32)
                pairs = np.concatenate([syn.diag_pairs(n)[:16], syn.random_pairs(n, 16, seed=n)])
                self.reqs.append(dict(M=M, a_p=a, c_p=c, dt=0.01, pairs=pairs))
            rowptr, col, val = syn.lattice_csr(4, seed=1)
            self.reqs.append(dict(csr=(rowptr, col, val, 64), a_p=a, c_p=c, dt=0.01,
                                  pairs=syn.diag_pairs(64)[:4]))

    wl = _Serving()
    T, S = gle.propagator(a, c, 0.01)
    served = {}
    for j, r in enumerate(wl.reqs[:3]):
        lam, U = np.linalg.eigh(r["M"].astype(np.float64))
        gm = gle.mode_response_mean(lam, T, S, 0.01, 0, 400)
        pr = r["pairs"]
        v = np.einsum("kj,kj->k", U[pr[:, 0]] * gm[None, :], U[pr[:, 1]])
        served[j] = (v, np.full(len(pr), 1e-3), 401)   # 401 pool steps: prologue + 400 samples
    served[3] = (np.zeros(4), np.ones(4), 401)          # a lattice request: not sampled
    out = bench.serving_exact(wl, served, nsample=3)
    assert out["requests"] == 3 and out["elements"] == 96
    assert out["rel_err"] < 1e-12 and out["max_abs_z"] < 1e-6 and out["frac_abs_z_below_4"] == 1.0
