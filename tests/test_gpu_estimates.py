"""Estimate-level parity of the force precision forms, full-size checks at the benchmark's
launch configuration, and the device error paths -- all through the C ABI.

Precision forms (FP32 FFMA, TF32 and split BF16 on tcgen05) change the force
contraction (Eq. 5) and, with every element tracked, the tensor-core forms stage the
samples in BF16 for the accumulation (each product off by at most 2^-7, averaging out
to ~1e-5 over a run); the estimator is Eq. 6 either way.  Run on the same seed, the
three forms and the FP64 oracle draw the same Philox normals, so the difference of two
estimates is (almost) free of statistical error: it isolates what each form's rounding
does to the estimate of <p_i p_j>.  The bounds are the measured errors with headroom
(normwise over the tracked set, relative to the FP64 same-noise estimate):
  FP32    1e-4   (trajectories agree to ~1e-6 of their scale)
  BF16X3  1e-3   (force error ~2^-16 of sum_k |M_ik q_k|)
  TF32    3e-2   (force error ~2^-11; its trajectories drift apart by ~1e-2 of their
                  scale over thousands of steps, and that drift does not average out)
"""
import numpy as np
import pytest

import fth_synth as syn
from oracle import gle, matfun
from oracle.fth import OracleFTH, fused_step_elements

from gpu_util import bf16_rn, gpu_ready

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not gpu_ready(), reason="needs a CUDA GPU and libfth.so")]

FORM_BOUND = {"fp32": 1e-4, "bf16x3": 1e-3, "tf32": 3e-2}


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


# ------------------------------------------------------------------ same-noise estimates
def test_precision_forms_same_noise_estimates():
    """FP32, TF32 and BF16x3 estimates against the FP64 oracle's estimate on the same
    noise (precision error of each form's estimate), and each against the exact
    expected running mean U g_mean U^T (statistical consistency: z-scores)."""
    from paper_1402_2095_gb300 import FTH
    n, R, steps, block, seed = 256, 64, 4000, 200, 1501
    M, _, _ = syn.dense_spd(n, 1.0, 100.0, seed=1502)
    M32 = M.astype(np.float32)
    Mo = M32.astype(np.float64)
    a, c = syn.random_gle(4, seed=1503, rate=3.0)
    dt = 0.1 / np.sqrt(100.0)
    pairs = np.concatenate([syn.diag_pairs(n), syn.random_pairs(n, 256, seed=1504)])
    o = OracleFTH(M=Mo, a_p=a, c_p=c, dt=dt, replicas=R, seed=seed, block=block, pairs=pairs)
    o.run(steps)
    vo, eo = o.elements()
    T, S = gle.propagator(a, c, dt)
    ref = matfun.g_mean_of_matrix(Mo, T, S, dt, 0, steps)[pairs[:, 0], pairs[:, 1]]
    z_o = (vo - ref) / eo
    assert 0.3 < np.mean(z_o ** 2) < 3.0
    report = {}
    for prec in ("fp32", "bf16x3", "tf32"):
        f = FTH(M=M32, a_p=a, c_p=c, dt=dt, replicas=R, seed=seed, precision=prec,
                track="all", block=block)
        f.run(steps)
        v, e = f.elements(pairs)
        d = _rel(v, vo)
        z = (v - ref) / e
        report[prec] = (d, float(np.mean(z ** 2)))
        assert d <= FORM_BOUND[prec], (prec, d)
        assert 0.3 < np.mean(z ** 2) < 3.0, (prec, np.mean(z ** 2))
        assert np.all(np.abs(z) < 6.0), prec
        # the block error bars follow the oracle's (same noise, same blocks)
        # (block means differ from their average by a few % of their value, so the
        # error bars move by tens of times the estimate's relative error)
        assert _rel(e, eo) <= max(50 * d, 2e-3), (prec, _rel(e, eo))
    print("same-noise estimate error vs FP64 oracle (normwise) and <z^2> vs exact:", report)


def test_stationary_tf32_dense():
    """TF32, the form of the dense benchmark: every sampled element within 4 block
    error bars of the exact expected running mean, <z^2> near 1."""
    from paper_1402_2095_gb300 import FTH
    n, R, steps, block = 64, 64, 20000, 500
    M, _, _ = syn.dense_spd(n, 1.0, 50.0, seed=41)
    a, c = syn.random_gle(4, seed=42, rate=3.0)
    dt = 0.1 / np.sqrt(50.0)
    f = FTH(M=M.astype(np.float32), a_p=a, c_p=c, dt=dt, replicas=R, seed=44, precision="tf32",
            track="all", block=block)
    f.run(steps)
    pairs = syn.upper_pairs(n)
    vals, errs = f.elements(pairs)
    T, S = gle.propagator(a, c, dt)
    ref = matfun.g_mean_of_matrix(M.astype(np.float32).astype(np.float64), T, S, dt, 0,
                                  steps)[pairs[:, 0], pairs[:, 1]]
    z = (vals - ref) / errs
    sample = np.random.default_rng(10).choice(len(pairs), 32, replace=False)
    assert np.all(np.abs(z[sample]) < 4.0), z[sample]
    assert 0.5 < np.mean(z ** 2) < 2.0


# ------------------------------------------------------------------ calibrated error bars
def _calibrated(a_p, c_p, dt, lo, hi):
    """Burn-in 10 tau_max and blocks of max(1000, 10 tau_max) samples, tau_max the
    library's correlation time of p^2 over [lo, hi] (fth_gle_response)."""
    from paper_1402_2095_gb300 import binding
    _, tau = binding.gle_response(a_p, c_p, dt, np.exp(np.linspace(np.log(lo), np.log(hi), 240)),
                                  tau=True)
    t = float(tau.max())
    return int(np.ceil(10 * t)), max(1000, int(np.ceil(10 * t)))


@pytest.mark.parametrize("kind", ["dense_tf32", "lattice_csr"])
def test_calibrated_error_bars_at_a_fitted_gle(kind):
    """With the stored Fermi fits (the benchmark's GLEs) and the calibrated burn-in and
    block length, the block error bars describe the actual error against the exact
    expected running mean: <z^2> within (0.5, 2) over every tracked element."""
    from paper_1402_2095_gb300 import FTH, fit
    nblocks = 20
    if kind == "dense_tf32":
        a, c, dt, rep = fit.load_gle("fermi_b5_dense4096")
        M, _, _ = syn.dense_spd(384, 1.0, 1000.0, seed=1601)
        Mo = M.astype(np.float32).astype(np.float64)
        burnin, block = _calibrated(a, c, dt, 1.0, 1000.0)
        pairs = syn.upper_pairs(384)
        f = FTH(M=M.astype(np.float32), a_p=a, c_p=c, dt=dt, replicas=64, seed=1602,
                precision="tf32", track="all", burnin=burnin, block=block)
    else:
        a, c, dt, rep = fit.load_gle("fermi_b2_lattice")
        L = 7
        rowptr, col, val = syn.lattice_csr(L, seed=1603)
        v32 = val.astype(np.float32)
        Mo = syn.csr_to_dense(rowptr, col, v32.astype(np.float64), L ** 3)
        burnin, block = _calibrated(a, c, dt, 0.5, 14.5)
        pairs = np.concatenate([syn.diag_pairs(L ** 3), syn.lattice_nn_pairs(L)])
        f = FTH(csr=(rowptr, col, v32, L ** 3), a_p=a, c_p=c, dt=dt, replicas=64, seed=1604,
                pairs=pairs, burnin=burnin, block=block)
    f.run(burnin + nblocks * block)
    assert f.info()["blocks"] == nblocks
    vals, errs = f.elements(pairs)
    T, S = gle.propagator(a, c, dt)
    ref = matfun.g_mean_of_matrix(Mo, T, S, dt, burnin, nblocks * block)[pairs[:, 0], pairs[:, 1]]
    z = (vals - ref) / errs
    print(kind, "burnin", burnin, "block", block, "<z^2>", float(np.mean(z ** 2)))
    assert 0.5 < np.mean(z ** 2) < 2.0
    sample = np.random.default_rng(11).choice(len(pairs), 32, replace=False)
    assert np.all(np.abs(z[sample]) < 5.0), z[sample]


# ------------------------------------------------------------------ full size
def test_full_size_dense_fp32_sampled():
    """N = 4096, R = 256 with the plain FP32 (FFMA) force: one fused step from a random
    primed state, sampled (i, r) against the oracle one by one.  Bound: 1e-6 of the
    value plus 2^-16 of the force's own error scale (FP32 sums of 4096 products)."""
    import torch
    from paper_1402_2095_gb300 import FTH
    n, R, dt = 4096, 256, 0.1 / np.sqrt(1000.0)
    M, _, _ = syn.dense_spd(n, 1.0, 1000.0, seed=1402 + 2)
    M32 = M.astype(np.float32)
    a, c = syn.random_gle(4, seed=74, rate=5.0)
    f = FTH(M=torch.from_numpy(M32).cuda(), a_p=a, c_p=c, dt=dt, replicas=R, seed=75,
            precision="fp32", track="diag", block=4)
    g = np.random.default_rng(76)
    q0 = g.standard_normal((R, n)).astype(np.float32).astype(np.float64)
    p0 = g.standard_normal((R, n)).astype(np.float32).astype(np.float64)
    s0 = g.standard_normal((R, 4, n)).astype(np.float32).astype(np.float64)
    f.run(0)
    f.set_state("q", q0)
    f.set_state("p", p0)
    f.set_state("s", s0)
    kappa = f.info()["steps"] + 1
    f.run(1)
    elems = [(int(i), int(r)) for i, r in zip(g.integers(0, n, 48), g.integers(0, R, 48))]
    T, S = gle.propagator(a, c, dt)
    M64 = M32.astype(np.float64)
    qn, pn, sn, _ = fused_step_elements(M64, q0, p0, s0, T, S, dt, 75, kappa, elems)
    q1, p1, s1 = f.get_state("q"), f.get_state("p"), f.get_state("s")
    for k, (i, r) in enumerate(elems):
        sc = dt * float(np.abs(M64[i]) @ np.abs(q0[r]))   # two half-kicks' error scale
        tol = 2.0 ** -16 * sc
        assert abs(p1[r, i] - pn[k]) <= 1e-6 * (1 + abs(pn[k])) + tol
        assert abs(q1[r, i] - qn[k]) <= 1e-6 * (1 + abs(qn[k])) + dt * tol
        assert np.all(np.abs(s1[r, :, i] - sn[k]) <= 1e-6 * (1 + np.abs(sn[k])) + tol)


def test_full_size_dense_tf32_accumulators_sampled():
    """N = 4096, R = 256, TF32 force and every element accumulated (tcgen05 SYRK over the
    staged samples, one pass per block of 8 here): three passes and three blocks, read back on a sample
    of 4096 elements.  With A_p = C_p = 0 the dynamics is noise-free velocity Verlet and
    the samples of q follow in FP64 from the same start, staged in BF16 (round to nearest)
    as the accumulation pass reads them; bound 2^-9 of the products' scale (TF32 force,
    FP32 sums), on values and block error bars."""
    import torch
    from paper_1402_2095_gb300 import FTH
    n, R, K, block = 4096, 256, 24, 8
    dt = 0.1 / np.sqrt(1000.0)
    M, _, _ = syn.dense_spd(n, 1.0, 1000.0, seed=1402 + 2)
    M64 = M.astype(np.float32).astype(np.float64)
    z = np.zeros((5, 5))
    f = FTH(M=torch.from_numpy(M64.astype(np.float32)).cuda(), a_p=z, c_p=z, dt=dt, replicas=R,
            seed=0, precision="tf32", track="all", block=block, observable="q")
    q0 = syn.gaussian_state((R, n), seed=77).astype(np.float32).astype(np.float64)
    f.set_state("q", q0)
    f.run(K)
    info = f.info()
    assert info["blocks"] == K // block and info["accumulated"] == K
    g = np.random.default_rng(78)
    pairs = np.concatenate([syn.diag_pairs(n)[g.choice(n, 512, replace=False)],
                            syn.random_pairs(n, 3584, seed=79)])
    vals, errs = f.elements(pairs)
    # reference: prologue kick and drift, then per step force, kick, sample q, kick, drift
    q, p = q0.copy(), np.zeros_like(q0)
    p -= 0.5 * dt * q @ M64.T
    q += dt * p
    ii, jj = pairs[:, 0], pairs[:, 1]
    bsum = np.zeros((K // block, len(pairs)))
    asum = np.zeros(len(pairs))
    for k in range(K):
        F = q @ M64.T
        p -= 0.5 * dt * F
        x = bf16_rn(q)
        bsum[k // block] += np.einsum("rk,rk->k", x[:, ii], x[:, jj])
        asum += np.einsum("rk,rk->k", np.abs(q[:, ii]), np.abs(q[:, jj]))
        p -= 0.5 * dt * F
        q += dt * p
    bmean = bsum / (block * R)
    ref = bmean.mean(axis=0)
    nb = K // block
    ref_err = np.sqrt(np.sum((bmean - ref) ** 2, axis=0) / (nb * (nb - 1)))
    scale = asum / (K * R)
    assert np.max(np.abs(vals - ref) / scale) <= 2.0 ** -9
    assert np.max(np.abs(errs - ref_err) / scale) <= 2.0 ** -8


# ------------------------------------------------------------------ error paths
def _nan_contexts():
    M, _, _ = syn.dense_spd(150, 1.0, 100.0, seed=301)
    a, c = syn.random_gle(4, seed=302, rate=3.0)
    rowptr, col, val = syn.lattice_csr(5, seed=303)
    pairs = np.concatenate([syn.diag_pairs(150)[:8], syn.random_pairs(150, 8, seed=304)])
    lat_pairs = syn.diag_pairs(125)[:16]
    return [
        ("dense fp32 list", dict(M=M.astype(np.float32), precision="fp32", pairs=pairs), pairs),
        ("dense tf32 all", dict(M=M.astype(np.float32), precision="tf32", track="all",
                                replicas=64), pairs),
        ("dense fp64 all", dict(M=M[:32, :32], precision="fp64", track="all"),
         syn.upper_pairs(32)[:16]),
        ("csr list", dict(csr=(rowptr, col, val.astype(np.float32), 125), pairs=lat_pairs),
         lat_pairs),
    ], a, c


@pytest.mark.parametrize("which", range(4))
def test_nonfinite_state_reaches_the_flush(which):
    """A NaN written into the momenta from the host spreads into the samples; the next
    FP64 block flush sees a non-finite block mean and every later read reports
    FTH_E_NONFINITE instead of returning numbers."""
    from paper_1402_2095_gb300 import FTH, FthError
    cases, a, c = _nan_contexts()
    name, kw, pairs = cases[which]
    kw = dict(kw)
    R = kw.pop("replicas", 8)
    f = FTH(**kw, a_p=a, c_p=c, dt=0.01, replicas=R, seed=5, block=5)
    f.run(7)
    f.poll()
    v, _ = f.elements(pairs)
    assert np.all(np.isfinite(v)), name
    p = f.get_state("p")
    p[R // 2, 3] = np.nan
    f.set_state("p", p)
    f.run(6)                                # completes at least one more block
    with pytest.raises(FthError) as ex:
        f.elements(pairs)
    assert ex.value.status == 7, name
    with pytest.raises(FthError) as ex:
        f.poll()
    assert ex.value.status == 7, name


@pytest.mark.parametrize("n,R", [(300, 64), (300, 256), (512, 256)])
def test_device_wait_timeout_is_reported(n, R):
    """fth_test_stall: the force launches issue no copies, so the main-loop waits of
    every CTA give up after 1 ms; the call reports FTH_E_TIMEOUT and the CUDA context
    stays usable (a new context afterwards runs and matches the oracle).  R = 64 takes
    the column-tiled kernel, n = 300 with R = 256 the split-K cluster kernel, n = 512
    with R = 256 the row-pair kernel with L2 reduce-adds."""
    from paper_1402_2095_gb300 import FTH, FthError
    M, _, _ = syn.dense_spd(n, 1.0, 100.0, seed=311)
    M32 = M.astype(np.float32)
    a, c = syn.random_gle(4, seed=312, rate=3.0)
    pairs = syn.diag_pairs(n)[:8]
    f = FTH(M=M32, a_p=a, c_p=c, dt=0.01, replicas=R, seed=6, precision="tf32", pairs=pairs,
            block=4)
    f.run(3)
    f.poll()
    f.test_stall(1_000_000)
    f.run(2)
    with pytest.raises(FthError) as ex:
        f.poll()
    assert ex.value.status == 6
    with pytest.raises(FthError) as ex:
        f.elements(pairs)
    assert ex.value.status == 6
    f.close()
    g = FTH(M=M32, a_p=a, c_p=c, dt=0.01, replicas=R, seed=7, precision="tf32", pairs=pairs,
            block=4)
    o = OracleFTH(M=M32.astype(np.float64), a_p=a, c_p=c, dt=0.01, replicas=R, seed=7, block=4,
                  pairs=pairs)
    g.run(20)
    o.run(20)
    g.poll()
    err = max(np.max(np.abs(g.get_state(k) - ref)) / np.max(np.abs(ref))
              for k, ref in (("q", o.q), ("p", o.p)))
    assert err <= 3e-2
