"""GPU parity: the CUDA path through the C ABI against the FP64 oracle on the same
seeded inputs and the same Philox noise stream.

Tolerances (derived from the arithmetic):
  FP32 paths  trajectories  max_t |x_gpu - x_cpu|_inf / max_t |x_cpu|_inf <= 1e-5
              (FP32 state and force, FP32 logf/sincospif normals vs FP64 libm: per-step
              relative round-off ~1e-7, damped linear dynamics does not amplify it);
  FP64 path   1e-11 (same arithmetic in FP64, normals differ in the last ulp);
  BF16X3      force relative error <= 2^-15 (hi+lo split keeps ~16 mantissa bits);
  TF32        force relative error <= 2^-9 (10-bit mantissa operands, FP32 accumulate);
  accumulators  FP32 block partials: values within 1e-4 of the diagonal scale.
"""
import numpy as np
import pytest

import fth_synth as syn
from oracle import matfun
from oracle.fth import fused_step_elements

from gpu_util import bf16_rn, gpu_ready, make_pair, state_rel_err, trace_terms

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not gpu_ready(), reason="needs a CUDA GPU and libfth.so")]


def _dense(n, lo=1.0, hi=100.0, seed=5):
    M, _, _ = syn.dense_spd(n, lo, hi, seed=seed)
    return M


def _trajectory(g, o, steps, chunks):
    diff = ref = 0.0
    for _ in range(chunks):
        g.run(steps // chunks)
        o.run(steps // chunks)
        for name, r in (("q", o.q), ("p", o.p), ("s", o.s)):
            if r.size:
                diff = max(diff, float(np.max(np.abs(g.get_state(name) - r))))
                ref = max(ref, float(np.max(np.abs(r))))
    return diff / ref


# ------------------------------------------------------------------ trajectories
@pytest.mark.parametrize("n,R,s", [(200, 12, 4), (37, 5, 2), (50, 8, 0), (1, 1, 4)])
def test_dense_fp32_trajectory(n, R, s):
    a, c = syn.random_gle(s, seed=11 + s, rate=3.0)
    g, o = make_pair(_dense(n), a_p=a, c_p=c, dt=0.01, R=R, seed=1234)
    assert _trajectory(g, o, 1000, 4) <= 1e-5


@pytest.mark.parametrize("L,R", [(6, 12), (5, 7)])
def test_csr_trajectory(L, R):
    rowptr, col, val = syn.lattice_csr(L, seed=9)
    a, c = syn.random_gle(4, seed=12, rate=2.0)
    g, o = make_pair(csr=(rowptr, col, val, L ** 3), a_p=a, c_p=c, dt=0.1 / np.sqrt(14.5), R=R,
                     seed=77)
    assert _trajectory(g, o, 1000, 4) <= 1e-5


@pytest.mark.parametrize("n,R", [(32, 16), (45, 3), (20, 5), (1, 2)])
def test_fp64_trajectory(n, R):
    a, c = syn.random_gle(4, seed=13, rate=3.0)
    g, o = make_pair(_dense(n), a_p=a, c_p=c, dt=0.01, R=R, seed=99, precision="fp64")
    assert _trajectory(g, o, 1000, 4) <= 1e-11


@pytest.mark.parametrize("precision,tol", [("tf32", 3e-2), ("bf16x3", 3e-4)])
def test_tensor_core_trajectory(precision, tol):
    a, c = syn.random_gle(4, seed=14, rate=3.0)
    g, o = make_pair(_dense(300), a_p=a, c_p=c, dt=0.01, R=70, seed=5, precision=precision,
                     M_oracle=_dense(300))
    assert _trajectory(g, o, 400, 2) <= tol


@pytest.mark.parametrize("n", [512, 470])
def test_tensor_core_trajectory_row_pair_kernel(n):
    """TF32 with the padded order a multiple of 256 and 128 < R <= 256: the row-pair force
    with L2 reduce-adds and the element-wise step that zeroes MQ after reading it, chained
    by programmatic dependent launch (n = 470 leaves a part-filled row tile and padding
    rows).  400 steps against the oracle on the first 16 of the 256 replicas: replicas
    evolve independently and draw their own noise, so the oracle needs no others."""
    from oracle.fth import OracleFTH
    from paper_1402_2095_gb300 import FTH
    R, Ro = 256, 16
    a, c = syn.random_gle(4, seed=14, rate=3.0)
    M = _dense(n).astype(np.float32)
    g = FTH(M=M, a_p=a, c_p=c, dt=0.01, replicas=R, seed=5, precision="tf32")
    o = OracleFTH(M=_dense(n), a_p=a, c_p=c, dt=0.01, replicas=Ro, seed=5)
    diff = ref = 0.0
    for _ in range(4):
        g.run(100)
        o.run(100)
        for name, r in (("q", o.q), ("p", o.p), ("s", o.s)):
            diff = max(diff, float(np.max(np.abs(g.get_state(name)[:Ro] - r))))
            ref = max(ref, float(np.max(np.abs(r))))
    g.poll()
    assert diff / ref <= 3e-2


# ------------------------------------------------------------------ force kernels alone
def _force_through_prologue(M, q0, precision, dt=0.01):
    """With A_p = 0 and C_p = 0 (T = I, S = 0) and p = 0, the prologue leaves
    p = -(dt/2) M q0, so the force GEMM is read back through the C ABI."""
    from paper_1402_2095_gb300 import FTH
    R, n = q0.shape
    z = np.zeros((5, 5))
    f = FTH(M=M, a_p=z, c_p=z, dt=dt, replicas=R, seed=0, precision=precision)
    f.set_state("q", q0)
    f.run(0)
    return -f.get_state("p") / (0.5 * dt)


@pytest.mark.parametrize("precision,bound", [("fp32", 2e-6), ("tf32", 2.0 ** -9),
                                             ("bf16x3", 2.0 ** -15)])
@pytest.mark.parametrize("n,R", [(300, 70), (128, 64), (77, 5),     # column-tiled kernel
                                 (300, 200), (77, 250), (640, 256),   # split-K cluster kernel
                                 (512, 200), (1000, 256), (1024, 140),   # several row blocks
                                 (2048, 256), (4096, 200)])   # K shares longer than the ring
def test_force_gemm(precision, bound, n, R):
    M = _dense(n, seed=21).astype(np.float32).astype(np.float64)
    q0 = syn.gaussian_state((R, n), seed=22)
    got = _force_through_prologue(M, q0, precision)
    ref = q0 @ M.T
    scale = np.abs(q0) @ np.abs(M).T          # sum_k |M_ik q_k|: the error scale
    assert np.max(np.abs(got - ref) / scale) <= bound


# ------------------------------------------------------------------ accumulators
@pytest.mark.parametrize("track", ["list", "diag", "all"])
def test_accumulation_parity_fp32(track):
    n, R = 130, 12
    a, c = syn.random_gle(4, seed=15, rate=3.0)
    pairs = np.concatenate([syn.random_pairs(n, 40, seed=3), syn.diag_pairs(n)[:10]])
    g, o = make_pair(_dense(n), a_p=a, c_p=c, dt=0.01, R=R, seed=3, track=track,
                     pairs=pairs if track == "list" else None, burnin=30, block=50, stack=3)
    g.run(333)
    o.run(333)
    vals_o, errs_o = o.elements()
    vals_g, errs_g = g.elements(o.pairs)
    scale = np.max(np.abs(vals_o))
    assert np.max(np.abs(vals_g - vals_o)) <= 1e-4 * scale
    assert np.allclose(errs_g, errs_o, rtol=1e-2, atol=1e-4 * scale)
    info = g.info()
    assert info["blocks"] == o.nblocks == (333 - 30) // 50


@pytest.mark.parametrize("R,stack", [(32, 4), (64, 4), (64, 8), (64, 16), (64, 3)])
def test_accumulation_parity_row_grouped_pairs(R, stack):
    # CSR lattice with diagonal + nearest-neighbour pairs: the row-grouped pass (a warp holds
    # row i's staged samples and streams its partners) for 128-, 256-, 512- and 1024-column
    # stacks (a block of 40 samples also ends in shorter stacks), and a 3-sample stack (192
    # columns: the ungrouped pass), against the oracle on the same noise
    L = 6
    n = L ** 3
    rowptr, col, val = syn.lattice_csr(L, seed=61)
    a, c = syn.random_gle(4, seed=62, rate=3.0)
    pairs = np.concatenate([syn.diag_pairs(n), syn.lattice_nn_pairs(L)])
    g, o = make_pair(csr=(rowptr, col, val, n), a_p=a, c_p=c, dt=0.1 / np.sqrt(14.5), R=R,
                     seed=63, pairs=pairs, burnin=10, block=40, stack=stack)
    g.run(333)
    o.run(333)
    vals_o, errs_o = o.elements()
    vals_g, errs_g = g.elements(o.pairs)
    scale = np.max(np.abs(vals_o))
    assert np.max(np.abs(vals_g - vals_o)) <= 1e-4 * scale
    assert np.allclose(errs_g, errs_o, rtol=1e-2, atol=1e-4 * scale)


def test_accumulation_parity_fp64_all():
    n, R = 24, 6
    a, c = syn.random_gle(4, seed=16, rate=3.0)
    g, o = make_pair(_dense(n), a_p=a, c_p=c, dt=0.01, R=R, seed=4, track="all",
                     precision="fp64", burnin=17, block=40)
    g.run(500)
    o.run(500)
    vals_o, errs_o = o.elements()
    vals_g, errs_g = g.elements(o.pairs)
    assert np.allclose(vals_g, vals_o, rtol=1e-10, atol=1e-12)
    assert np.allclose(errs_g, errs_o, rtol=1e-8, atol=1e-14)


@pytest.mark.parametrize("precision,n", [("tf32", 300), ("bf16x3", 300), ("fp32", 300),
                                         ("tf32", 500), ("bf16x3", 500)])
def test_all_elements_one_sample(precision, n):
    # A_p = C_p = 0, p0 = 0, observable q: the single sample of run(1) is
    # q1 = q0 - (dt^2/2) M q0 exactly, so <q1 q1^T> is known for every element.
    # n = 300: three 128-row blocks (128 x 256 accumulator tiles); n = 500: four blocks,
    # 256 x 256 tiles on and off the diagonal, padded rows at the end.
    from paper_1402_2095_gb300 import FTH
    R, dt = 64, 0.01
    M = _dense(n, seed=31).astype(np.float32).astype(np.float64)
    q0 = syn.gaussian_state((R, n), seed=32)
    z = np.zeros((5, 5))
    f = FTH(M=M, a_p=z, c_p=z, dt=dt, replicas=R, seed=0, precision=precision, track="all",
            block=1, observable="q")
    f.set_state("q", q0)
    f.run(1)
    q1 = q0 - 0.5 * dt * dt * q0 @ M.T
    # the tensor-core forms stage the sample in BF16 (round to nearest) for the SYRK
    x1 = bf16_rn(q1) if precision != "fp32" else q1
    pairs = syn.upper_pairs(n)
    vals, _ = f.elements(pairs)
    ref = np.einsum("ri,rj->ij", x1, x1)[pairs[:, 0], pairs[:, 1]] / R
    scale = np.einsum("ri,rj->ij", np.abs(q1), np.abs(q1))[pairs[:, 0], pairs[:, 1]] / R
    bound = 2.0 ** -9 if precision != "fp32" else 1e-6
    assert np.max(np.abs(vals - ref) / scale) <= bound
    if precision != "fp32":
        # and not the unrounded products: BF16 staging moves them by up to 2^-7
        unrounded = np.einsum("ri,rj->ij", q1, q1)[pairs[:, 0], pairs[:, 1]] / R
        assert np.max(np.abs(vals - unrounded) / scale) > 2.0 ** -12


def test_all_elements_one_sample_more_blocks_than_sms():
    # n = 4608: 171 blocks of 256 x 256 on or above the diagonal, more than the 152 SMs,
    # so accumulation CTAs loop over several blocks (copies of the next block run ahead
    # while the accumulator drains).  Same closed form as above, on sampled elements.
    from paper_1402_2095_gb300 import FTH
    n, R, dt = 4608, 64, 0.01
    M = _dense(n, seed=41).astype(np.float32).astype(np.float64)
    q0 = syn.gaussian_state((R, n), seed=42)
    z = np.zeros((5, 5))
    f = FTH(M=M, a_p=z, c_p=z, dt=dt, replicas=R, seed=0, precision="tf32", track="all",
            block=1, observable="q")
    f.set_state("q", q0)
    f.run(1)
    q1 = q0 - 0.5 * dt * dt * q0 @ M.T
    x1 = bf16_rn(q1)
    g = np.random.default_rng(43)
    pairs = np.concatenate([syn.diag_pairs(n)[g.choice(n, 1024, replace=False)],
                            syn.random_pairs(n, 60000, seed=44)])
    vals, _ = f.elements(pairs)
    i, j = pairs[:, 0], pairs[:, 1]
    ref = np.einsum("rk,rk->k", x1[:, i], x1[:, j]) / R
    scale = np.einsum("rk,rk->k", np.abs(q1[:, i]), np.abs(q1[:, j])) / R
    assert np.max(np.abs(vals - ref) / scale) <= 2.0 ** -9


# ------------------------------------------------------------------ stationary estimate
def _zscores(vals, errs, ref):
    return (vals - ref) / errs


def test_stationary_fp64_small_dense():
    # N = 32 dense, lambda log-uniform [1, 100], R = 16, 1e5 steps: every one of the
    # 528 elements of <p p^T> against the exact expected estimate U g U^T.
    n, R, steps, block = 32, 16, 100000, 1000
    M = _dense(n, 1.0, 100.0, seed=1403)
    a, c = syn.random_gle(4, seed=1404, rate=4.0)
    dt = 0.1 / np.sqrt(100.0)
    from paper_1402_2095_gb300 import FTH
    f = FTH(M=M, a_p=a, c_p=c, dt=dt, replicas=R, seed=1405, precision="fp64", track="all",
            block=block)
    f.run(steps)
    pairs = syn.upper_pairs(n)
    vals, errs = f.elements(pairs)
    from oracle import gle
    T, S = gle.propagator(a, c, dt)
    ref = matfun.g_mean_of_matrix(M, T, S, dt, 0, steps)[pairs[:, 0], pairs[:, 1]]
    z = _zscores(vals, errs, ref)
    sample = np.random.default_rng(7).choice(len(pairs), 32, replace=False)
    assert np.all(np.abs(z[sample]) < 4.0), z[sample]
    assert np.all(np.abs(z) < 5.0)
    assert 0.5 < np.mean(z ** 2) < 2.0


@pytest.mark.parametrize("precision", ["fp32", "bf16x3"])
def test_stationary_fp32_dense(precision):
    n, R, steps, block = 64, 64, 20000, 500
    M = _dense(n, 1.0, 50.0, seed=41)
    a, c = syn.random_gle(4, seed=42, rate=3.0)
    dt = 0.1 / np.sqrt(50.0)
    from paper_1402_2095_gb300 import FTH
    f = FTH(M=M.astype(np.float32), a_p=a, c_p=c, dt=dt, replicas=R, seed=43,
            precision=precision, track="all", block=block)
    f.run(steps)
    pairs = syn.upper_pairs(n)
    vals, errs = f.elements(pairs)
    from oracle import gle
    T, S = gle.propagator(a, c, dt)
    ref = matfun.g_mean_of_matrix(M.astype(np.float32).astype(np.float64), T, S, dt, 0,
                                  steps)[pairs[:, 0], pairs[:, 1]]
    z = _zscores(vals, errs, ref)
    sample = np.random.default_rng(8).choice(len(pairs), 32, replace=False)
    assert np.all(np.abs(z[sample]) < 4.0), z[sample]
    assert 0.5 < np.mean(z ** 2) < 2.0


def test_stationary_csr_lattice():
    L, R, steps, block = 6, 64, 20000, 500
    rowptr, col, val = syn.lattice_csr(L, seed=51)
    n = L ** 3
    a, c = syn.random_gle(4, seed=52, rate=3.0)
    dt = 0.1 / np.sqrt(14.5)
    pairs = np.concatenate([syn.diag_pairs(n), syn.lattice_nn_pairs(L)])
    from paper_1402_2095_gb300 import FTH
    f = FTH(csr=(rowptr, col, val.astype(np.float32), n), a_p=a, c_p=c, dt=dt, replicas=R,
            seed=53, pairs=pairs, block=block)
    f.run(steps)
    vals, errs = f.elements(pairs)
    from oracle import gle
    T, S = gle.propagator(a, c, dt)
    Md = syn.csr_to_dense(rowptr, col, val.astype(np.float32).astype(np.float64), n)
    ref = matfun.g_mean_of_matrix(Md, T, S, dt, 0, steps)[pairs[:, 0], pairs[:, 1]]
    z = _zscores(vals, errs, ref)
    sample = np.random.default_rng(9).choice(len(pairs), 32, replace=False)
    assert np.all(np.abs(z[sample]) < 4.0), z[sample]
    assert 0.5 < np.mean(z ** 2) < 2.0


# ------------------------------------------------------------------ edge cases and errors
def test_edge_cases():
    from paper_1402_2095_gb300 import FTH, FthError
    a, c = syn.random_gle(4, seed=61, rate=2.0)
    M = _dense(10)
    f = FTH(M=M, a_p=a, c_p=c, dt=0.01, replicas=3, seed=1, pairs=np.zeros((0, 2)), burnin=5)
    f.run(0)
    assert f.info()["primed"] == 1 and f.info()["steps"] == 0
    f.run(3)
    assert f.elements(np.zeros((0, 2))) [0].size == 0
    f2 = FTH(M=M, a_p=a, c_p=c, dt=0.01, replicas=3, seed=1, pairs=[[0, 1]], burnin=100)
    f2.run(10)
    v, e = f2.elements([[1, 0]])
    assert np.isnan(v[0]) and np.isnan(e[0])       # still in burn-in
    with pytest.raises(FthError) as ex:
        f2.elements([[2, 3]])
    assert ex.value.status == 8
    bad = M.copy()
    bad[3, 3] = -1.0
    with pytest.raises(FthError) as ex:
        FTH(M=bad, a_p=a, c_p=c, dt=0.01, replicas=2)
    assert ex.value.status == 2
    with pytest.raises(FthError) as ex:
        FTH(M=M, a_p=a, c_p=c, dt=0.01, replicas=2, pairs=[[0, 10]])
    assert ex.value.status == 1


# ------------------------------------------------------------------ full-size samples
def test_full_size_dense_tf32_all_sampled():
    # N = 4096, R = 256, TF32 force, all elements: the launch configuration of the
    # benchmark.  Checked on sampled (i, r) against the oracle computed one by one.
    import torch
    from paper_1402_2095_gb300 import FTH
    n, R, dt = 4096, 256, 0.1 / np.sqrt(1000.0)
    M, _, _ = syn.dense_spd(n, 1.0, 1000.0, seed=1402 + 2)
    M32 = M.astype(np.float32)
    a, c = syn.random_gle(4, seed=71, rate=5.0)
    f = FTH(M=torch.from_numpy(M32).cuda(), a_p=a, c_p=c, dt=dt, replicas=R, seed=72,
            precision="tf32", track="all", block=4)
    g = np.random.default_rng(73)
    q0 = g.standard_normal((R, n))
    p0 = g.standard_normal((R, n))
    s0 = g.standard_normal((R, 4, n))
    f.run(0)                       # prologue done: the state below is a primed state
    f.set_state("q", q0)
    f.set_state("p", p0)
    f.set_state("s", s0)
    kappa = f.info()["steps"] + 1
    f.run(1)
    elems = [(int(i), int(r)) for i, r in zip(g.integers(0, n, 48), g.integers(0, R, 48))]
    from oracle import gle
    T, S = gle.propagator(a, c, dt)
    qn, pn, sn, _ = fused_step_elements(M32.astype(np.float64), q0, p0, s0, T, S, dt, 72, kappa,
                                        elems)
    q1, p1, s1 = f.get_state("q"), f.get_state("p"), f.get_state("s")
    for k, (i, r) in enumerate(elems):
        assert abs(q1[r, i] - qn[k]) <= 1e-3 * (1 + abs(qn[k]))
        assert abs(p1[r, i] - pn[k]) <= 2e-3 * (1 + abs(pn[k]))
        assert np.allclose(s1[r, :, i], sn[k], rtol=1e-3, atol=1e-3)


def test_full_size_lattice_sampled():
    # 64^3 lattice (N = 262144), R = 64, CSR FP32: one fused step from a random
    # primed state, sampled elements against the oracle one by one.
    from paper_1402_2095_gb300 import FTH
    L, R = 64, 64
    n = L ** 3
    rowptr, col, val = syn.lattice_csr(L, seed=1402 + 3)
    v32 = val.astype(np.float32)
    a, c = syn.random_gle(4, seed=81, rate=2.0)
    dt = 0.1 / np.sqrt(14.5)
    f = FTH(csr=(rowptr, col, v32, n), a_p=a, c_p=c, dt=dt, replicas=R, seed=82, track="diag",
            block=8)
    g = np.random.default_rng(83)
    q0 = g.standard_normal((R, n)).astype(np.float32).astype(np.float64)
    p0 = g.standard_normal((R, n)).astype(np.float32).astype(np.float64)
    s0 = g.standard_normal((R, 4, n)).astype(np.float32).astype(np.float64)
    f.run(0)
    f.set_state("q", q0)
    f.set_state("p", p0)
    f.set_state("s", s0)
    kappa = f.info()["steps"] + 1
    f.run(1)
    elems = [(int(i), int(r)) for i, r in zip(g.integers(0, n, 64), g.integers(0, R, 64))]
    from oracle import gle
    T, S = gle.propagator(a, c, dt)
    import scipy.sparse as sp
    Ms = sp.csr_matrix((v32.astype(np.float64), col, rowptr), shape=(n, n))
    qn, pn, sn, _ = fused_step_elements(Ms, q0, p0, s0, T, S, dt, 82, kappa, elems)
    q1, p1, s1 = f.get_state("q"), f.get_state("p"), f.get_state("s")
    for k, (i, r) in enumerate(elems):
        assert abs(q1[r, i] - qn[k]) <= 1e-5 * (1 + abs(qn[k]))
        assert abs(p1[r, i] - pn[k]) <= 1e-5 * (1 + abs(pn[k]))
        assert np.allclose(s1[r, :, i], sn[k], rtol=1e-5, atol=1e-5)


# ------------------------------------------------------------------ linear functionals
def _functional_from_samples(samples, burnin, block, pairs, w):
    """Value and block error bar of sum_k w_k <x_i x_j> straight from the oracle's
    samples (steps, R, n): per-sample replica averages, blocks of `block` samples."""
    x = samples[burnin:]
    per = np.einsum("k,tkr->t", w, x[:, :, pairs[:, 0]].transpose(0, 2, 1) *
                    x[:, :, pairs[:, 1]].transpose(0, 2, 1)) / x.shape[1]
    nb = per.shape[0] // block
    bm = per[:nb * block].reshape(nb, block).mean(axis=1)
    err = np.sqrt(np.sum((bm - bm.mean()) ** 2) / (nb * (nb - 1))) if nb >= 2 else np.nan
    return per.mean(), err


def test_functionals_csr_trace_and_trace_with_operator():
    """Tr f(M) and Tr M f(M) on a lattice (tracked: diagonal + nearest neighbours)."""
    import scipy.sparse as sp
    L = 5
    n = L ** 3
    rowptr, col, val = syn.lattice_csr(L, seed=31)
    a, c = syn.random_gle(4, seed=32, rate=2.0)
    pairs = np.concatenate([syn.diag_pairs(n), syn.lattice_nn_pairs(L)])
    g, o = make_pair(csr=(rowptr, col, val, n), a_p=a, c_p=c, dt=0.1 / np.sqrt(14.5), R=8,
                     seed=33, pairs=pairs, burnin=20, block=40)
    Mo = sp.csr_matrix((val.astype(np.float32).astype(np.float64), col, rowptr), shape=(n, n))
    terms = [trace_terms(n=n), trace_terms(O=Mo)]
    # the library builds the weights itself (NULL operator: Tr f(M); a CSR operator)
    ids = [g.add_trace(), g.add_trace(O=Mo)]
    g.run(420)
    samples = o.run(420, keep_samples=True)
    for fid, (p, w) in zip(ids, terms):
        v, e = g.functional(fid)
        vo, eo = _functional_from_samples(samples, 20, 40, p, w)
        assert abs(v - vo) <= 1e-4 * abs(vo)
        assert abs(e - eo) <= 1e-3 * eo
        # the value is the weighted sum of the element estimates
        ve, _ = g.elements(p)
        assert abs(v - float(np.dot(w, ve))) <= 1e-12 * abs(v)


def test_functional_fp64_dense_operator():
    n = 12
    M = _dense(n)
    a, c = syn.random_gle(3, seed=34, rate=3.0)
    g, o = make_pair(M, a_p=a, c_p=c, dt=0.01, R=4, seed=35, precision="fp64", track="all",
                     burnin=0, block=25)
    p, w = trace_terms(O=M)
    fid = g.add_trace(O=M)                     # dense FP64 operator, weights built by the library
    g.run(250)
    samples = o.run(250, keep_samples=True)
    v, e = g.functional(fid)
    vo, eo = _functional_from_samples(samples, 0, 25, p, w)
    assert abs(v - vo) <= 1e-10 * abs(vo)
    assert abs(e - eo) <= 1e-8 * eo


def test_functional_dense_all_elements_tf32_tiles():
    """Functionals over the tile-packed all-elements accumulators of the tensor-core path
    (SYRK on the side stream, block fold before the flush)."""
    n = 200
    M = _dense(n, seed=71)
    a, c = syn.random_gle(4, seed=72, rate=3.0)
    g, o = make_pair(M, a_p=a, c_p=c, dt=0.01, R=64, seed=73, precision="bf16x3", track="all",
                     burnin=10, block=30, M_oracle=M)
    p, w = trace_terms(O=M)
    fid = g.add_functional(p, w)               # explicit weights through fth_functional_add
    tid = g.add_trace()
    g.run(310)
    samples = o.run(310, keep_samples=True)
    for f_id, (pp, ww) in ((fid, (p, w)), (tid, trace_terms(n=n))):
        v, e = g.functional(f_id)
        vo, eo = _functional_from_samples(samples, 10, 30, pp, ww)
        # BF16x3 force: trajectories agree to ~3e-4 of their scale
        assert abs(v - vo) <= 2e-3 * abs(vo)
        assert abs(e - eo) <= 2e-2 * eo


def test_trace_of_log_on_paper_m1_lattice():
    """End to end on the paper's M1 recipe at n = 7: the ln fit on [e, 100e], M1 scaled
    into it, Tr ln(r M1) from the trace functional, against the oracle's exact expected
    running mean (within 4 error bars) and through the inverse transform against
    Tr ln M1 (within the error bar plus the fit's bias)."""
    import scipy.sparse as sp
    import scipy.sparse.linalg as spla
    from oracle import gle
    from paper_1402_2095_gb300 import FTH, fit, transforms
    n1 = 7
    N = n1 ** 3
    rowptr, col, val = syn.m1_csr(n1, seed=91)
    A = sp.csr_matrix((val, col, rowptr), shape=(N, N))
    lo = float(spla.eigsh(A, k=1, which="SA", return_eigenvectors=False)[0])
    a_p, c_p, dt, rep = fit.load_gle("log_e_100e")
    r = float(np.e) * 1.0005 / lo
    v32 = (r * val).astype(np.float32)
    g = FTH(csr=(rowptr, col, v32, N), a_p=a_p, c_p=c_p, dt=dt, replicas=64, seed=92,
            track="diag", block=500)
    fid = g.add_trace()
    steps = 6000
    g.run(steps)
    tr_s, err_s = g.functional(fid)
    Ms = sp.csr_matrix((v32.astype(np.float64), col, rowptr), shape=(N, N)).toarray()
    lam = np.linalg.eigvalsh(Ms)
    T, S = gle.propagator(a_p, c_p, dt)
    expected = float(np.sum(gle.mode_response_mean(lam, T, S, dt, 0, steps)))
    assert abs(tr_s - expected) <= 4 * err_s
    exact_log_trace = float(np.sum(np.log(np.linalg.eigvalsh(A.toarray()))))
    got = transforms.log_trace_from_scaled(tr_s, N, r)
    assert abs(got - exact_log_trace) <= 4 * err_s + 2 * rep["max_rel_err"] * abs(tr_s)
