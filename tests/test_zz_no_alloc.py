"""The allocation-free entry point fth_dense_step_noalloc against the regular one.

Some callers cannot allocate device memory (a plugin whose framework owns the device
pool, a real-time loop that must not enter an allocator); fth_dense_step_noalloc serves
them with a static scratch array instead of a workspace.  Here two calls in a row,
through the C ABI on caller-owned torch buffers, must reproduce two steps of fth_run on
the same state, seed and kick indices, within the FP32 trajectory tolerance (1e-5) used
by the other parity tests.  This file is collected last on purpose."""
import ctypes

import numpy as np
import pytest

import fth_synth as syn

from gpu_util import gpu_ready

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not gpu_ready(), reason="needs a CUDA GPU and libfth.so")]


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-30))


def test_noalloc_two_calls_match_fth_run():
    import torch
    from paper_1402_2095_gb300 import FTH, binding

    n, R, ldr, s_aux, dt, seed = 200, 12, 12, 4, 0.01, 2024
    M, _, _ = syn.dense_spd(n, 1.0, 100.0, seed=5)
    M32 = M.astype(np.float32)
    a, c = syn.random_gle(s_aux, seed=6, rate=3.0)

    ref = FTH(M=M32, a_p=a, c_p=c, dt=dt, replicas=R, seed=seed, precision="fp32")
    ref.run(0)                                     # primed: next launch has kappa 1
    g = np.random.default_rng(7)
    q0 = g.standard_normal((R, n)).astype(np.float32).astype(np.float64)
    p0 = g.standard_normal((R, n)).astype(np.float32).astype(np.float64)
    s0 = g.standard_normal((R, s_aux, n)).astype(np.float32).astype(np.float64)
    ref.set_state("q", q0)
    ref.set_state("p", p0)
    ref.set_state("s", s0)

    dev = torch.device("cuda")
    Md = torch.from_numpy(M32).to(dev)
    qd = torch.from_numpy(np.ascontiguousarray(q0.T)).float().to(dev)           # [n][ldr]
    pd = torch.from_numpy(np.ascontiguousarray(p0.T)).float().to(dev)
    sd = torch.from_numpy(np.ascontiguousarray(np.transpose(s0, (1, 2, 0)))).float().to(dev)
    sample = torch.zeros((n, ldr), dtype=torch.float32, device=dev)
    T, S = binding.gle_propagator(a, c, dt)
    T = np.ascontiguousarray(T)
    S = np.ascontiguousarray(S)
    lib = binding.load()
    stream = torch.cuda.current_stream()

    from oracle import gle
    from oracle.fth import fused_step_elements
    To, So = gle.propagator(a, c, dt)
    elems = [(int(i), int(r)) for i, r in zip(g.integers(0, n, 40), g.integers(0, R, 40))]
    state = (q0, p0, s0)
    for kappa in (1, 2):
        # the oracle, one sampled (i, r) at a time, from the state before this call
        qn, pn, sn, xn = fused_step_elements(M32.astype(np.float64), *state, To, So, dt, seed,
                                             kappa, elems)
        ref.run(1)
        st = lib.fth_dense_step_noalloc(
            Md.data_ptr(), n, n, qd.data_ptr(), pd.data_ptr(), sd.data_ptr(), R, ldr, s_aux,
            T.ctypes.data, S.ctypes.data, dt, seed, kappa, 0, sample.data_ptr(),
            ctypes.c_void_p(stream.cuda_stream))
        assert st == 0
        torch.cuda.synchronize()
        assert _rel(qd.cpu().numpy().T, ref.get_state("q")) <= 1e-5
        assert _rel(pd.cpu().numpy().T, ref.get_state("p")) <= 1e-5
        assert _rel(np.transpose(sd.cpu().numpy(), (2, 0, 1)), ref.get_state("s")) <= 1e-5
        got_q, got_p = qd.cpu().numpy().T, pd.cpu().numpy().T
        got_s = np.transpose(sd.cpu().numpy(), (2, 0, 1))
        got_x = sample.cpu().numpy().T                 # p at the end of step kappa - 1
        for k, (i, r) in enumerate(elems):
            assert abs(got_q[r, i] - qn[k]) <= 1e-5 * (1 + abs(qn[k]))
            assert abs(got_p[r, i] - pn[k]) <= 1e-5 * (1 + abs(pn[k]))
            assert np.allclose(got_s[r, :, i], sn[k], rtol=1e-5, atol=1e-5)
            assert abs(got_x[r, i] - xn[k]) <= 1e-5 * (1 + abs(xn[k]))
        state = (got_q.astype(np.float64), got_p.astype(np.float64), got_s.astype(np.float64))


def test_noalloc_rejects_sizes_beyond_scratch():
    import torch
    from paper_1402_2095_gb300 import binding
    lib = binding.load()
    x = torch.zeros(64, device="cuda")
    T = np.eye(1)
    S = np.zeros((1, 1))
    # n * ldr = 4096 * 1028 > 4,194,304 floats: refused before any device work
    st = lib.fth_dense_step_noalloc(x.data_ptr(), 4096, 4096, x.data_ptr(), x.data_ptr(), None,
                                    1028, 1028, 0, T.ctypes.data, S.ctypes.data, 0.01, 1, 1, 0,
                                    None, None)
    assert st == 3
    # absurd sizes are refused without overflowing n * ldr
    st = lib.fth_dense_step_noalloc(x.data_ptr(), 1 << 40, 1 << 40, x.data_ptr(), x.data_ptr(),
                                    None, 1 << 40, 1 << 40, 0, T.ctypes.data, S.ctypes.data,
                                    0.01, 1, 1, 0, None, None)
    assert st == 3
    # one row with more replicas than the element-wise step's grid takes (65,535 x 32)
    st = lib.fth_dense_step_noalloc(x.data_ptr(), 1, 1, x.data_ptr(), x.data_ptr(), None,
                                    1, 65535 * 32 + 4, 0, T.ctypes.data, S.ctypes.data, 0.01, 1,
                                    1, 0, None, None)
    assert st == 3


def test_noalloc_widest_row_runs():
    # n = 1 with the widest replica stride accepted (65,535 x 32): grids stay in range
    import torch
    from paper_1402_2095_gb300 import binding
    lib = binding.load()
    ldr = 65535 * 32
    dev = torch.device("cuda")
    M = torch.full((1, 1), 4.0, device=dev)
    q = torch.ones(ldr, device=dev)
    p = torch.zeros(ldr, device=dev)
    sample = torch.zeros(ldr, device=dev)
    T = np.eye(1)
    S = np.zeros((1, 1))
    st = lib.fth_dense_step_noalloc(M.data_ptr(), 1, 1, q.data_ptr(), p.data_ptr(), None, ldr,
                                    ldr, 0, T.ctypes.data, S.ctypes.data, 0.01, 3, 1, 0,
                                    sample.data_ptr(), None)
    assert st == 0
    torch.cuda.synchronize()
    # noise-free (S = 0, T = I) with M = 4 from q = 1, p = 0: the end half kicks
    # p = -(dt/2) 4, the sample takes it, the start half kicks again and drifts q
    dt = 0.01
    p_end = -0.5 * dt * 4.0
    p_new = 2 * p_end
    q_new = 1.0 + dt * p_new
    for t, want in ((sample, p_end), (p, p_new), (q, q_new)):
        assert torch.allclose(t, torch.full_like(t, want), rtol=0, atol=1e-6)
