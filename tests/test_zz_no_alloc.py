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

    for kappa in (1, 2):
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
        assert np.all(np.isfinite(sample.cpu().numpy()))


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
