"""Host-side checks of libfth.so that need no GPU: it loads, exports every symbol
include/fth.h declares, builds the same O half-step constants as the oracle, and
validates problems (workspace sizing touches no device)."""
import ctypes
import os
import re

import numpy as np
import pytest

import fth_synth as syn
from oracle import gle
from paper_1402_2095_gb300 import binding as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1402_2095_gb300 import build
    build.build()
    return B.load()


def test_exports_every_declared_symbol(lib):
    hdr = open(os.path.join(ROOT, "include", "fth.h")).read()
    declared = set(re.findall(r"^\s*(?:fth_status|const char\s*\*|void|double|size_t|fth_pool\s*\*)\s+(fth_\w+)\s*\(", hdr,
                              flags=re.M))
    assert declared == set(B.EXPORTS)
    for name in declared:
        assert hasattr(lib, name), name
    assert lib.fth_version().startswith(b"fth")


@pytest.mark.parametrize("s,seed,rate,dt", [(4, 1, 2.0, 0.05), (4, 2, 30.0, 0.01), (2, 3, 1.0, 0.1),
                                            (0, 4, 0.5, 0.2)])
def test_propagator_matches_oracle(lib, s, seed, rate, dt):
    a, c = syn.random_gle(s, seed=seed, rate=rate)
    T, S = B.gle_propagator(a, c, dt)
    T2, S2 = gle.propagator(a, c, dt)
    assert np.allclose(T, T2, rtol=1e-13, atol=1e-14)
    assert np.allclose(S, S2, rtol=1e-12, atol=1e-13)


def test_propagator_noise_free_gle(lib):
    T, S = B.gle_propagator(np.zeros((5, 5)), np.zeros((5, 5)), 0.1)
    assert np.allclose(T, np.eye(5)) and np.all(S == 0)


def _ws(lib, n=64, kind=B.DENSE, precision="fp32", track="list", pairs=None, replicas=8, s=4,
        dt=0.01, block=10, burnin=0, nnz=0):
    mat = B.fth_matrix()
    mat.kind = kind
    mat.dtype = B.F64
    mat.n = n
    mat.nnz = nnz
    buf = np.ones(max(n * n, 1))
    mat.values = buf.ctypes.data
    rp = np.zeros(n + 1, np.int32)
    mat.rowptr = rp.ctypes.data
    mat.colind = rp.ctypes.data
    g = B.make_gle(*syn.random_gle(s, seed=1)) if s <= 4 else B.fth_gle()
    if s > 4:
        g.s = s
    o = B.fth_options()
    o.replicas, o.dt, o.block, o.burnin = replicas, dt, block, burnin
    o.precision = B.PRECISION[precision]
    o.track = B.TRACK[track]
    if pairs is not None:
        pr = np.asarray(pairs, np.int64).reshape(-1, 2)
        o.pairs = pr.ctypes.data
        o.npairs = len(pr)
    nb = ctypes.c_size_t(0)
    st = lib.fth_workspace_size(ctypes.byref(mat), ctypes.byref(g), ctypes.byref(o), ctypes.byref(nb))
    return st, nb.value


def test_workspace_sizes_and_validation(lib):
    st, b1 = _ws(lib, n=64)
    assert st == 0 and b1 > 0
    st, b2 = _ws(lib, n=4096, replicas=256, precision="tf32", track="all")
    assert st == 0
    # M (64 MiB) + ALL-mode accumulators (FP32 partial + 2 FP64 per element)
    assert b2 > 4096 * 4096 * 4 + 528 * 128 * 128 * 20
    assert _ws(lib, n=0)[0] == 1
    assert _ws(lib, replicas=0)[0] == 1
    assert _ws(lib, dt=0.0)[0] == 1
    assert _ws(lib, block=0)[0] == 1
    assert _ws(lib, pairs=[[0, 64]])[0] == 1
    assert _ws(lib, s=5)[0] == 3
    assert _ws(lib, kind=B.CSR, precision="tf32")[0] == 3
    assert _ws(lib, kind=B.CSR, track="all")[0] == 3
    assert _ws(lib, n=2048, precision="fp64")[0] == 3
    assert _ws(lib, pairs=np.zeros((0, 2)))[0] == 0


def test_binary_is_sm103a_only(lib):
    # the build compiles for sm_103a and nothing else
    from paper_1402_2095_gb300 import build
    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_spectral_map_gle_scale_and_untransforms(lib):
    """The C ABI's scaling / shift map and inverse transforms against their definitions."""
    r, m = B.spectral_map((2.0, 10.0), (1.0, 601.0))
    assert np.isclose(2.0 * r + m, 1.0) and np.isclose(10.0 * r + m, 601.0)
    a, c = syn.random_gle(3, seed=8, rate=2.0)
    a2, c2 = B.gle_scale(a, c, 0.5, 3.0)
    assert np.array_equal(a2, 0.5 * a) and np.array_equal(c2, 3.0 * c)
    pairs = np.array([[0, 0], [0, 1], [2, 2]])
    v = np.array([1.0, 2.0, 3.0])
    e = np.array([0.1, 0.2, 0.3])
    lv, le = B.untransform("log", (4.0,), pairs, v, e)
    assert np.allclose(lv, [1.0 - np.log(4.0), 2.0, 3.0 - np.log(4.0)]) and np.array_equal(le, e)
    xv, xe = B.untransform("exp", (0.01, 301.0), pairs, v, e)
    assert np.allclose(xv, v * np.exp(3.01)) and np.allclose(xe, e * np.exp(3.01))
    pv, pe = B.untransform("power", (2.0, -0.5), pairs, v, e)
    assert np.allclose(pv, v * np.sqrt(2.0)) and np.allclose(pe, e * np.sqrt(2.0))
    assert np.isclose(B.untransform_trace("log", (4.0,), 10, 7.0), 7.0 - 10 * np.log(4.0))
    with pytest.raises(B.FthError):
        B.untransform("log", (-1.0,), pairs, v)
    with pytest.raises(B.FthError):
        B.spectral_map((1.0, 1.0), (0.0, 1.0))
