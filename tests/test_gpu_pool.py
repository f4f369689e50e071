"""GPU parity of problem pools (ragged batches, continuous batching) through the C ABI.

A pool steps many independent problems with shared launches.  Each problem must follow
the same trajectory as the FP64 oracle run on it alone (its first pool step is its
prologue, so `pool.run(1 + k)` matches `oracle.run(k)`), and its results must not depend
on the other problems in the pool, on graph replay, or on the autotuner's choice:
identical bits alone and in any mix.

Tolerances as for the standalone contexts: BF16X3 trajectories 3e-4, TF32 3e-2 (the
force operands carry 16 and 10 mantissa bits), CSR (FP32 SpMM) 1e-5.
"""
import numpy as np
import pytest

import fth_synth as syn
from oracle.fth import OracleFTH

from gpu_util import gpu_ready

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not gpu_ready(), reason="needs a CUDA GPU and libfth.so")]

WS = 1 << 28


def _pool(**kw):
    from paper_1402_2095_gb300 import Pool
    return Pool(kw.pop("workspace", WS), **kw)


def _dense(n, seed):
    M, _, _ = syn.dense_spd(n, 1.0, 100.0, seed=seed)
    return M


def _gle(s, seed):
    return syn.random_gle(s, seed=seed, rate=3.0)


def _compare(pool, h, o, steps, chunks):
    """Run both sides in chunks; max state deviation relative to the largest state."""
    diff = ref = 0.0
    first = True
    for _ in range(chunks):
        pool.run(steps // chunks + (1 if first else 0))
        first = False
        o.run(steps // chunks)
        for name, r in (("q", o.q), ("p", o.p), ("s", o.s)):
            if r.size:
                diff = max(diff, float(np.max(np.abs(pool.get_state(h, name) - r))))
                ref = max(ref, float(np.max(np.abs(r))))
    return diff / ref


@pytest.mark.parametrize("precision,R,n,tol", [("bf16x3", 32, 300, 3e-4), ("tf32", 64, 200, 3e-2),
                                               ("bf16x3", 128, 129, 3e-4)])
def test_pool_dense_trajectory(precision, R, n, tol):
    M = _dense(n, seed=21)
    a, c = _gle(4, 22)
    pool = _pool(replicas=R, precision=precision)
    h = pool.add(M, a_p=a, c_p=c, dt=0.01, seed=55)
    o = OracleFTH(M=M, a_p=a, c_p=c, dt=0.01, replicas=R, seed=55)
    assert _compare(pool, h, o, 400, 2) <= tol
    assert pool.info(h)["steps"] == 400


def test_pool_csr_trajectory():
    L = 6
    rowptr, col, val = syn.lattice_csr(L, seed=9)
    v32 = val.astype(np.float32)
    a, c = _gle(3, 23)
    dt = 0.1 / np.sqrt(14.5)
    pool = _pool(replicas=32)
    h = pool.add(csr=(rowptr, col, v32, L ** 3), a_p=a, c_p=c, dt=dt, seed=7)
    o = OracleFTH(csr=(rowptr, col, v32.astype(np.float64), L ** 3), a_p=a, c_p=c, dt=dt,
                  replicas=32, seed=7)
    assert _compare(pool, h, o, 600, 3) <= 1e-5


def test_pool_replica_offset_and_observable():
    M = _dense(96, seed=24)
    a, c = _gle(2, 25)
    pool = _pool(replicas=32)
    h = pool.add(M, a_p=a, c_p=c, dt=0.01, seed=3, replica_offset=64, observable="q")
    o = OracleFTH(M=M, a_p=a, c_p=c, dt=0.01, replicas=32, seed=3, replica_offset=64)
    assert _compare(pool, h, o, 200, 1) <= 3e-4


def _mix_problems():
    """Dense problems of ragged order (1, 64, 129, 300, 700), a CSR lattice, several
    GLE sizes; (kwargs, is_csr)."""
    out = []
    for k, (n, s) in enumerate([(300, 4), (1, 0), (700, 2), (129, 4), (64, 1)]):
        a, c = _gle(s, 30 + k)
        out.append(dict(M=_dense(n, seed=40 + k), a_p=a, c_p=c, dt=0.01, seed=100 + k,
                        pairs=syn.random_pairs(n, 20, seed=k) if n > 1 else [(0, 0)],
                        burnin=3, block=7))
    rowptr, col, val = syn.lattice_csr(5, seed=8)
    a, c = _gle(4, 36)
    out.append(dict(csr=(rowptr, col, val.astype(np.float32), 125), a_p=a, c_p=c,
                    dt=0.1 / np.sqrt(14.5), seed=106, pairs=syn.lattice_nn_pairs(5)[:40],
                    burnin=3, block=7))
    return out


def _states(pool, h):
    return [pool.get_state(h, x) for x in ("q", "p", "s")]


def test_pool_mix_is_bit_identical_to_alone():
    probs = _mix_problems()
    mixed = _pool(replicas=32, graph_steps=8)
    hs = [mixed.add(**kw) for kw in probs]
    mixed.run(45)   # 5 graph replays + 5 direct steps
    assert mixed.stats()["graphs"] == 1
    for k, kw in enumerate(probs):
        alone = _pool(replicas=32, graph_steps=0)
        h = alone.add(**kw)
        alone.run(20)
        alone.run(25)
        for x, y in zip(_states(mixed, hs[k]), _states(alone, h)):
            assert np.array_equal(x, y), f"problem {k}"
        pairs = kw["pairs"]
        vm, em = mixed.elements(hs[k], pairs)
        va, ea = alone.elements(h, pairs)
        assert np.array_equal(vm, va) and np.array_equal(em, ea, equal_nan=True)


def test_pool_statistics_match_oracle():
    """Tracked elements, burn-in, blocks and error bars against the oracle (CSR problem:
    FP32 SpMM, so the trajectories agree to 1e-5 and the statistics closely)."""
    kw = _mix_problems()[-1]
    rowptr, col, v32, n = kw["csr"]
    pool = _pool(replicas=32)
    h = pool.add(**kw)
    o = OracleFTH(csr=(rowptr, col, v32.astype(np.float64), n), a_p=kw["a_p"], c_p=kw["c_p"],
                  dt=kw["dt"], replicas=32, seed=kw["seed"], burnin=3, block=7,
                  pairs=np.asarray(kw["pairs"]))
    pool.run(1 + 73)
    o.run(73)
    info = pool.info(h)
    assert info["samples"] == o.nsamples and info["blocks"] == o.nblocks == 10
    vg, eg = pool.elements(h, kw["pairs"])
    vo, eo = o.elements()
    scale = float(np.max(np.abs(vo)))
    assert np.max(np.abs(vg - vo)) <= 1e-4 * scale
    assert np.max(np.abs(eg - eo)) <= 1e-3 * scale


def test_pool_admission_and_reuse():
    M = _dense(256, seed=50)
    a, c = _gle(4, 51)
    pool = _pool(replicas=32, workspace=32 << 20)
    need = pool.footprint(M, a_p=a, c_p=c, dt=0.01)
    slab = pool.stats()["slab_bytes"]
    from paper_1402_2095_gb300 import FthError
    hs = []
    while True:
        try:
            hs.append(pool.add(M, a_p=a, c_p=c, dt=0.01, seed=len(hs)))
        except FthError as e:
            assert e.status == 4 and "not admitted" in str(e)   # FTH_E_WORKSPACE
            break
    assert len(hs) == slab // need
    assert pool.stats()["used_bytes"] == len(hs) * need
    pool.run(5)
    # free one, admit a different problem in its place, which then starts fresh
    pool.remove(hs[1])
    M2 = _dense(200, seed=52)
    h2 = pool.add(M2, a_p=a, c_p=c, dt=0.01, seed=9)
    o = OracleFTH(M=M2, a_p=a, c_p=c, dt=0.01, replicas=32, seed=9)
    assert _compare(pool, h2, o, 100, 2) <= 3e-4
    assert pool.info(hs[0])["steps"] == 4 + 101   # prologue, then every launch a step


def test_pool_rejects_invalid_problems():
    from paper_1402_2095_gb300 import FthError
    a, c = _gle(1, 60)
    pool = _pool(replicas=32)
    bad = _dense(8, seed=61)
    bad[3, 3] = -1.0
    with pytest.raises(FthError):
        pool.add(bad, a_p=a, c_p=c, dt=0.01)
    with pytest.raises(FthError):
        pool.add(_dense(8, seed=62), a_p=a, c_p=c, dt=-0.1)
    with pytest.raises(FthError):
        pool.add(_dense(8, seed=62), a_p=a, c_p=c, dt=0.01, pairs=[(0, 8)])
    assert pool.stats()["live"] == 0 and pool.stats()["used_bytes"] == 0


def test_pool_graph_recaptured_after_membership_change():
    """A problem added after a graph was captured joins the next graph; every problem
    still matches its oracle (the graph reads the rebuilt work lists)."""
    pool = _pool(replicas=32, graph_steps=10)
    M1 = _dense(150, seed=80)
    a, c = _gle(4, 81)
    h1 = pool.add(M1, a_p=a, c_p=c, dt=0.01, seed=5)
    o1 = OracleFTH(M=M1, a_p=a, c_p=c, dt=0.01, replicas=32, seed=5)
    pool.run(1 + 40)
    o1.run(40)
    M2 = _dense(90, seed=82)
    h2 = pool.add(M2, a_p=a, c_p=c, dt=0.01, seed=6)
    o2 = OracleFTH(M=M2, a_p=a, c_p=c, dt=0.01, replicas=32, seed=6)
    pool.run(1 + 39)
    o1.run(40)
    o2.run(39)
    assert pool.stats()["graphs"] >= 2
    for h, o in ((h1, o1), (h2, o2)):
        for name, ref in (("q", o.q), ("p", o.p)):
            got = pool.get_state(h, name)
            assert np.max(np.abs(got - ref)) <= 3e-4 * np.max(np.abs(ref))
