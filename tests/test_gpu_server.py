"""GPU tests of the serving loop (continuous batching over a problem pool).

Requests arrive while others run, are admitted when they fit, and are retired when
their error bar meets their target.  Each retired result must be bit-identical to the
same problem run alone in a pool for the same number of steps (its noise key is its own
seed and the pool's arithmetic per problem does not depend on the mix).
"""
import numpy as np
import pytest

import fth_synth as syn

from gpu_util import gpu_ready

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not gpu_ready(), reason="needs a CUDA GPU and libfth.so")]


def _gle(s, seed):
    return syn.random_gle(s, seed=seed, rate=3.0)


def _requests():
    out = []
    for k, n in enumerate([96, 200, 64, 150]):
        M, _, _ = syn.dense_spd(n, 1.0, 100.0, seed=70 + k)
        a, c = _gle(4, 80 + k)
        pairs = np.concatenate([syn.diag_pairs(n)[:16], syn.random_pairs(n, 16, seed=90 + k)])
        out.append(dict(M=M, a_p=a, c_p=c, dt=0.01, seed=500 + k, block=50, pairs=pairs))
    rowptr, col, val = syn.lattice_csr(5, seed=11)
    a, c = _gle(3, 85)
    pairs = np.concatenate([syn.diag_pairs(125)[:16], syn.lattice_nn_pairs(5)[:16]])
    out.append(dict(csr=(rowptr, col, val.astype(np.float32), 125), a_p=a, c_p=c,
                    dt=0.1 / np.sqrt(14.5), seed=505, block=50, pairs=pairs))
    return out


def _alone(kw, steps):
    from paper_1402_2095_gb300 import Pool
    pool = Pool(1 << 26, replicas=32)
    h = pool.add(**kw)
    pool.run(steps)
    v, e = pool.elements(h, kw["pairs"])
    pool.close()
    return v, e


def test_server_results_equal_alone_and_arrivals_overlap():
    from paper_1402_2095_gb300 import Server
    reqs = _requests()
    srv = Server(1 << 27, replicas=32, max_problems=8, chunk_steps=100, min_blocks=2)
    ids = []
    # staggered arrivals: two now, one after each of the next steps
    ids.append(srv.submit(**reqs[0], target=0.5))
    ids.append(srv.submit(**reqs[1], target=0.5, max_steps=400))
    srv.step()
    ids.append(srv.submit(**reqs[2], target=1e-9, max_steps=300))   # budget-bound
    srv.step()
    ids.append(srv.submit(**reqs[3], target=0.5))
    ids.append(srv.submit(**reqs[4], target=0.5))
    for _ in range(20):
        c = srv.step()
        if c["running"] == 0 and c["queued"] == 0:
            break
    states = []
    for rid, kw in zip(ids, reqs):
        info, v, e = srv.result(rid)
        states.append(info["state"])
        assert info["state"] in ("done", "budget"), info
        assert info["steps"] % 100 == 0 and info["steps"] > 0
        assert info["t_submit"] <= info["t_admit"] <= info["t_done"]
        va, ea = _alone(kw, info["steps"])
        assert np.array_equal(v, va), rid
        assert np.array_equal(e, ea, equal_nan=True), rid
        if info["state"] == "done":
            assert info["rel_err"] <= 0.5
    assert states[2] == "budget"
    srv.close()


def _slab(ws, max_problems):
    from paper_1402_2095_gb300 import Pool
    p = Pool(ws, replicas=32, max_problems=max_problems)
    b = p.stats()["slab_bytes"]
    p.close()
    return b


def test_server_admission_by_footprint():
    """Two requests fill the workspace, the third waits until they retire."""
    from paper_1402_2095_gb300 import Pool, Server
    allr = _requests()
    reqs = [allr[3], allr[0], allr[2]]          # n = 150, 96, then 64 waits
    probe = Pool(1 << 26, replicas=32, max_problems=8)
    need = [probe.footprint(kw["M"], a_p=kw["a_p"], c_p=kw["c_p"], dt=0.01, pairs=kw["pairs"])
            for kw in reqs]
    probe.close()
    want = need[0] + need[1] + 4096             # slab that holds the first two only
    ws = (1 << 26) - _slab(1 << 26, 8) + want
    ws += want - _slab(ws, 8)                   # the header grows slightly with the workspace
    slab = _slab(ws, 8)
    assert need[0] + need[1] <= slab < need[0] + need[1] + need[2] and need[2] <= slab
    srv = Server(ws, replicas=32, max_problems=8, chunk_steps=100, min_blocks=2, max_bypass=0)
    ids = [srv.submit(**kw, target=1e-9, max_steps=200) for kw in reqs]
    c = srv.step()
    assert c["admitted"] == 2 and c["queued"] == 1
    assert srv.result(ids[2])[0]["state"] == "queued"
    srv.step()                                  # the first two spend their budget and retire
    c = srv.step()
    assert srv.result(ids[2])[0]["state"] in ("running", "budget")
    for _ in range(5):
        c = srv.step()
    info, v, _ = srv.result(ids[2])
    assert info["state"] == "budget" and np.all(np.isfinite(v))
    assert info["t_admit"] >= srv.result(ids[0])[0]["t_done"]
    srv.close()


def test_server_rejects_invalid_and_keeps_serving():
    from paper_1402_2095_gb300 import Server
    reqs = _requests()
    bad = dict(reqs[0])
    M = bad["M"].copy()
    M[5, 5] = -1.0
    bad["M"] = M
    srv = Server(1 << 26, replicas=32, max_problems=4, chunk_steps=100, min_blocks=2)
    ib = srv.submit(**bad, target=0.5)
    ig = srv.submit(**reqs[2], target=0.5, max_steps=300)
    for _ in range(5):
        srv.step()
    assert srv.result(ib)[0]["state"] == "failed"
    assert srv.result(ig)[0]["state"] in ("done", "budget")
    srv.close()


def test_server_fails_requests_that_can_never_fit():
    """A request larger than the whole workspace fails instead of blocking the queue."""
    from paper_1402_2095_gb300 import Server
    reqs = _requests()
    big = dict(reqs[1])
    M, _, _ = syn.dense_spd(2000, 1.0, 100.0, seed=99)
    big["M"] = M
    big["pairs"] = np.concatenate([syn.diag_pairs(2000)[:16], syn.random_pairs(2000, 16, seed=1)])
    srv = Server(24 << 20, replicas=32, max_problems=4, chunk_steps=100, min_blocks=2,
                 max_bypass=0)
    ib = srv.submit(**big, target=0.5)
    ig = srv.submit(**reqs[2], target=0.5, max_steps=300)
    for _ in range(6):
        srv.step()
    assert srv.result(ib)[0]["state"] == "failed"
    assert srv.result(ig)[0]["state"] in ("done", "budget")
    srv.close()
