"""GPU tests of the serving loop (continuous batching over a problem pool).

Requests arrive while others run, are admitted when they fit, and are retired when
their error bar meets their target.  Each retired result must be bit-identical to the
same problem run alone in a pool for the same number of steps (its noise key is its own
seed and the pool's arithmetic per problem does not depend on the mix), and equal to the
FP64 oracle: on the same noise within the precision of the pool's force (BF16x3 dense,
FP32 CSR), and within a few block error bars of the exact expected running mean
(paper Eq. 6 for the fitted GLE's discrete response, from the zero state).
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


def test_served_results_match_the_oracle():
    """A dense and a lattice request served together, retired on their step budget:
    each served element against the oracle run on the same noise (same seed, same
    number of samples) and against the exact expected running mean after the request's
    own number of samples (z-scores of the block error bars)."""
    from oracle import gle, matfun
    from oracle.fth import OracleFTH
    from paper_1402_2095_gb300 import Server
    reqs = _requests()
    chosen = [reqs[1], reqs[4]]                # dense n = 200 (BF16x3), lattice 5^3 (CSR)
    srv = Server(1 << 27, replicas=32, max_problems=4, chunk_steps=100, min_blocks=2)
    ids = [srv.submit(**kw, target=1e-9, max_steps=2000) for kw in chosen]
    for _ in range(30):
        c = srv.step()
        if c["running"] == 0 and c["queued"] == 0:
            break
    for rid, kw, tol in zip(ids, chosen, (2e-3, 1e-4)):
        info, v, e = srv.result(rid)
        assert info["state"] == "budget" and info["steps"] == 2000
        nsamples = info["steps"] - 1           # the first pool step is the prologue
        if "M" in kw:
            Mo = np.asarray(kw["M"], dtype=np.float32).astype(np.float64)
            o = OracleFTH(M=Mo, a_p=kw["a_p"], c_p=kw["c_p"], dt=kw["dt"], replicas=32,
                          seed=kw["seed"], block=kw["block"], pairs=kw["pairs"])
        else:
            rowptr, col, val, n = kw["csr"]
            o = OracleFTH(csr=(rowptr, col, np.asarray(val, np.float32).astype(np.float64), n),
                          a_p=kw["a_p"], c_p=kw["c_p"], dt=kw["dt"], replicas=32,
                          seed=kw["seed"], block=kw["block"], pairs=kw["pairs"])
            Mo = syn.csr_to_dense(rowptr, col, np.asarray(val, np.float32).astype(np.float64), n)
        o.run(nsamples)
        vo, eo = o.elements()
        # same noise: the pool's force precision
        assert np.max(np.abs(v - vo)) <= tol * np.max(np.abs(vo)), (rid, np.max(np.abs(v - vo)))
        # exact expected running mean of the fitted GLE after nsamples samples
        T, S = gle.propagator(kw["a_p"], kw["c_p"], kw["dt"])
        pr = np.asarray(kw["pairs"])
        want = matfun.g_mean_of_matrix(Mo, T, S, kw["dt"], 0, nsamples)[pr[:, 0], pr[:, 1]]
        z = (v - want) / e
        assert np.all(np.abs(z) < 4.5), (rid, z)
        assert 0.3 < np.mean(z ** 2) < 3.0, (rid, np.mean(z ** 2))
    srv.close()
