"""World-size-2 gloo test of the multi-process path on CPU: two ranks each run the
oracle on their replica slice (replica_offset = rank * R, same seed) and combine.  The
combined value equals a single run over all replicas, because the noise streams are
the same; the combined error bar is the independent-ranks formula."""
import os
import socket

import numpy as np
import torch.multiprocessing as mp

import fth_synth as syn


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _problem():
    M, _, _ = syn.dense_spd(6, 1.0, 20.0, seed=3)
    a, c = syn.random_gle(4, seed=4, rate=3.0)
    return M, a, c, syn.upper_pairs(6)


def _rank(rank, world, port, R, steps, q):
    os.environ["OMP_NUM_THREADS"] = "1"   # tiny problem: no OpenMP team per rank
    os.environ["GLOO_SOCKET_IFNAME"] = "lo"   # loopback: no hostname lookup
    import torch.distributed as dist
    from oracle.fth import OracleFTH
    from paper_1402_2095_gb300.multi import combine
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    M, a, c, pairs = _problem()
    o = OracleFTH(M=M, a_p=a, c_p=c, dt=0.05, replicas=R, seed=11, block=100, pairs=pairs,
                  replica_offset=rank * R)
    o.run(steps)
    v, e = o.elements()
    cv, ce = combine(v, e, o.nsamples * R)
    if rank == 0:
        q.put((cv, ce))
    dist.destroy_process_group()


def test_two_rank_combine_equals_single_run():
    R, steps, world = 4, 3000, 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, R, steps, q)) for r in range(world)]
    saved = os.environ.get("OMP_NUM_THREADS")
    os.environ["OMP_NUM_THREADS"] = "1"      # children inherit it before any runtime starts
    try:
        for p in procs:
            p.start()
    finally:
        if saved is None:
            os.environ.pop("OMP_NUM_THREADS")
        else:
            os.environ["OMP_NUM_THREADS"] = saved
    cv, ce = q.get(timeout=300)
    for p in procs:
        p.join(timeout=300)
        assert p.exitcode == 0
    from oracle.fth import OracleFTH
    M, a, c, pairs = _problem()
    o = OracleFTH(M=M, a_p=a, c_p=c, dt=0.05, replicas=world * R, seed=11, block=100,
                  pairs=pairs)
    o.run(steps)
    v, e = o.elements()
    assert np.allclose(cv, v, rtol=1e-12, atol=1e-14)
    # error bars: same order (block means of the full run mix both slices)
    ratio = ce / e
    assert np.all((ratio > 0.5) & (ratio < 2.0)), ratio
