"""Combining per-process estimates when the replicas of one problem are split across
processes (one GPU each).

Replicas are independent (the paper's closing discussion: trivially parallel
simulations), so each rank runs its own slice of replicas with replica_offset =
rank * R and the same seed: together the ranks draw exactly the noise of one run with
world * R replicas, and no data crosses ranks during a step.  The single exchange is
this FP64 combination at the end:
  value = sum_w c_w v_w / sum_w c_w            (c_w = accumulated samples x replicas)
  err   = sqrt(sum_w (c_w / C)^2 err_w^2)      (ranks independent)
"""
from __future__ import annotations

import numpy as np


def combine(values, errbars, count, group=None):
    """All-reduce one rank's (values, errbars, count) into the combined estimate."""
    import torch
    import torch.distributed as dist

    v = torch.as_tensor(np.asarray(values, dtype=np.float64))
    e = torch.as_tensor(np.asarray(errbars, dtype=np.float64))
    c = float(count)
    dev = "cuda" if dist.get_backend(group) == "nccl" else "cpu"
    buf = torch.cat([v * c, (e * c) ** 2, torch.tensor([c], dtype=torch.float64)]).to(dev)
    dist.all_reduce(buf, op=dist.ReduceOp.SUM, group=group)
    buf = buf.cpu().numpy()
    k = len(v)
    C = buf[-1]
    return buf[:k] / C, np.sqrt(buf[k:2 * k]) / C
