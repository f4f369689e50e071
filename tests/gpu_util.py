"""Shared helpers of the GPU parity tests: build both sides from the same seeded
inputs (fth_synth) and compare.  The CUDA side is always driven through the C ABI
(paper_1402_2095_gb300.binding); the oracle side through oracle/."""
import numpy as np

import fth_synth as syn
from oracle.fth import OracleFTH


def gpu_ready():
    try:
        import torch
        if not torch.cuda.is_available():
            return False
        from paper_1402_2095_gb300 import build
        build.build()
        return True
    except Exception:
        return False


def make_pair(M=None, csr=None, *, a_p, c_p, dt, R, seed, precision="fp32", track="list",
              pairs=None, burnin=0, block=10, observable="p", stack=0, M_oracle=None):
    """(gpu, oracle) driven by identical inputs.  M is given to both in float32-rounded
    form unless the precision is fp64, so both integrate the same matrix."""
    from paper_1402_2095_gb300 import FTH
    obs = 0 if observable == "p" else 1
    if M is not None:
        Mg = M if precision == "fp64" else M.astype(np.float32)
        g = FTH(M=Mg, a_p=a_p, c_p=c_p, dt=dt, replicas=R, seed=seed, precision=precision,
                track=track, pairs=pairs, burnin=burnin, block=block, observable=observable,
                stack=stack)
        Mo = Mg.astype(np.float64) if M_oracle is None else M_oracle
        o = OracleFTH(M=Mo, a_p=a_p, c_p=c_p, dt=dt, replicas=R, seed=seed, burnin=burnin,
                      block=block, observable=obs, pairs=_oracle_pairs(pairs, track, Mo.shape[0]))
    else:
        rowptr, col, val, n = csr
        v32 = val.astype(np.float32)
        g = FTH(csr=(rowptr, col, v32, n), a_p=a_p, c_p=c_p, dt=dt, replicas=R, seed=seed,
                precision=precision, track=track, pairs=pairs, burnin=burnin, block=block,
                observable=observable, stack=stack)
        o = OracleFTH(csr=(rowptr, col, v32.astype(np.float64), n), a_p=a_p, c_p=c_p, dt=dt,
                      replicas=R, seed=seed, burnin=burnin, block=block, observable=obs,
                      pairs=_oracle_pairs(pairs, track, n))
    return g, o


def _oracle_pairs(pairs, track, n):
    if track == "list":
        return pairs
    if track == "diag":
        return syn.diag_pairs(n)
    return syn.upper_pairs(n)


def state_rel_err(g, o):
    """max over q, p, s of ||x_gpu - x_cpu||_inf / ||x_cpu||_inf."""
    errs = []
    for name, ref in (("q", o.q), ("p", o.p), ("s", o.s)):
        if ref.size == 0:
            continue
        got = g.get_state(name)
        errs.append(np.max(np.abs(got - ref)) / max(np.max(np.abs(ref)), 1e-300))
    return max(errs)


def trace_terms(n=None, O=None):
    """The tests' own (pairs, weights) of Tr f(M) = sum_i <p_i p_i> (O None; n = order)
    or Tr O f(M) = sum_ij O_ij <p_i p_j> for a symmetric O (dense array or scipy sparse):
    O_ii on (i, i) and 2 O_ij on (i, j), i < j -- to check the library's own weights."""
    import scipy.sparse as sp
    if O is None:
        idx = np.arange(int(n), dtype=np.int64)
        return np.stack([idx, idx], axis=1), np.ones(int(n))
    A = O.toarray() if sp.issparse(O) else np.asarray(O, dtype=np.float64)
    i, j = np.triu_indices(A.shape[0])
    v = A[i, j]
    w = np.where(i == j, v, 2.0 * v)
    keep = w != 0
    return np.stack([i[keep], j[keep]], axis=1).astype(np.int64), w[keep]


def bf16_rn(x):
    """x rounded to FP32, then to BF16 with round to nearest, ties to even (returned in
    float64): the staging of the samples that the tensor-core accumulation pass reads."""
    u = np.ascontiguousarray(np.asarray(x, dtype=np.float32)).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)
