"""OracleFTH: the FP64 f-thermostat run, step by step (oracle; test infrastructure only).

Mirrors what the library computes, in the paper's order (Eq. 2 integrated by the
cited modified velocity Verlet scheme, Eq. 5 force, Eq. 6 estimator):
  run(k): if the state is at a step boundary, apply the start half of the current
  step (prologue, kick index t); then k fused launches, each computing the force
  at the current positions, finishing the current step (B, O, sample) and starting
  the next one (O, B, A).
  elements(): value = running mean of x_i x_j over every accumulated sample and
  replica; error bar = sqrt(M2 / (nb (nb - 1))) over the nb completed blocks
  (NaN when nb < 2), blocks of `block` samples each averaged over the replicas.
"""
from __future__ import annotations

import numpy as np

from . import gle, native


class OracleFTH:
    def __init__(self, M=None, csr=None, a_p=None, c_p=None, dt=0.01, replicas=1, seed=0,
                 burnin=0, block=1, observable=0, pairs=None, T=None, S=None,
                 replica_offset=0):
        if (M is None) == (csr is None):
            raise ValueError("give exactly one of M (dense) or csr=(rowptr, col, val, n)")
        if M is not None:
            self.kind = 0
            self.Md = np.ascontiguousarray(M, dtype=np.float64)
            self.n = self.Md.shape[0]
            self.rowptr = self.col = self.val = None
        else:
            rowptr, col, val, n = csr
            self.kind = 1
            self.Md = None
            self.n = int(n)
            self.rowptr = np.ascontiguousarray(rowptr, dtype=np.int64)
            self.col = np.ascontiguousarray(col, dtype=np.int64)
            self.val = np.ascontiguousarray(val, dtype=np.float64)
        if T is None:
            T, S = gle.propagator(a_p, c_p, dt)
        self.T = np.ascontiguousarray(T, dtype=np.float64)
        self.S = np.ascontiguousarray(S, dtype=np.float64)
        self.T2 = np.ascontiguousarray(self.T @ self.T)
        self.Lj = np.ascontiguousarray(gle.joint_noise(self.T, self.S))
        self.ns = self.T.shape[0]
        self.dt = float(dt)
        self.R = int(replicas)
        self.seed = int(seed)
        self.burnin = int(burnin)
        self.block = int(block)
        self.observable = int(observable)
        self.roff = int(replica_offset)
        n, R, ns = self.n, self.R, self.ns
        self.q = np.zeros((R, n))
        self.p = np.zeros((R, n))
        self.s = np.zeros((R, max(ns - 1, 0), n))
        self.t = 0
        self.primed = False
        self.pairs = (np.zeros((0, 2), np.int64) if pairs is None
                      else np.ascontiguousarray(np.asarray(pairs, dtype=np.int64).reshape(-1, 2)))
        k = len(self.pairs)
        self.partial = np.zeros(k)
        self.bmean = np.zeros(k)
        self.bm2 = np.zeros(k)
        self._nsamp = np.zeros(1, np.int64)
        self._inblock = np.zeros(1, np.int64)
        self._nblocks = np.zeros(1, np.int64)

    def set_state(self, q, p, s):
        self.q[...] = q
        self.p[...] = p
        self.s[...] = s

    def _common(self, joint=False):
        P = native.ptr
        head = (native.I64(self.n), native.I64(self.R), native.INT(self.ns), native.INT(self.kind),
                P(self.Md), P(self.rowptr), P(self.col), P(self.val), P(self.T), P(self.S))
        extra = (P(self.T2), P(self.Lj)) if joint else ()
        return head + extra + (native.D(self.dt), native.U64(self.seed), native.U32(self.roff))

    def run(self, steps: int, keep_samples: bool = False):
        L = native.lib()
        P = native.ptr
        if not self.primed:
            rc = L.oracle_prologue(*self._common(), native.U32(self.t), P(self.q), P(self.p),
                                   P(self.s))
            if rc != 0:
                raise RuntimeError(f"oracle_prologue rc={rc}")
            self.primed = True
        samples = np.zeros((steps, self.R, self.n)) if keep_samples else None
        rc = L.oracle_steps(*self._common(joint=True), native.U32(self.t + 1), native.I64(steps),
                            P(self.q), P(self.p), P(self.s), native.INT(self.observable),
                            P(samples), native.I64(len(self.pairs)), P(self.pairs),
                            native.I64(self.burnin), native.I64(self.block),
                            P(self._nsamp), P(self.partial), P(self._inblock),
                            P(self._nblocks), P(self.bmean), P(self.bm2))
        if rc != 0:
            raise RuntimeError(f"oracle_steps rc={rc}")
        self.t += steps
        return samples

    @property
    def nblocks(self) -> int:
        return int(self._nblocks[0])

    @property
    def nsamples(self) -> int:
        return int(self._nsamp[0])

    def elements(self):
        nb = self.nblocks
        inb = int(self._inblock[0])
        count = (nb * self.block + inb) * self.R
        total = self.bmean * (nb * self.block * self.R) + self.partial
        vals = total / count if count > 0 else np.full(len(self.pairs), np.nan)
        if nb >= 2:
            errs = np.sqrt(self.bm2 / (nb * (nb - 1)))
        else:
            errs = np.full(len(self.pairs), np.nan)
        return vals, errs


def force(M, q):
    """F = -M q_r for each replica row of q (dense M), via the C core."""
    M = np.ascontiguousarray(M, dtype=np.float64)
    q = np.ascontiguousarray(q, dtype=np.float64)
    R, n = q.shape
    F = np.zeros_like(q)
    native.lib().oracle_force(native.I64(n), native.I64(R), native.INT(0), native.ptr(M), None,
                              None, None, native.ptr(q), native.ptr(F))
    return F


def fused_step_elements(M, q, p, s, T, S, dt, seed, kappa, elems, observable=0):
    """One fused launch (kick index kappa) for a few sampled (i, r), computed one by
    one: force (M q_r)_i from the full current positions, then B(dt/2), O(dt/2),
    sample, O(dt/2), B(dt/2), A(dt) on that (i, r) alone (the two O half-steps drawn
    jointly, gle.joint_noise).

    M: [N][N] float64 array or scipy.sparse CSR matrix, q/p: [R][N], s: [R][ns-1][N];
    elems: iterable of (i, r).
    Returns arrays (q_new, p_new, s_new[ns-1], sample) per element."""
    ns = T.shape[0]
    Lj = gle.joint_noise(T, S)
    out_q, out_p, out_s, out_x = [], [], [], []
    for i, r in elems:
        i, r = int(i), int(r)
        if hasattr(M, "getrow"):          # scipy.sparse matrix
            mq = float((M.getrow(i) @ q[r])[0])
        else:
            mq = float(np.dot(M[i], q[r]))
        zeta = native.replica_normals(seed, kappa, i, r, ns + 1, ns + 1)
        v = np.concatenate([[p[r, i]], s[r, :, i]])
        qi = float(q[r, i])
        v[0] -= 0.5 * dt * mq
        xy = Lj @ zeta                     # joint noise of the two O half-steps
        x = qi if observable else float(T[0] @ v + xy[0])
        v = T @ (T @ v) + xy[1:]
        v[0] -= 0.5 * dt * mq
        qi += dt * v[0]
        out_q.append(qi)
        out_p.append(v[0])
        out_s.append(v[1:].copy())
        out_x.append(x)
    return np.array(out_q), np.array(out_p), np.array(out_s), np.array(out_x)
