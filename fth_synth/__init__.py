"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the CPU oracle.

This module holds input recipes only: matrices, GLE parameter sets, index lists and
request streams.  It contains none of the f-thermostat arithmetic (no propagators,
no integrator, no covariance solves), so both the library side and the oracle side
may take their inputs from here without sharing any of the method's code.

The recipes follow the workloads of the paper (Sec. "Results and benchmarks" and the
Appendix) as stand-ins: the paper's own matrices, GLE parameters and Supporting
Information are not available, so every input is drawn from a seeded generator with
the same structure (dense SPD with a prescribed spectrum, periodic cubic lattices with
a nearest-neighbour stencil, ragged batches, Poisson request streams).
"""
from __future__ import annotations

import numpy as np

BASE_SEED = 1402


def rng(seed: int) -> np.random.Generator:
    return np.random.default_rng(int(seed))


# ----------------------------------------------------------------------------------
# Dense SPD matrices with a prescribed spectrum
# ----------------------------------------------------------------------------------
def haar_orthogonal(n: int, g: np.random.Generator) -> np.ndarray:
    """Haar-distributed orthogonal matrix: QR of a Gaussian matrix with the signs of
    R's diagonal folded into Q (Mezzadri, Notices AMS 54 (2007) 592)."""
    z = g.standard_normal((n, n))
    q, r = np.linalg.qr(z)
    d = np.sign(np.diag(r))
    d[d == 0] = 1.0
    return q * d[None, :]


def log_uniform(n: int, lo: float, hi: float, g: np.random.Generator) -> np.ndarray:
    return np.exp(g.uniform(np.log(lo), np.log(hi), size=n))


def dense_spd(n: int, lam_lo: float, lam_hi: float, seed: int):
    """M = Q diag(lam) Q^T with Q Haar and lam log-uniform in [lam_lo, lam_hi].

    Returns (M, lam, Q) in float64; M is symmetrised exactly."""
    g = rng(seed)
    lam = log_uniform(n, lam_lo, lam_hi, g)
    q = haar_orthogonal(n, g)
    m = (q * lam[None, :]) @ q.T
    m = 0.5 * (m + m.T)
    return m, lam, q


# ----------------------------------------------------------------------------------
# Sparse periodic cubic lattices (7-point stencil)
# ----------------------------------------------------------------------------------
def shell_offsets(shells: int = 6):
    """Lattice offsets (dx, dy, dz) of the first `shells` neighbour shells of a simple
    cubic lattice, by squared distance 1, 2, 3, 4, 5, 6 (6 + 12 + 8 + 6 + 24 + 24 = 80
    neighbours for six shells), in a fixed order."""
    out = []
    r = 3
    for d2 in range(1, 64):
        sh = [(x, y, z) for x in range(-r, r + 1) for y in range(-r, r + 1)
              for z in range(-r, r + 1) if x * x + y * y + z * z == d2]
        if sh:
            out.append(sh)
        if len(out) == shells:
            break
    return [o for sh in out for o in sh]


def m1_csr(n: int, seed: int, onsite: float = 100.0, hop_hi: float = 2.0, shells: int = 6):
    """The paper's M1 matrices (Appendix, logarithm example): a periodic n^3 cubic
    lattice, dof i at site (i / n^2, (i % n^2) / n, i % n); diagonal = the on-site term;
    hopping uniform in [0, hop_hi] between every pair of sites up to the `shells`-th
    neighbour shell (periodic distance), one draw per pair (the matrix is symmetric).
    n >= 7 keeps the 80 neighbours of six shells distinct under periodicity.

    Returns (rowptr int32[N+1], col int32[nnz], val float64[nnz]), columns sorted."""
    if n < 2 * 3 + 1:
        raise ValueError("n >= 7 keeps the periodic neighbour shells distinct")
    g = rng(seed)
    N = n ** 3
    idx = np.arange(N, dtype=np.int64)
    x, y, z = idx // (n * n), (idx % (n * n)) // n, idx % n
    offs = shell_offsets(shells)
    half = [o for o in offs if o > (0, 0, 0)]          # one of each +/- pair
    rows, cols, vals = [idx], [idx], [np.full(N, float(onsite))]
    for (dx, dy, dz) in half:
        j = ((x + dx) % n) * n * n + ((y + dy) % n) * n + (z + dz) % n
        h = g.uniform(0.0, hop_hi, size=N)
        rows += [idx, j]
        cols += [j, idx]
        vals += [h, h]
    r = np.concatenate(rows)
    c = np.concatenate(cols)
    v = np.concatenate(vals)
    order = np.lexsort((c, r))
    r, c, v = r[order], c[order], v[order]
    rowptr = np.zeros(N + 1, dtype=np.int64)
    np.add.at(rowptr, r + 1, 1)
    return np.cumsum(rowptr).astype(np.int32), c.astype(np.int32), v


def m2_dense(m: int, seed: int, a: float = -300.0, b: float = 300.0) -> np.ndarray:
    """The paper's M2 matrices (Appendix, exponential example): diagonal D(i) uniform in
    [a + (b-a)/4, b - (b-a)/4]; then, row by row (i ascending, j = 0 .. i-1), the element
    (i, j) = (j, i) is uniform in [-r/(i-j), r/(i-j)] with
    r = min[D(i)-R(i)-a, b-D(i)-R(i), D(j)-R(j)-a, b-D(j)-R(j)], and both Gerschgorin
    radii R(i), R(j) grow by its absolute value: every eigenvalue lies in (a, b)."""
    g = rng(seed)
    D = g.uniform(a + (b - a) / 4.0, b - (b - a) / 4.0, size=m)
    R = np.zeros(m)
    M = np.diag(D)
    for i in range(1, m):
        u = g.uniform(-1.0, 1.0, size=i)
        for j in range(i):
            r = min(D[i] - R[i] - a, b - D[i] - R[i], D[j] - R[j] - a, b - D[j] - R[j])
            xv = u[j] * r / (i - j)
            M[i, j] = M[j, i] = xv
            R[i] += abs(xv)
            R[j] += abs(xv)
    return M


def lattice_site(i: int, L: int):
    """Site coordinates of dof i on an L^3 lattice, in the index order of the
    paper's Appendix (x = i / L^2, y = (i % L^2) / L, z = i % L)."""
    return i // (L * L), (i % (L * L)) // L, i % L


def lattice_csr(L: int, seed: int, diag_lo: float = 6.0, diag_hi: float = 8.0,
                shift: float = 0.5, hop: float = -1.0):
    """Periodic L^3 cubic lattice, on-site term uniform in [diag_lo, diag_hi] plus
    `shift`, hopping `hop` to the 6 nearest neighbours.  Gershgorin puts the spectrum
    inside [diag_lo + shift - 6|hop|, diag_hi + shift + 6|hop|].

    Returns (rowptr int32[N+1], col int32[nnz], val float64[nnz]) with the columns of
    each row sorted; the matrix is symmetric and stored in full."""
    n = L ** 3
    g = rng(seed)
    diag = g.uniform(diag_lo, diag_hi, size=n) + shift
    idx = np.arange(n, dtype=np.int64)
    x, y, z = idx // (L * L), (idx % (L * L)) // L, idx % L

    def site(a, b, c):
        return (a % L) * L * L + (b % L) * L + (c % L)

    nbrs = [site(x + 1, y, z), site(x - 1, y, z), site(x, y + 1, z),
            site(x, y - 1, z), site(x, y, z + 1), site(x, y, z - 1)]
    cols = np.stack([idx] + nbrs, axis=1)              # [n, 7]
    vals = np.concatenate([diag[:, None], np.full((n, 6), float(hop))], axis=1)
    if L <= 2:
        # neighbours coincide on tiny lattices: merge duplicates
        rows = np.repeat(idx, 7)
        import scipy.sparse as sp
        a = sp.csr_matrix((vals.ravel(), (rows, cols.ravel())), shape=(n, n))
        a.sum_duplicates()
        a.sort_indices()
        return (a.indptr.astype(np.int32), a.indices.astype(np.int32), a.data.astype(np.float64))
    order = np.argsort(cols, axis=1, kind="stable")
    cols = np.take_along_axis(cols, order, axis=1)
    vals = np.take_along_axis(vals, order, axis=1)
    rowptr = (np.arange(n + 1, dtype=np.int64) * 7).astype(np.int32)
    return rowptr, cols.ravel().astype(np.int32), vals.ravel().astype(np.float64)


def csr_to_dense(rowptr, col, val, n):
    m = np.zeros((n, n), dtype=np.float64)
    for i in range(n):
        for k in range(int(rowptr[i]), int(rowptr[i + 1])):
            m[i, int(col[k])] += float(val[k])
    return m


# ----------------------------------------------------------------------------------
# GLE parameter sets
# ----------------------------------------------------------------------------------
def random_gle(s: int, seed: int, rate: float = 1.0, temp: float = 1.0):
    """A valid random GLE (drift A_p, free-particle covariance C_p), size (s+1).

    C_p is a random SPD matrix and A_p = (D + W) C_p^{-1} with D SPD and W skew, so
    that A_p C_p + C_p A_p^T = 2 D is positive definite (a valid B_p B_p^T of Eq. 4)
    and every eigenvalue of A_p has a positive real part.  `rate` scales A_p (the
    inverse memory time) and `temp` scales C_p."""
    ns = s + 1
    g = rng(seed)
    x = g.standard_normal((ns, ns))
    c = x @ x.T / ns + 0.5 * np.eye(ns)
    y = g.standard_normal((ns, ns))
    d = y @ y.T / ns + 0.25 * np.eye(ns)
    w = g.standard_normal((ns, ns))
    w = 0.5 * (w - w.T)
    a = (d + w) @ np.linalg.inv(c)
    return rate * a, temp * c


def white_noise_gle(gamma: float, temp: float = 1.0):
    """s = 0: plain Langevin friction gamma at temperature temp (A_p = [gamma], C_p = [temp])."""
    return np.array([[float(gamma)]]), np.array([[float(temp)]])


# ----------------------------------------------------------------------------------
# Tracked-element lists
# ----------------------------------------------------------------------------------
def diag_pairs(n: int) -> np.ndarray:
    i = np.arange(n, dtype=np.int64)
    return np.stack([i, i], axis=1)


def upper_pairs(n: int) -> np.ndarray:
    i, j = np.triu_indices(n)
    return np.stack([i.astype(np.int64), j.astype(np.int64)], axis=1)


def lattice_nn_pairs(L: int) -> np.ndarray:
    """(i, +x neighbour), (i, +y neighbour), (i, +z neighbour) for every site."""
    n = L ** 3
    idx = np.arange(n, dtype=np.int64)
    x, y, z = idx // (L * L), (idx % (L * L)) // L, idx % L
    out = []
    for dx, dy, dz in ((1, 0, 0), (0, 1, 0), (0, 0, 1)):
        j = ((x + dx) % L) * L * L + ((y + dy) % L) * L + (z + dz) % L
        out.append(np.stack([idx, j], axis=1))
    return np.concatenate(out, axis=0)


def random_pairs(n: int, k: int, seed: int, offdiag: bool = True) -> np.ndarray:
    g = rng(seed)
    i = g.integers(0, n, size=k)
    j = g.integers(0, n, size=k)
    if offdiag and n > 1:
        same = i == j
        j[same] = (j[same] + 1 + g.integers(0, n - 1, size=int(same.sum()))) % n
    return np.stack([i, j], axis=1).astype(np.int64)


# ----------------------------------------------------------------------------------
# Ragged batches and request streams
# ----------------------------------------------------------------------------------
def ragged_sizes(count: int, seed: int, unit: int = 64, umax: int = 16) -> np.ndarray:
    """Sizes N_k = unit * u, u uniform on {1..umax}."""
    g = rng(seed)
    return unit * g.integers(1, umax + 1, size=count)


def poisson_arrivals(rate: float, duration: float, seed: int) -> np.ndarray:
    """Arrival times of a Poisson process of `rate` per second over [0, duration)."""
    g = rng(seed)
    t, out = 0.0, []
    while True:
        t += g.exponential(1.0 / rate)
        if t >= duration:
            return np.asarray(out)
        out.append(t)


def gaussian_state(shape, seed: int, scale: float = 1.0) -> np.ndarray:
    return scale * rng(seed).standard_normal(shape)
