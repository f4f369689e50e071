"""CPU checks of the workload generators of the paper's Appendix (M1, M2) and of the
host-side scaling / inverse-transform relations."""
import numpy as np
import scipy.linalg as sla

import fth_synth as syn
from paper_1402_2095_gb300 import transforms as tr


def _dense_from_csr(rowptr, col, val, n):
    M = np.zeros((n, n))
    for i in range(n):
        M[i, col[rowptr[i]:rowptr[i + 1]]] = val[rowptr[i]:rowptr[i + 1]]
    return M


def test_m1_structure():
    n = 7
    rowptr, col, val = syn.m1_csr(n, seed=3)
    N = n ** 3
    M = _dense_from_csr(rowptr, col, val, N)
    assert np.array_equal(M, M.T)
    assert np.all(np.diff(rowptr) == 81)
    assert np.all(np.diag(M) == 100.0)
    off = M - np.diag(np.diag(M))
    assert off.min() >= 0.0 and off.max() <= 2.0
    # neighbours are exactly the first six shells under periodic distance
    i = 123
    xi, yi, zi = syn.lattice_site(i, n)
    for j in np.nonzero(off[i])[0]:
        xj, yj, zj = syn.lattice_site(int(j), n)
        d = [min(abs(p - q), n - abs(p - q)) for p, q in ((xi, xj), (yi, yj), (zi, zj))]
        assert 1 <= sum(t * t for t in d) <= 6
    shells = [sum(1 for o in syn.shell_offsets() if sum(t * t for t in o) == d2)
              for d2 in range(1, 7)]
    assert shells == [6, 12, 8, 6, 24, 24]


def test_m2_spectrum_inside_interval():
    a, b = -300.0, 300.0
    M = syn.m2_dense(300, seed=4, a=a, b=b)
    assert np.array_equal(M, M.T)
    d = np.diag(M)
    assert d.min() >= a + (b - a) / 4 and d.max() <= b - (b - a) / 4
    lam = np.linalg.eigvalsh(M)
    assert lam.min() > a and lam.max() < b
    R = np.abs(M).sum(axis=1) - np.abs(d)
    assert np.all(d - R >= a - 1e-9) and np.all(d + R <= b + 1e-9)
    assert np.count_nonzero(M) > 0.9 * M.size          # almost completely filled


def test_affine_map_and_transforms():
    r, m = tr.affine_map((1.0, 2.0), (3.0, 4.0))
    assert (r, m) == (1.0, 2.0)                          # the paper's check case: m = +2
    r, m = tr.affine_map((-300.0, 300.0), (1.0, 601.0))
    assert np.isclose(r, 1.0) and np.isclose(m, 301.0)
    g = np.random.default_rng(9)
    Q, _ = np.linalg.qr(g.standard_normal((6, 6)))
    M = (Q * np.array([70.0, 80.0, 90.0, 120.0, 150.0, 170.0])) @ Q.T
    r = np.e / 70.0
    lnM = sla.logm(M).real
    lnrM = sla.logm(r * M).real
    pairs = np.array([(i, j) for i in range(6) for j in range(i, 6)])
    got = tr.log_from_scaled(lnrM[pairs[:, 0], pairs[:, 1]], pairs, r)
    assert np.allclose(got, lnM[pairs[:, 0], pairs[:, 1]], atol=1e-10)
    assert np.isclose(tr.log_trace_from_scaled(np.trace(lnrM), 6, r), np.trace(lnM))
    A = 0.01
    E = sla.expm(-A * (M - 200.0 * np.eye(6)))
    Es = sla.expm(-A * M)
    assert np.allclose(tr.exp_from_shifted(Es, A, 200.0), E)     # M - 200 I shifted by m = 200
    ap, cp = tr.scale_gle(np.eye(2), np.eye(2), alpha=2.0, gamma=3.0)
    assert np.allclose(ap, 2 * np.eye(2)) and np.allclose(cp, 3 * np.eye(2))


def test_power_law_rescale():
    g = np.random.default_rng(10)
    Q, _ = np.linalg.qr(g.standard_normal((5, 5)))
    M = (Q * np.array([0.6, 1.5, 4.0, 9.0, 14.0])) @ Q.T
    r = 2.0
    f = lambda A: sla.fractional_matrix_power(A, -0.5).real
    assert np.allclose(tr.power_from_scaled(f(r * M), r, -0.5), f(M))


def test_time_scaled_gle_samples_the_scaled_spectrum():
    """A_p -> alpha A_p with dt -> dt / alpha leaves the discrete OU propagator unchanged and
    multiplies lambda dt^2 by 1 / alpha^2: the GLE then samples f(M / alpha^2).  Checked on
    the oracle's exact per-mode response of the discrete integrator."""
    from oracle import gle
    a_p, c_p = syn.random_gle(4, seed=31, rate=3.0)
    dt, alpha = 0.02, 2.0 ** -0.5
    a2, c2 = tr.scale_gle(a_p, c_p, alpha=alpha)
    T1, S1 = gle.propagator(a_p, c_p, dt)
    T2, S2 = gle.propagator(a2, c2, dt / alpha)
    lams = np.array([0.5, 1.3, 3.0, 7.7, 14.5])
    g2 = gle.mode_response(lams, T2, S2, dt / alpha)
    g1 = gle.mode_response(lams / alpha ** 2, T1, S1, dt)
    assert np.allclose(g2, g1, rtol=1e-10, atol=0)
