"""Pins for the oracle's matrix functions (special cases, library cross-checks,
Chebyshev route against the eigendecomposition)."""
import numpy as np
import scipy.linalg as sla

import fth_synth as syn
from oracle import gle, matfun


def test_scalar_and_diagonal_matrices():
    f = lambda x: matfun.f_scalar("inv_sqrt", x)
    assert np.allclose(matfun.f_of_matrix(4.0 * np.eye(5), f), 0.5 * np.eye(5))
    d = np.array([1.0, 4.0, 9.0, 16.0])
    assert np.allclose(matfun.f_of_matrix(np.diag(d), f), np.diag(1 / np.sqrt(d)))


def test_inverse_square_root_identities():
    M, _, _ = syn.dense_spd(40, 1.0, 100.0, seed=3)
    X = matfun.f_of_matrix(M, lambda x: matfun.f_scalar("inv_sqrt", x))
    assert np.allclose(X @ X @ M, np.eye(40), atol=1e-10)
    Y = sla.fractional_matrix_power(M, -0.5)
    assert np.allclose(X, np.real(Y), atol=1e-10)


def test_fermi_complement_and_exp():
    M, _, _ = syn.dense_spd(30, 1.0, 50.0, seed=4)
    fa = matfun.f_of_matrix(M, lambda x: matfun.f_scalar("fermi", x, (2.0, 10.0)))
    fb = matfun.f_of_matrix(M, lambda x: 1.0 / (1.0 + np.exp(-2.0 * (x - 10.0))))
    assert np.allclose(fa + fb, np.eye(30), atol=1e-12)
    e = matfun.f_of_matrix(M, lambda x: matfun.f_scalar("exp", x, (0.1,)))
    assert np.allclose(e, sla.expm(-0.1 * M), atol=1e-12)


def test_chebyshev_route_matches_eigendecomposition():
    L = 6
    rowptr, col, val = syn.lattice_csr(L, seed=5)
    n = L ** 3
    a, c = syn.random_gle(4, seed=6, rate=2.0)
    dt = 0.1 / np.sqrt(14.5)
    T, S = gle.propagator(a, c, dt)
    pairs = np.concatenate([syn.diag_pairs(n)[:20], syn.lattice_nn_pairs(L)[:40]])
    vals, tail = matfun.g_elements_sparse(rowptr, col, val, n, T, S, dt, pairs, degree=200)
    Md = syn.csr_to_dense(rowptr, col, val, n)
    ref = matfun.g_of_matrix(Md, T, S, dt)
    want = np.array([ref[i, j] for i, j in pairs])
    assert tail < 1e-10
    assert np.allclose(vals, want, atol=1e-10)


def test_multi_function_chebyshev_route_matches_eigendecomposition():
    """Several functions through one shared recurrence: the stationary response g, the
    exact expected running mean after 50 samples and a Fermi function, each against the
    eigendecomposition."""
    L = 6
    rowptr, col, val = syn.lattice_csr(L, seed=7)
    n = L ** 3
    a, c = syn.random_gle(4, seed=8, rate=2.0)
    dt = 0.1 / np.sqrt(14.5)
    T, S = gle.propagator(a, c, dt)
    fns = [lambda x: gle.mode_response(x, T, S, dt),
           lambda x: gle.mode_response_mean(x, T, S, dt, 0, 50),
           lambda x: matfun.f_scalar("fermi", x, (2.0, 7.0))]
    pairs = np.concatenate([syn.diag_pairs(n)[:10], syn.lattice_nn_pairs(L)[:10]])
    vals, tails = matfun.fn_elements_sparse(rowptr, col, val, n, fns, pairs, degree=300)
    Md = syn.csr_to_dense(rowptr, col, val, n)
    lam, U = np.linalg.eigh(Md)
    for k, fn in enumerate(fns):
        ref = (U * fn(lam)[None, :]) @ U.T
        assert tails[k] < 1e-10
        assert np.allclose(vals[k], [ref[i, j] for i, j in pairs], atol=1e-10)


def test_lattice_spectrum_inside_gershgorin_interval():
    rowptr, col, val = syn.lattice_csr(5, seed=7)
    lo, hi = matfun.gershgorin(rowptr, col, val, 125)
    w = np.linalg.eigvalsh(syn.csr_to_dense(rowptr, col, val, 125))
    assert lo >= 0.5 - 1e-12 and hi <= 14.5 + 1e-12
    assert w.min() >= lo - 1e-12 and w.max() <= hi + 1e-12
