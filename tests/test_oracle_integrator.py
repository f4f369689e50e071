"""Pins for the oracle's FP64 integrator and block statistics."""
import numpy as np
import pytest

import fth_synth as syn
from oracle import gle, matfun, native
from oracle.fth import OracleFTH


def test_noise_free_verlet_conserves_shadow_energy():
    # With T = I and S = 0 the step is plain velocity Verlet, which conserves
    # p^T p / 2 + q^T (M - dt^2 M^2 / 4) q / 2 exactly at the step boundaries.
    n, R, dt = 6, 3, 0.08
    M, _, _ = syn.dense_spd(n, 1.0, 50.0, seed=1)
    o = OracleFTH(M=M, T=np.eye(5), S=np.zeros((5, 5)), dt=dt, replicas=R)
    g = np.random.default_rng(2)
    o.set_state(g.standard_normal((R, n)), g.standard_normal((R, n)), g.standard_normal((R, 4, n)))
    K = M - dt * dt / 4 * M @ M
    energies = []
    for _ in range(300):
        q_at_sample = o.q.copy()
        p_at_sample = o.run(1, keep_samples=True)[0]
        energies.append(0.5 * np.sum(p_at_sample ** 2, axis=1)
                        + 0.5 * np.einsum("ri,ij,rj->r", q_at_sample, K, q_at_sample))
    e = np.array(energies[1:])
    assert np.max(np.abs(e - e[0])) < 1e-11 * np.max(np.abs(e[0]))


def test_fused_step_matches_mode_matrices():
    # Diagonal M: every dof is a normal mode.  With S = 0 one fused launch maps the
    # mid-step state x through Y = O B (to the sample point) and Z = A B O (to the
    # next mid-step state); compare with the matrices of the per-mode chain.
    lams = np.array([0.5, 3.0, 11.0, 40.0])
    n, R, dt = len(lams), 2, 0.05
    a, c = syn.random_gle(4, seed=5, rate=2.0)
    T, _ = gle.propagator(a, c, dt)
    o = OracleFTH(M=np.diag(lams), T=T, S=np.zeros((5, 5)), dt=dt, replicas=R)
    o.primed = True
    g = np.random.default_rng(3)
    q0, p0, s0 = g.standard_normal((R, n)), g.standard_normal((R, n)), g.standard_normal((R, 4, n))
    o.set_state(q0, p0, s0)
    samp = o.run(1, keep_samples=True)[0]
    for k, lam in enumerate(lams):
        O = np.eye(6)
        O[1:, 1:] = T
        B = np.eye(6)
        B[1, 0] = -0.5 * dt * lam
        A = np.eye(6)
        A[0, 1] = dt
        for r in range(R):
            x = np.concatenate([[q0[r, k], p0[r, k]], s0[r, :, k]])
            y = O @ B @ x
            z = A @ B @ O @ y
            assert np.isclose(samp[r, k], y[1], rtol=1e-13, atol=1e-14)
            got = np.concatenate([[o.q[r, k], o.p[r, k]], o.s[r, :, k]])
            assert np.allclose(got, z, rtol=1e-13, atol=1e-14)


def _python_integrator(Mfull, T, S, dt, seed, R, steps):
    """Independent pure-Python restatement, element by element (tiny sizes only)."""
    n = Mfull.shape[0]
    ns = T.shape[0]
    q = np.zeros((R, n))
    v = np.zeros((R, n, ns))   # v[..., 0] = p, v[..., 1:] = s

    def F(qq):
        return np.array([[-sum(Mfull[i, k] * qq[r, k] for k in range(n)) for i in range(n)]
                         for r in range(R)])

    def O(vec, xi):
        return np.array([sum(T[a, b] * vec[b] for b in range(ns))
                         + sum(S[a, b] * xi[b] for b in range(a + 1)) for a in range(ns)])

    # joint law of (sample noise, two-half-step noise), written out from its definition
    C1 = S @ S.T
    sig = np.zeros((ns + 1, ns + 1))
    sig[0, 0] = C1[0, 0]
    for a in range(ns):
        sig[a + 1, 0] = sig[0, a + 1] = sum(T[a, b] * C1[b, 0] for b in range(ns))
    TCT = T @ C1 @ T.T
    for a in range(ns):
        for b in range(ns):
            sig[a + 1, b + 1] = TCT[a, b] + C1[a, b]
    Lj = gle.chol_psd(sig)

    f = F(q)
    for r in range(R):
        for i in range(n):
            # replica r takes positions (r % 2) (ns + 1) .. of the stream of pair r // 2
            xi = native.normals(seed, 0, i, r // 2, 2 * (ns + 1))[(r % 2) * (ns + 1):][:ns]
            v[r, i] = O(v[r, i], xi)
            v[r, i, 0] += 0.5 * dt * f[r, i]
            q[r, i] += dt * v[r, i, 0]
    samples = []
    for t in range(1, steps + 1):
        f = F(q)
        X = np.zeros((R, n))
        for r in range(R):
            for i in range(n):
                zeta = native.normals(seed, t, i, r // 2, 2 * (ns + 1))[(r % 2) * (ns + 1):][:ns + 1]
                xy = [sum(Lj[a, b] * zeta[b] for b in range(a + 1)) for a in range(ns + 1)]
                v[r, i, 0] += 0.5 * dt * f[r, i]
                X[r, i] = sum(T[0, b] * v[r, i, b] for b in range(ns)) + xy[0]
                tv = [sum(T[a, b] * v[r, i, b] for b in range(ns)) for a in range(ns)]
                v[r, i] = [sum(T[a, b] * tv[b] for b in range(ns)) + xy[a + 1] for a in range(ns)]
                v[r, i, 0] += 0.5 * dt * f[r, i]
                q[r, i] += dt * v[r, i, 0]
        samples.append(X)
    return q, v, np.array(samples)


@pytest.mark.parametrize("sparse", [False, True])
def test_c_integrator_equals_python_restatement(sparse):
    L = 2
    rowptr, col, val = syn.lattice_csr(L, seed=4)
    n = L ** 3
    Mfull = syn.csr_to_dense(rowptr, col, val, n)
    a, c = syn.random_gle(4, seed=6, rate=2.0)
    dt, seed, R, steps = 0.07, 99, 2, 4
    T, S = gle.propagator(a, c, dt)
    if sparse:
        o = OracleFTH(csr=(rowptr, col, val, n), T=T, S=S, dt=dt, replicas=R, seed=seed)
    else:
        o = OracleFTH(M=Mfull, T=T, S=S, dt=dt, replicas=R, seed=seed)
    samp = o.run(steps, keep_samples=True)
    q, v, ps = _python_integrator(Mfull, T, S, dt, seed, R, steps)
    assert np.allclose(o.q, q, rtol=1e-12, atol=1e-13)
    assert np.allclose(o.p, v[..., 0], rtol=1e-12, atol=1e-13)
    assert np.allclose(o.s, np.transpose(v[..., 1:], (0, 2, 1)), rtol=1e-12, atol=1e-13)
    assert np.allclose(samp, ps, rtol=1e-12, atol=1e-13)


def test_first_sample_covariance_is_one_step_noise():
    # From x = 0 the first sample has covariance Qn exactly (one sample-to-sample map).
    lams = np.array([0.7, 5.0, 30.0])
    a, c = syn.random_gle(4, seed=8, rate=3.0)
    dt, R = 0.05, 40000
    T, S = gle.propagator(a, c, dt)
    o = OracleFTH(M=np.diag(lams), T=T, S=S, dt=dt, replicas=R, seed=5)
    x = o.run(1, keep_samples=True)[0]
    for k, lam in enumerate(lams):
        _, Qn = gle.mode_chain(lam, T, S, dt)
        var = np.mean(x[:, k] ** 2)
        assert abs(var - Qn[1, 1]) < 5 * np.sqrt(2.0 / R) * Qn[1, 1]


def test_block_statistics_match_samples():
    n, R = 4, 3
    M, _, _ = syn.dense_spd(n, 1.0, 10.0, seed=9)
    a, c = syn.random_gle(4, seed=10, rate=2.0)
    pairs = syn.upper_pairs(n)
    o = OracleFTH(M=M, a_p=a, c_p=c, dt=0.05, replicas=R, seed=3, burnin=7, block=5,
                  pairs=pairs)
    samp = o.run(60, keep_samples=True)
    vals, errs = o.elements()
    used = samp[7:]
    prod = np.einsum("tri,trj->tij", used, used) / R       # per-sample replica mean
    blocks = prod[: (len(used) // 5) * 5].reshape(-1, 5, n, n).mean(axis=1)
    nb = blocks.shape[0]
    assert o.nblocks == nb
    for e, (i, j) in enumerate(pairs):
        assert np.isclose(vals[e], prod[:, i, j].mean(), rtol=1e-12)
        sd = blocks[:, i, j].std(ddof=1) / np.sqrt(nb)
        assert np.isclose(errs[e], sd, rtol=1e-10)


def test_stationary_estimate_within_block_errors():
    # Long run of a small dense problem: every element of <p p^T> lies within 4 block
    # errors of the exact expected estimate U diag(g_mean) U^T (transient included).
    n, R, steps, block = 5, 32, 6000, 300
    M, _, _ = syn.dense_spd(n, 1.0, 20.0, seed=12)
    a, c = syn.random_gle(4, seed=13, rate=3.0)
    dt = 0.1 / np.sqrt(20.0)
    pairs = syn.upper_pairs(n)
    o = OracleFTH(M=M, a_p=a, c_p=c, dt=dt, replicas=R, seed=21, burnin=0, block=block,
                  pairs=pairs)
    o.run(steps)
    vals, errs = o.elements()
    ref = matfun.g_mean_of_matrix(M, o.T, o.S, dt, 0, steps)
    z = np.array([(vals[e] - ref[i, j]) / errs[e] for e, (i, j) in enumerate(pairs)])
    assert np.all(np.abs(z) < 4.0), z
    # and not trivially: the estimate moved far from zero
    assert np.all(np.abs(np.diag(ref)) > 10 * errs[[e for e, (i, j) in enumerate(pairs) if i == j]])


def test_elementwise_step_equals_c_integrator():
    n, R = 7, 3
    M, _, _ = syn.dense_spd(n, 1.0, 30.0, seed=31)
    a, c = syn.random_gle(4, seed=32, rate=2.0)
    dt, seed = 0.05, 77
    o = OracleFTH(M=M, a_p=a, c_p=c, dt=dt, replicas=R, seed=seed)
    o.run(5)
    q0, p0, s0 = o.q.copy(), o.p.copy(), o.s.copy()
    kappa = o.t + 1
    x = o.run(1, keep_samples=True)[0]
    from oracle.fth import fused_step_elements
    elems = [(i, r) for i in range(n) for r in range(R)]
    qn, pn, sn, xn = fused_step_elements(M, q0, p0, s0, o.T, o.S, dt, seed, kappa, elems)
    for k, (i, r) in enumerate(elems):
        assert np.isclose(qn[k], o.q[r, i], rtol=1e-13, atol=1e-14)
        assert np.isclose(pn[k], o.p[r, i], rtol=1e-13, atol=1e-14)
        assert np.allclose(sn[k], o.s[r, :, i], rtol=1e-13, atol=1e-14)
        assert np.isclose(xn[k], x[r, i], rtol=1e-13, atol=1e-14)


def test_joint_half_steps_have_the_two_step_law():
    """The joint draw reproduces the law of two independent O half-steps around the
    sample: L L^T equals the covariance of (e_0^T S xi1, T S xi1 + S xi2) formed by
    brute force over a basis of (xi1, xi2), and for s = 0 it reduces to the scalar
    closed form."""
    a, c = syn.random_gle(4, seed=41, rate=2.5)
    T, S = gle.propagator(a, c, 0.07)
    ns = T.shape[0]
    Lj = gle.joint_noise(T, S)
    assert np.allclose(np.triu(Lj, 1), 0.0)
    # the map (xi1, xi2) -> (x, y) is linear: its matrix K gives the covariance K K^T
    K = np.zeros((ns + 1, 2 * ns))
    for k in range(2 * ns):
        e = np.zeros(2 * ns)
        e[k] = 1.0
        x = (S @ e[:ns])[0]
        y = T @ (S @ e[:ns]) + S @ e[ns:]
        K[:, k] = np.concatenate([[x], y])
    assert np.allclose(Lj @ Lj.T, K @ K.T, rtol=1e-12, atol=1e-14)
    # s = 0: T = t, S = sqrt(1 - t^2) (unit kT): x ~ N(0, 1 - t^2), y = t x' + ...
    t = 0.8
    L0 = gle.joint_noise(np.array([[t]]), np.array([[np.sqrt(1 - t * t)]]))
    c1 = 1 - t * t
    assert np.allclose(L0 @ L0.T, [[c1, t * c1], [t * c1, t * t * c1 + c1]])
