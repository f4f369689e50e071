"""Pins for the oracle's noise source: Philox4x32-10 and the Box-Muller normals."""
import os

import numpy as np

from oracle import native

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")


def _kat_rows():
    rows = []
    with open(GOLDEN) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            rows.append([int(x, 16) for x in line.split()])
    return rows


def test_philox_known_answers():
    rows = _kat_rows()
    assert len(rows) >= 2
    for row in rows:
        ctr, key, want = row[0:4], row[4:6], row[6:10]
        got = native.philox4x32_10(ctr, key)
        assert [int(x) for x in got] == want


def test_philox_counter_sensitivity():
    # every output word changes when any single counter bit flips (avalanche)
    base = native.philox4x32_10([1, 2, 3, 4], [5, 6])
    for w in range(4):
        for bit in (0, 17, 31):
            c = [1, 2, 3, 4]
            c[w] ^= 1 << bit
            out = native.philox4x32_10(c, [5, 6])
            assert np.all(out != base)


def _many_normals(count_per_call=10, calls=20000, seed=1234):
    out = np.empty((calls, count_per_call))
    for c in range(calls):
        out[c] = native.normals(seed, c, c % 97, c % 13, count_per_call)
    return out


def test_normals_moments():
    z = _many_normals().ravel()
    n = z.size
    # mean 0, variance 1, fourth moment 3: each within 5 standard errors
    assert abs(z.mean()) < 5 / np.sqrt(n)
    assert abs(z.var() - 1.0) < 5 * np.sqrt(2.0 / n)
    assert abs(np.mean(z ** 4) - 3.0) < 5 * np.sqrt(96.0 / n)
    # the 10 normals of one (kappa, i, r) are mutually uncorrelated
    blocks = _many_normals()
    c = np.corrcoef(blocks.T)
    off = c[~np.eye(10, dtype=bool)]
    assert np.max(np.abs(off)) < 5 / np.sqrt(blocks.shape[0])


def test_normals_follow_box_muller_of_philox_words():
    seed, kappa, i, r = 0x1234_5678_9ABC_DEF0, 7, 11, 3
    z = native.normals(seed, kappa, i, r, 8)
    key = [seed & 0xFFFFFFFF, seed >> 32]
    for k in range(2):
        x = native.philox4x32_10([kappa, i, r, k], key)
        u = ((x.astype(np.uint64) >> 9) * 2 + 1) / 2.0 ** 24
        for h in range(2):
            rho = np.sqrt(-2 * np.log(u[2 * h]))
            th = 2 * np.pi * u[2 * h + 1]
            assert np.isclose(z[4 * k + 2 * h], rho * np.cos(th), rtol=0, atol=1e-15)
            assert np.isclose(z[4 * k + 2 * h + 1], rho * np.sin(th), rtol=0, atol=1e-15)


def test_uniform_map_is_open_interval():
    # u(0) = 2^-24 and u(2^32-1) = 1 - 2^-24: never 0 (log) nor 1
    lo = ((0 >> 9) * 2 + 1) / 2.0 ** 24
    hi = (((2 ** 32 - 1) >> 9) * 2 + 1) / 2.0 ** 24
    assert lo == 2.0 ** -24 and hi == 1 - 2.0 ** -24


def test_replica_normals_take_their_half_of_the_pair_stream():
    """Replicas 2j and 2j + 1 share the stream of counter word j: the even one takes
    positions 0..W-1, the odd one W..2W-1; all four words of every call are used."""
    seed, kappa, i, W = 99, 5, 17, 6
    for j in (0, 3, 1000):
        raw = native.normals(seed, kappa, i, j, 12)
        assert np.array_equal(native.replica_normals(seed, kappa, i, 2 * j, W, W), raw[:W])
        assert np.array_equal(native.replica_normals(seed, kappa, i, 2 * j + 1, W, W), raw[W:])
        # the prologue's first W - 1 of the same slot
        assert np.array_equal(native.replica_normals(seed, kappa, i, 2 * j + 1, W, W - 1),
                              raw[W:2 * W - 1])
    # odd width: the second replica starts mid-call
    raw = native.normals(seed, kappa, i, 7, 12)
    assert np.array_equal(native.replica_normals(seed, kappa, i, 15, 5, 5), raw[5:10])


def test_replica_pair_normals_are_uncorrelated():
    n = 40000
    a = np.array([native.replica_normals(3, k, k % 31, 2 * (k % 17), 6, 6) for k in range(n)])
    b = np.array([native.replica_normals(3, k, k % 31, 2 * (k % 17) + 1, 6, 6) for k in range(n)])
    c = np.corrcoef(np.concatenate([a, b], axis=1).T)
    off = c[~np.eye(12, dtype=bool)]
    assert np.max(np.abs(off)) < 5 / np.sqrt(n)
    assert abs(np.mean(np.concatenate([a, b]) ** 2) - 1.0) < 5 * np.sqrt(2.0 / (12 * n))
