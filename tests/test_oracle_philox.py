"""Pins for the oracle's sketching-matrix generator (Algorithm 1 step 1, reading c6)."""
import os

import numpy as np

from oracle import philox

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")


def _kat():
    for line in open(GOLDEN):
        if line.startswith("#") or not line.strip():
            continue
        w = [int(t, 16) for t in line.split()]
        yield w[0:4], w[4:6], w[6:10]


def test_philox_known_answers():
    n = 0
    for ctr, key, want in _kat():
        got = [int(v) for v in philox.philox4x32_10(ctr, key)]
        assert got == want
        n += 1
    assert n == 3


def test_philox_vectorised_matches_scalar():
    ctrs = [(i, 7, 123456789 + i, 3) for i in range(5)]
    vec = philox.philox4x32_10([np.array([c[j] for c in ctrs]) for j in range(4)], (11, 22))
    for i, c in enumerate(ctrs):
        one = philox.philox4x32_10(c, (11, 22))
        assert [int(v[i]) for v in vec] == [int(v) for v in one]


def test_omega_gaussian_moments():
    z = philox.omega(1234, 0, np.arange(100_000, dtype=np.uint64), 4).ravel()
    assert np.all(np.isfinite(z))
    assert abs(z.mean()) < 0.01
    assert abs(z.var() - 1.0) < 0.01
    assert abs(np.mean(z ** 4) - 3.0) < 0.06            # N(0,1) kurtosis
    assert abs(np.mean(np.abs(z) < 1.0) - 0.6827) < 0.005


def test_omega_prefix_nesting_and_mode_independence():
    cols = np.arange(5000, dtype=np.uint64)
    a = philox.omega(99, 1, cols, 7)
    b = philox.omega(99, 1, cols, 4)
    assert np.array_equal(a[:, :4], b)                    # keyed by s: nested in p
    c = philox.omega(99, 2, cols, 4)
    assert abs(np.corrcoef(b[:, 0], c[:, 0])[0, 1]) < 0.05
    d = philox.omega(100, 1, cols, 4)
    assert abs(np.corrcoef(b[:, 0], d[:, 0])[0, 1]) < 0.05


def test_omega_box_muller_pairs_share_radius():
    cols = np.arange(10, dtype=np.uint64)
    z = philox.omega(5, 0, cols, 2)
    # both members of a Box-Muller pair come from one Philox call: rho^2 = z0^2 + z1^2 = -2 ln u1
    r0, r1, _, _ = philox.philox4x32_10((np.zeros(10, np.uint64), np.zeros(10, np.uint64),
                                         cols, np.zeros(10, np.uint64)), (5, 0))
    u1 = ((r0 >> np.uint64(5)).astype(float) * 2.0 ** 26 + (r1 >> np.uint64(6)).astype(float) + 1) * 2.0 ** -53
    np.testing.assert_allclose(z[:, 0] ** 2 + z[:, 1] ** 2, -2 * np.log(u1), rtol=1e-13)
