"""Pins for the divide-and-conquer decomposition (oracle.divide, Sec. 4.1.2):
K = 1 is the one-pass decomposition; the parts tile X (brute-force reassembly, sizes differ
by at most one); the squared error of the concatenated approximation is the sum of the
parts' |X_k|^2 - |G_k|^2; a part tensor of exact multilinear rank is recovered exactly."""
import numpy as np
import pytest

import synth
from oracle import divide, metrics, rbki


@pytest.mark.parametrize("size,parts", [(10, 1), (10, 3), (250, 5), (256, 4), (7, 7)])
def test_parts_tile_the_mode(size, parts):
    b = divide.part_bounds(size, parts)
    assert b[0][0] == 0 and b[-1][1] == size
    assert all(b[k][1] == b[k + 1][0] for k in range(parts - 1))
    lens = [hi - lo for lo, hi in b]
    assert min(lens) >= 1 and max(lens) - min(lens) <= 1


def test_split_reassembles():
    g = synth.rng(2)
    x = g.standard_normal((6, 5, 13))
    for mode in range(3):
        for parts in (1, 2, 5):
            if parts > x.shape[mode]:
                continue
            np.testing.assert_array_equal(np.concatenate(divide.split(x, mode, parts), axis=mode), x)


def test_one_part_is_one_pass():
    wl = synth.config_small_fp64(mc=9, dims=(40, 36, 48), core=(5, 4, 6), p=3, q=2)
    a = divide.divide_and_conquer(wl.x, 2, 1, [wl.ranks], wl.p, wl.q, wl.seed)
    b = rbki.rbki_tucker(wl.x, wl.ranks, wl.p, wl.q, wl.seed)
    np.testing.assert_array_equal(a["parts"][0]["core"], b["core"])


def test_error_is_the_sum_over_parts():
    wl = synth.config_small_fp64(mc=10, dims=(40, 36, 60), core=(5, 4, 6), p=3, q=2)
    ranks = [[5, 4, 3]] * 3
    res = divide.divide_and_conquer(wl.x, 2, 3, ranks, wl.p, wl.q, wl.seed)
    err2 = metrics.fnorm(wl.x - divide.reconstruct(res, 2)) ** 2
    assert abs(err2 - res["err2"]) <= 1e-10 * res["x_norm2"]
    # distinct sketches per part (seed + k)
    assert not np.allclose(res["parts"][0]["factors"][0], res["parts"][1]["factors"][0])


def test_exact_recovery_per_part():
    g = synth.rng(4)
    parts = []
    for k in range(2):                       # each half of mode 2 has multilinear rank (3, 3, 2)
        c = g.standard_normal((3, 3, 2))
        fac = [synth.haar_factor(g, 30, 3), synth.haar_factor(g, 24, 3), synth.haar_factor(g, 20, 2)]
        parts.append(synth.tucker_full(c, fac))
    x = np.concatenate(parts, axis=2)
    res = divide.divide_and_conquer(x, 2, 2, [[3, 3, 2]] * 2, 2, 1, 5)
    assert metrics.fnorm(x - divide.reconstruct(res, 2)) <= 1e-12 * metrics.fnorm(x)
