"""Pins for the oracle's tensor algebra (Sec. 2.1) against brute-force index loops."""
import itertools

import numpy as np

from oracle import tensor


def _loops_unfold(x, n):
    dims = x.shape
    rest = [k for k in range(x.ndim) if k != n]
    out = np.zeros((dims[n], int(np.prod([dims[k] for k in rest]))))
    for idx in itertools.product(*[range(d) for d in dims]):
        col = 0
        for k in rest:                                    # C-order over remaining modes
            col = col * dims[k] + idx[k]
        out[idx[n], col] = x[idx]
    return out


def test_unfold_fold_bruteforce():
    x = np.random.default_rng(0).standard_normal((2, 3, 4, 5))
    for n in range(4):
        u = tensor.unfold(x, n)
        np.testing.assert_array_equal(u, _loops_unfold(x, n))
        np.testing.assert_array_equal(tensor.fold(u, n, x.shape), x)


def test_ttm_bruteforce():
    g = np.random.default_rng(1)
    x = g.standard_normal((3, 4, 5))
    m = g.standard_normal((6, 4))
    y = tensor.ttm(x, m, 1)
    want = np.zeros((3, 6, 5))
    for i, j, k, l in itertools.product(range(3), range(6), range(5), range(4)):
        want[i, j, k] += m[j, l] * x[i, l, k]
    np.testing.assert_allclose(y, want, rtol=1e-13, atol=1e-13)


def test_tucker_and_tr_bruteforce():
    g = np.random.default_rng(2)
    core = g.standard_normal((2, 3, 2))
    us = [g.standard_normal((4, 2)), g.standard_normal((3, 3)), g.standard_normal((5, 2))]
    t = tensor.tucker(core, us)
    want = np.zeros((4, 3, 5))
    for i, j, k in itertools.product(range(4), range(3), range(5)):
        for a, b, c in itertools.product(range(2), range(3), range(2)):
            want[i, j, k] += core[a, b, c] * us[0][i, a] * us[1][j, b] * us[2][k, c]
    np.testing.assert_allclose(t, want, rtol=1e-12, atol=1e-12)

    cores = [g.standard_normal((2, 3, 3)), g.standard_normal((3, 4, 2)), g.standard_normal((2, 2, 2))]
    x = tensor.tr(cores)
    want = np.zeros((3, 4, 2))
    for i, j, k in itertools.product(range(3), range(4), range(2)):
        want[i, j, k] = np.trace(cores[0][:, i, :] @ cores[1][:, j, :] @ cores[2][:, k, :])
    np.testing.assert_allclose(x, want, rtol=1e-12, atol=1e-12)
