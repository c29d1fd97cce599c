"""Pins for TR-SVD (oracle.tr.tr_svd, the alternative step 3 of Algorithm 3):
with closing rank r_{N-1} = 1 (a tensor train) it recovers a TT tensor of matching ranks
exactly (the sequential SVDs only rotate within each bond; with r_{N-1} > 1 the first
split of the rank product is arbitrary, so a ring is not recovered in general); |G - TR|^2
equals the sum of the steps' truncation errors (nested orthogonal projections); N = 2 with
closing rank 1 is the Eckart-Young truncated SVD."""
import numpy as np
import pytest

import synth
from oracle import tr as otr
from oracle.tensor import tr as tr_full


def _ring(dims, ranks, seed):
    g = np.random.default_rng(seed)
    n = len(dims)
    return [g.standard_normal((ranks[k - 1], dims[k], ranks[k])) for k in range(n)]


@pytest.mark.parametrize("dims,ranks", [((12, 10, 9), (3, 2, 1)), ((10, 10, 10, 10), (3, 3, 3, 1)),
                                        ((16, 5, 6, 7, 8), (2, 3, 2, 2, 1))])
def test_exact_recovery_tensor_train(dims, ranks):
    g = tr_full(_ring(dims, ranks, sum(dims)))
    cores, errs = otr.tr_svd(g, ranks)
    for k, c in enumerate(cores):
        assert c.shape == (ranks[k - 1], dims[k], ranks[k])
    assert np.linalg.norm(tr_full(cores) - g) <= 1e-10 * np.linalg.norm(g)
    assert sum(errs) <= 1e-20 * np.sum(g * g) + 1e-24


@pytest.mark.parametrize("ranks", [(2, 2, 2), (3, 2, 3), (1, 3, 2)])
def test_error_is_the_sum_of_step_errors(ranks):
    g = synth.rng(3).standard_normal((10, 9, 8))
    cores, errs = otr.tr_svd(g, ranks)
    err2 = float(np.sum((g - tr_full(cores)) ** 2))
    assert abs(err2 - sum(errs)) <= 1e-10 * np.sum(g * g)
    assert abs(otr.tr_fit(g, cores) - (1 - np.sqrt(sum(errs) / np.sum(g * g)))) <= 1e-12


def test_two_modes_is_truncated_svd():
    a = synth.rng(4).standard_normal((20, 15))
    cores, _ = otr.tr_svd(a, (5, 1))                 # core 0: (1, 20, 5), core 1: (5, 15, 1)
    u, s, vt = np.linalg.svd(a)
    best = (u[:, :5] * s[:5]) @ vt[:5]
    np.testing.assert_allclose(tr_full(cores), best, atol=1e-12 * np.abs(a).max())
