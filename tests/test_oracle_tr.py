"""Pins for the oracle's TR-ALS and rBKI-TK-TR (Algorithm 3)."""
import numpy as np

import synth
from oracle import metrics, tensor, tr


def _cores(g, dims, ranks):
    return [g.standard_normal((ranks[k - 1], dims[k], ranks[k])) for k in range(len(dims))]


def test_subchain_reproduces_tr_model():
    """Eq. unTR: G_(k) = Z_k(2) B_{!=k}^T exactly, for every k (pins subchain's ordering
    against the brute-force-pinned TR model)."""
    g = np.random.default_rng(0)
    dims, ranks = [3, 4, 2, 5], [2, 3, 2, 4]
    cores = _cores(g, dims, ranks)
    x = tensor.tr(cores)
    for k in range(4):
        b = tr.subchain(cores, k)
        zk2 = cores[k].transpose(1, 0, 2).reshape(dims[k], -1)
        np.testing.assert_allclose(tr.unfold_cyclic(x, k), zk2 @ b.T, rtol=1e-12, atol=1e-12)


def test_contraction_identity():
    """Algorithm 3 step 4: R[[Z_n x_2 U_n]] = R[[Z_n]] x_1 U_1 ... x_N U_N (exact)."""
    g = np.random.default_rng(1)
    dims, ranks = [3, 4, 2], [2, 3, 2]
    cores = _cores(g, dims, ranks)
    us = [g.standard_normal((6, 3)), g.standard_normal((5, 4)), g.standard_normal((7, 2))]
    lhs = tensor.tr([tr.contract_factor(c, u) for c, u in zip(cores, us)])
    rhs = tensor.tucker(tensor.tr(cores), us)
    np.testing.assert_allclose(lhs, rhs, rtol=1e-12, atol=1e-12)


def test_als_monotone_and_noiseless_recovery():
    g = np.random.default_rng(2)
    dims, ranks = [5, 6, 4, 5], [2, 3, 2, 2]
    true = _cores(g, dims, ranks)
    x = tensor.tr(true)
    # exact LS updates: the residual never increases
    init = _cores(np.random.default_rng(3), dims, ranks)
    _, fits = tr.tr_als(x, init, maxit=15, tol=0.0)
    assert all(b >= a - 1e-12 for a, b in zip(fits, fits[1:]))
    # from a nearby start ALS recovers the noiseless ring
    near = [c + 1e-4 * g.standard_normal(c.shape) for c in true]
    cores, fits = tr.tr_als(x, near, maxit=20, tol=0.0)
    assert fits[-1] >= 1 - 1e-8


def test_rbki_tk_tr_small_end_to_end():
    wl = synth.config_htr(order=4, size=8, tr_rank=3, tucker_rank=8, p=2, q=1, snr_db=30.0)
    res = tr.rbki_tk_tr(wl.x, wl.ranks, wl.p, wl.q, wl.seed, wl.tr_init, maxit=20, tol=1e-3)
    xh = tensor.tr(res["cores"])
    assert res["cores"][0].shape == (3, 8, 3)
    assert metrics.fit(wl.clean, xh) > 95.0
    assert len(res["fits"]) <= 20
