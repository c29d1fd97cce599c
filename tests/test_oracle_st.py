"""Pins for the sequential-truncation reading of Algorithm 2 (oracle.rbki.rbki_st_tucker).

* With b_n >= I_n on every mode the Krylov space is the whole space, so the method must be
  the textbook sequentially truncated HOSVD: at step n, U^(n) = leading left singular
  vectors of the already contracted tensor's mode-n unfolding (here from LAPACK SVD).
* Error decomposition: the truncation error splits exactly into the residuals of the steps,
  |X - X^|^2 = sum_n |Y_n - Y_n x_n U U^T|^2, because each step is an orthogonal projection
  of the previous residual-free part; and |X - X^|^2 = |X|^2 - |G|^2.
* Exact recovery of a noiseless tensor of the requested multilinear rank.
* The first mode's factor equals the HOSVD reading's (both sketch the original X)."""
import numpy as np

import synth
from oracle import metrics, rbki
from oracle.tensor import ttm, unfold


def _st_hosvd_svd(x, ranks):
    y = np.asarray(x, dtype=np.float64)
    us = []
    for n, r in enumerate(ranks):
        u, _, _ = np.linalg.svd(unfold(y, n), full_matrices=False)
        us.append(u[:, :r])
        y = ttm(y, u[:, :r].T, n)
    return us, y


def test_full_width_equals_textbook_st_hosvd():
    g = synth.rng(11)
    x = synth.gaussian_tucker(g, 3, 12, 4) + 0.2 * g.standard_normal((12, 12, 12))
    ranks = [4, 5, 3]
    out = rbki.rbki_st_tucker(x, ranks, p=8, q=1, seed=3)          # b = 2 (R+p) >= 12: Gram path
    assert out["path"] == ["gram"] * 3
    us, core = _st_hosvd_svd(x, ranks)
    # the Gram path takes eigenvectors of Y_(n) Y_(n)^T: rounding there is eps |Y|^2 over the
    # eigengap, about 1e-12 here, so the bar is 1e-10 (a wrong index or sign gives O(1))
    for u, v in zip(out["factors"], us):
        assert metrics.max_principal_sine(v, u) <= 1e-10
    np.testing.assert_allclose(np.abs(out["core"]), np.abs(core), rtol=0, atol=1e-10 * np.abs(core).max())


def test_error_splits_into_step_residuals():
    wl = synth.config_small_fp64(mc=4)
    out = rbki.rbki_st_tucker(wl.x, wl.ranks, wl.p, wl.q, wl.seed)
    assert out["path"][0] == "krylov"
    err2 = metrics.fnorm(wl.x - rbki.reconstruct(out["core"], out["factors"])) ** 2
    assert abs(err2 - (out["x_norm2"] - out["core_norm2"])) <= 1e-10 * out["x_norm2"]
    assert abs(err2 - sum(out["step_res2"])) <= 1e-10 * out["x_norm2"]
    for u in out["factors"]:
        assert np.linalg.norm(u.T @ u - np.eye(u.shape[1])) <= 1e-13


def test_exact_recovery_noiseless():
    wl = synth.config_small_fp64(mc=5, snr_db=None)
    out = rbki.rbki_st_tucker(wl.x, wl.ranks, wl.p, wl.q, wl.seed)
    x_hat = rbki.reconstruct(out["core"], out["factors"])
    assert metrics.fnorm(wl.x - x_hat) <= 1e-12 * metrics.fnorm(wl.x)


def test_first_mode_matches_hosvd_reading():
    wl = synth.config_small_fp64(mc=6)
    st = rbki.rbki_st_tucker(wl.x, wl.ranks, wl.p, wl.q, wl.seed)
    ho = rbki.rbki_tucker(wl.x, wl.ranks, wl.p, wl.q, wl.seed)
    assert metrics.max_principal_sine(ho["factors"][0], st["factors"][0]) <= 1e-12
    np.testing.assert_allclose(st["eigvals"][0], ho["eigvals"][0], rtol=1e-12)
