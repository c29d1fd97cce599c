"""Pins for the oracle's rBKI sketching (Algorithm 1) and rBKI-TK (Algorithm 2).

Each test checks the oracle against something other than itself: a LAPACK route
(QR + SVD), a theorem or identity of the paper, a special case that reduces to the
T-SVD benchmark, or the numbers the paper prints (Tables 3-4, statistical)."""
import json
import os

import numpy as np
import pytest

import synth
from oracle import metrics, philox, rbki
from oracle.tensor import ttm, unfold

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_tables.json")


def _orth_err(q):
    return float(np.linalg.norm(q.T @ q - np.eye(q.shape[1])))


def test_orth_block_orthonormal_and_span():
    g = np.random.default_rng(0)
    prev = np.linalg.qr(g.standard_normal((200, 20)))[0]
    v = g.standard_normal((200, 12)) @ np.diag(10.0 ** -np.arange(12))   # ill-conditioned block
    q = rbki.orth_block(v, prev)
    assert q.shape[1] == 12
    full = np.concatenate([prev, q], axis=1)
    assert _orth_err(full) <= 1e-13
    k = np.concatenate([prev, v], axis=1)
    resid = k - full @ (full.T @ k)
    assert np.linalg.norm(resid) / np.linalg.norm(k) <= 1e-12


def test_orth_block_deflates_dependent_columns():
    g = np.random.default_rng(1)
    prev = np.linalg.qr(g.standard_normal((50, 5)))[0]
    a = g.standard_normal((50, 3))
    v = np.concatenate([a, a[:, :1] + a[:, 1:2], prev[:, :2] @ g.standard_normal((2, 2))], axis=1)
    q = rbki.orth_block(v, prev)
    assert q.shape[1] == 3                                # the 3 dependent columns dropped
    assert _orth_err(np.concatenate([prev, q], axis=1)) <= 1e-13


def test_q0_equals_randomized_range_finder():
    """q = 0 is the Gaussian randomized range finder (Sec. 2.2, Lemma 2): U from the SVD
    of Q^T X with Q = qr(X Omega) - computed here by LAPACK QR + SVD."""
    wl = synth.config_small_fp64(mc=1)
    x, r, p = wl.x, wl.ranks, wl.p
    res = rbki.rbki_tucker(x, r, p, 0, wl.seed)
    for n in range(3):
        xn = unfold(x, n)
        om = philox.omega_mode(wl.seed, n, x.shape, r[n] + p)
        qq, _ = np.linalg.qr(xn @ om)
        ub, _, _ = np.linalg.svd(qq.T @ xn, full_matrices=False)
        u_ref = qq @ ub[:, : r[n]]
        assert metrics.max_principal_sine(u_ref, res["factors"][n]) <= 1e-12


@pytest.mark.parametrize("force_krylov", [False, True])
def test_full_width_equals_tsvd(force_krylov):
    """b_n >= I_n: the Krylov space is all of R^{I_n}, so rBKI-TK equals truncated HOSVD
    (reading c7); checked both via the Gram path and via the Krylov recurrence."""
    g = synth.rng(7)
    x = synth.gaussian_tucker(g, 3, 10, 3) + 0.3 * g.standard_normal((10, 10, 10))
    ref = rbki.tsvd(x, [3, 3, 3])
    if force_krylov:
        for n in range(3):
            qb = rbki.krylov_basis(x, n, 5, 1, seed=11)       # b = 10 = I
            assert qb.shape[1] == 10
            u, _, _ = rbki.rayleigh_ritz(unfold(x, n), qb, 3)
            assert metrics.max_principal_sine(ref["factors"][n], u) <= 1e-12
    else:
        res = rbki.rbki_tucker(x, [3, 3, 3], 2, 1, 11)
        assert res["path"] == ["gram"] * 3
        for n in range(3):
            assert metrics.max_principal_sine(ref["factors"][n], res["factors"][n]) <= 1e-12
            np.testing.assert_allclose(res["factors"][n], ref["factors"][n], atol=1e-10)


def test_exact_recovery_noiseless():
    wl = synth.config_small_fp64(mc=2, snr_db=None)
    res = rbki.rbki_tucker(wl.x, wl.ranks, wl.p, wl.q, wl.seed)
    xh = rbki.reconstruct(res["core"], res["factors"])
    assert metrics.fnorm(wl.x - xh) / metrics.fnorm(wl.x) <= 1e-12
    for n in range(3):
        assert metrics.max_principal_sine(wl.true_factors[n], res["factors"][n]) <= 1e-12


def test_exact_recovery_power_law_spectrum():
    """Superdiagonal core g_kkk = k^-1/2 with Haar factors: mode spectra are exactly
    sigma_k = k^-1/2 (closed form), and rBKI-TK recovers the tensor exactly."""
    wl = synth.config_large(size=48, rank=6, snr_db=None, p=4, q=2, dtype=np.float64)
    res = rbki.rbki_tucker(wl.x, wl.ranks, wl.p, wl.q, wl.seed)
    xh = rbki.reconstruct(res["core"], res["factors"])
    assert metrics.fnorm(wl.x - xh) / metrics.fnorm(wl.x) <= 1e-12
    for n in range(3):
        np.testing.assert_allclose(res["eigvals"][n], 1.0 / np.arange(1, 7), rtol=1e-12)


def test_theorem1_rayleigh_ritz_optimal_in_span():
    """Theorem 1: within span(Q), Q (Q^T X)_k is the best rank-k approximation; no other
    R-dimensional subspace of span(Q) does better.  Also Remark 1's identity
    |X - U U^T X|^2 = |X|^2 - sum_{i<=R} lambda_i(Z) and Cauchy interlacing."""
    wl = synth.config_small_fp64(mc=3)
    x, r = wl.x, wl.ranks[0]
    xn = unfold(x, 0)
    qb = rbki.krylov_basis(x, 0, r + wl.p, wl.q, wl.seed)
    u, lam, z = rbki.rayleigh_ritz(xn, qb, r)
    best = metrics.fnorm(xn - u @ (u.T @ xn))
    g = np.random.default_rng(5)
    for _ in range(20):
        v = qb @ np.linalg.qr(g.standard_normal((qb.shape[1], r)))[0]
        assert best <= metrics.fnorm(xn - v @ (v.T @ xn)) + 1e-12
    np.testing.assert_allclose(best ** 2, metrics.fnorm(xn) ** 2 - lam.sum(), rtol=1e-11)
    sig2 = np.linalg.svd(xn, compute_uv=False) ** 2
    lz = np.sort(np.linalg.eigvalsh(z))[::-1]
    assert np.all(lz <= sig2[: lz.size] * (1 + 1e-12) + 1e-12)


def test_core_identity_pythagorean_and_theorem2():
    """|X - X^|^2 = |X|^2 - |G|^2 (orthogonal projectors); Eq. Pythagorean; Theorem 2
    upper bound |X - X~_k| <= 2 alpha + beta with alpha = |X - X x_n Q Q^T| and the
    truncated-HOSVD error as beta (reading c14)."""
    wl = synth.config_small_fp64(mc=4, snr_db=5.0)
    x = wl.x
    res = rbki.rbki_tucker(x, wl.ranks, wl.p, wl.q, wl.seed)
    xh = rbki.reconstruct(res["core"], res["factors"])
    err2 = metrics.fnorm(x - xh) ** 2
    np.testing.assert_allclose(err2, res["x_norm2"] - res["core_norm2"], rtol=1e-10)
    per_mode = sum(metrics.fnorm(x - ttm(x, u @ u.T, n)) ** 2 for n, u in enumerate(res["factors"]))
    assert err2 <= per_mode * (1 + 1e-12)
    xt = x
    for n in range(3):
        qb = rbki.krylov_basis(x, n, wl.ranks[n] + wl.p, wl.q, wl.seed)
        xt = ttm(xt, qb @ qb.T, n)
    alpha = metrics.fnorm(x - xt)
    ts = rbki.tsvd(x, wl.ranks)
    beta = metrics.fnorm(x - rbki.reconstruct(ts["core"], ts["factors"]))
    e = metrics.fnorm(x - xh)
    assert e <= 2 * alpha + beta
    assert e >= beta * (1 - 2e-3)                       # RErr ~ 1 (may dip below 1 slightly)


def test_energy_nested_in_q_and_p():
    """Nested Krylov spaces: captured energy sum_{i<=R} lambda_i(Z) is non-decreasing in q
    (fixed Omega) and in p (Omega columns keyed by s)."""
    wl = synth.config_small_fp64(mc=5, snr_db=0.0)
    xn = unfold(wl.x, 1)
    r = wl.ranks[1]
    prev = -1.0
    for q in range(4):
        qb = rbki.krylov_basis(wl.x, 1, r + 2, q, wl.seed)
        _, lam, _ = rbki.rayleigh_ritz(xn, qb, r)
        assert lam.sum() >= prev * (1 - 1e-13)
        prev = lam.sum()
    prev = -1.0
    for p in range(0, 8, 2):
        qb = rbki.krylov_basis(wl.x, 1, r + p, 1, wl.seed)
        _, lam, _ = rbki.rayleigh_ritz(xn, qb, r)
        assert lam.sum() >= prev * (1 - 1e-13)
        prev = lam.sum()


def test_rank_deficient_completion():
    """Fewer surviving directions than R: U completed by an orthonormal complement."""
    g = synth.rng(9)
    x = synth.tucker_full(g.standard_normal((2, 2, 2)), [synth.haar_factor(g, 12, 2)] * 3)
    res = rbki.rbki_tucker(x, [4, 4, 4], 0, 0, 3)       # S = 4, true rank 2
    for n in range(3):
        u = res["factors"][n]
        assert _orth_err(u) <= 1e-12
        assert res["kept"][n] == 2
    xh = rbki.reconstruct(res["core"], res["factors"])
    assert metrics.fnorm(x - xh) / metrics.fnorm(x) <= 1e-12


def test_fig3_singular_value_ratio():
    """Fig. 3: sigma1/sigma2 of X_(1) ~ 1.6 for Gaussian data and ~ 5 for power-functional
    data ([N=3, I=10, R=5], 20 dB); the Gaussian ratio is a median over seeds."""
    ratios = []
    for s in range(40):
        g = synth.rng(400 + s)
        x = synth.add_noise_snr(synth.gaussian_tucker(g, 3, 10, 5), 20.0, g)
        sv = np.linalg.svd(unfold(x, 0), compute_uv=False)
        ratios.append(sv[0] / sv[1])
    assert 1.2 <= np.median(ratios) <= 2.2
    x = synth.add_noise_snr(synth.power_functional(3, 10), 20.0, synth.rng(1))
    sv = np.linalg.svd(unfold(x, 0), compute_uv=False)
    assert 4.0 <= sv[0] / sv[1] <= 6.5


@pytest.mark.slow
@pytest.mark.parametrize("idx", [0, 1, 2])
def test_table3_gaussian(idx):
    """Table 3 (statistical): T-SVD Fit within 1.0 point of the paper; rBKI RErr <= 1.05."""
    tab = json.load(open(GOLDEN))["gaussian_3_200_10"]
    snr = tab["snr_db"][idx]
    fits, rerrs = [], []
    for mc in range(2):
        g = synth.rng(100 + mc)
        clean = synth.gaussian_tucker(g, 3, 200, 10)
        x = synth.add_noise_snr(clean, snr, g)
        ts = rbki.tsvd(x, [10] * 3)
        xt = rbki.reconstruct(ts["core"], ts["factors"])
        rb = rbki.rbki_tucker(x, [10] * 3, 5, 2, 42 + mc)
        xr = rbki.reconstruct(rb["core"], rb["factors"])
        fits.append(metrics.fit(clean, xt))
        rerrs.append(metrics.rerr(clean, xr, xt))
    assert abs(np.mean(fits) - tab["tsvd_fit"][idx]) <= 1.0
    assert np.mean(rerrs) <= 1.05


@pytest.mark.slow
def test_table4_power_functional():
    """Table 4, [N=3, I=200, R=10] at 5 dB: T-SVD Fit 97.09; rBKI RErr 1.10 (q = 2)."""
    tab = json.load(open(GOLDEN))["power_3_200_10"]
    clean = synth.power_functional(3, 200)
    fits, rerrs = [], []
    for mc in range(2):
        x = synth.add_noise_snr(clean, tab["snr_db"], synth.rng(200 + mc))
        ts = rbki.tsvd(x, [10] * 3)
        xt = rbki.reconstruct(ts["core"], ts["factors"])
        rb = rbki.rbki_tucker(x, [10] * 3, 5, 2, 42 + mc)
        xr = rbki.reconstruct(rb["core"], rb["factors"])
        fits.append(metrics.fit(clean, xt))
        rerrs.append(metrics.rerr(clean, xr, xt))
    assert abs(np.mean(fits) - tab["tsvd_fit"]) <= 1.0
    assert abs(np.mean(rerrs) - tab["rbki_rerr"]) <= 0.05
