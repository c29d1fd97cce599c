"""Pins for the in-framework baselines and the adaptive depth (oracle.rbki):

* power iteration (Sec. 3.1, "P-iter"): span(Q_q) equals the span of (X X^T)^q X Omega taken
  by one LAPACK QR of the raw power; q = 0 is the randomized range finder; the block Krylov
  space contains Q_q, so rBKI captures at least as much energy for every q (Theorem 1);
* mode_fit equals the explicit fit of the projection U U^T X_(n);
* adaptive q: the fits are non-decreasing in j (nested spaces), and the result equals the
  fixed-depth decomposition at the depth a brute-force scan of fixed depths selects."""
import numpy as np
import pytest

import synth
from oracle import metrics, philox, rbki
from oracle.tensor import unfold


def _mat(seed, n=60, d=400, decay=0.8):
    g = np.random.default_rng(seed)
    u, _ = np.linalg.qr(g.standard_normal((n, n)))
    v, _ = np.linalg.qr(g.standard_normal((d, n)))
    return (u * decay ** np.arange(n)[None, :]) @ v.T


@pytest.mark.parametrize("q", [0, 1, 2, 3])
def test_power_span_equals_raw_power(q):
    x = _mat(q)
    om = np.random.default_rng(9).standard_normal((x.shape[1], 8))
    qp = rbki.power_basis(x, om, q)
    raw = x @ om
    for _ in range(q):
        raw = x @ (x.T @ raw)
    qr_, _ = np.linalg.qr(raw)
    assert qp.shape == (60, 8)
    assert metrics.max_principal_sine(qr_, qp) <= 1e-9
    assert np.linalg.norm(qp.T @ qp - np.eye(8)) <= 1e-13


def test_krylov_contains_power_and_captures_more():
    wl = synth.config_small_fp64(mc=7)
    for q in (1, 2, 3):
        kr = rbki.rbki_tucker(wl.x, wl.ranks, wl.p, q, wl.seed)
        pw = rbki.rbki_tucker(wl.x, wl.ranks, wl.p, q, wl.seed, variant="power")
        for n in range(3):
            assert np.sum(kr["eigvals"][n]) >= np.sum(pw["eigvals"][n]) - 1e-12 * np.sum(kr["eigvals"][n])
    # the last power block lies inside the Krylov space of the same depth
    xn = unfold(wl.x, 0)
    s = wl.ranks[0] + wl.p
    om = philox.omega_mode(wl.seed, 0, wl.x.shape, s)
    kb = np.concatenate(rbki.rbki(xn, om, 2), axis=1)
    pb = rbki.power_basis(xn, om, 2)
    assert np.linalg.norm(pb - kb @ (kb.T @ pb)) <= 1e-10


def test_mode_fit_is_the_projection_fit():
    wl = synth.config_small_fp64(mc=8)
    xn = unfold(wl.x, 1)
    s = wl.ranks[1] + wl.p
    om = philox.omega_mode(wl.seed, 1, wl.x.shape, s)
    qb = np.concatenate(rbki.rbki(xn, om, 2), axis=1)
    u, lam, _ = rbki.rayleigh_ritz(xn, qb, wl.ranks[1])
    explicit = 1 - np.linalg.norm(xn - u @ (u.T @ xn)) / np.linalg.norm(xn)
    assert abs(rbki.mode_fit(lam, float(np.sum(xn * xn))) - explicit) <= 1e-12


@pytest.mark.parametrize("tol", [1e-2, 1e-3, 1e-4, 1e-6])
def test_adaptive_q_equals_brute_force_depth(tol):
    g = synth.rng(21)
    clean = synth.gaussian_tucker(g, 3, 80, 6)
    x = synth.add_noise_snr(clean, -5.0, g)
    ranks, p, q_max, seed = [6, 6, 6], 3, 6, 4
    ad = rbki.rbki_tucker(x, ranks, p, q_max, seed, q_tol=tol)
    for n in range(3):
        xn = unfold(x, n)
        x2 = float(np.sum(xn * xn))
        fits = []
        for q in range(q_max + 1):
            fx = rbki.rbki_tucker(x, ranks, p, q, seed)
            fits.append(rbki.mode_fit(fx["eigvals"][n], x2))
        assert all(b >= a - 1e-12 for a, b in zip(fits, fits[1:]))
        q_star = next((j for j in range(1, q_max + 1) if abs(fits[j] - fits[j - 1]) <= tol), q_max)
        for j in range(1, q_star + 1):            # the decisions are not borderline
            assert abs(abs(fits[j] - fits[j - 1]) - tol) > 1e-9
        assert ad["q_used"][n] == q_star
        fixed = rbki.rbki_tucker(x, ranks, p, q_star, seed)
        assert metrics.max_principal_sine(fixed["factors"][n], ad["factors"][n]) <= 1e-12
