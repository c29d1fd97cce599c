"""Pins of the oracle's Rayleigh-Ritz refinement (refine_rr, reading c17).

* It recovers the eigenbasis from any rotation of it: for U holding the leading Ritz
  vectors of a mode, refine_rr(X_(n), U G) with a random orthogonal G returns U again (the
  expected value is the unrefined oracle factor, not refine_rr's own output).
* On the oracle's own factors it is the identity (Z_r is diagonal in exact arithmetic).
* It never changes the projector U U^T, so the reconstruction error is unchanged."""
import numpy as np

import synth
from oracle import metrics, rbki
from oracle.tensor import unfold


def _wl():
    return synth.config_small_fp64(mc=0, dims=(30, 26, 34), core=(4, 3, 5), p=3, q=2)


def test_refine_recovers_the_eigenbasis_from_a_rotation():
    wl = _wl()
    ref = rbki.rbki_tucker(wl.x, wl.ranks, wl.p, wl.q, wl.seed)
    g = np.random.default_rng(11)
    for n in range(3):
        u = ref["factors"][n]
        rot, _ = np.linalg.qr(g.standard_normal((u.shape[1], u.shape[1])))
        u2, lam2 = rbki.refine_rr(unfold(wl.x, n), u @ rot)
        np.testing.assert_allclose(u2, u, atol=1e-10)
        np.testing.assert_allclose(lam2, ref["eigvals"][n], rtol=1e-10)


def test_refine_is_the_identity_on_ritz_vectors_and_keeps_the_projector():
    wl = _wl()
    ref = rbki.rbki_tucker(wl.x, wl.ranks, wl.p, wl.q, wl.seed)
    rr = rbki.rbki_tucker(wl.x, wl.ranks, wl.p, wl.q, wl.seed, refine=True)
    for n in range(3):
        np.testing.assert_allclose(rr["factors"][n], ref["factors"][n], atol=1e-10)
        np.testing.assert_allclose(rr["eigvals"][n], ref["eigvals"][n], rtol=1e-10)
        assert metrics.max_principal_sine(rr["factors"][n], ref["factors"][n]) <= 1e-10
    assert abs(rr["core_norm2"] - ref["core_norm2"]) <= 1e-12 * ref["x_norm2"]


def test_refine_of_a_perturbed_basis_keeps_its_span():
    wl = _wl()
    xn = unfold(wl.x, 0)
    g = np.random.default_rng(5)
    u, _ = np.linalg.qr(g.standard_normal((xn.shape[0], 4)))
    u2, lam = rbki.refine_rr(xn, u)
    np.testing.assert_allclose(u2 @ u2.T, u @ u.T, atol=1e-12)
    assert np.all(np.diff(lam) <= 0)
    np.testing.assert_allclose(np.diag(u2.T @ xn @ xn.T @ u2), lam, rtol=1e-10)
