"""Edge cases of the oracle's variants (CPU):
* column sampling of a noiseless tensor of multilinear rank R recovers it exactly: any
  generic sample of >= R columns spans X_(n)'s column space;
* adaptive depth: q_tol = inf stops at the first check (q = 1), q_tol = -1 never stops early
  (q = bound); power iteration with q = 0 is the rBKI basis with q = 0;
* power iteration and the sequential reading recover noiseless low-rank tensors exactly;
* divide-and-conquer with one index per part."""
import numpy as np

import synth
from oracle import divide, metrics, rbki


def _noiseless(mc=20, dims=(48, 40, 36), core=(4, 3, 5)):
    return synth.config_small_fp64(mc=mc, dims=dims, core=core, snr_db=None, p=3, q=1)


def test_sampling_recovers_noiseless_low_rank():
    wl = _noiseless()
    for om in (0.05, 0.3, 0.7):
        out = rbki.rbki_tucker(wl.x, wl.ranks, wl.p, wl.q, wl.seed, omega=om)
        xr = rbki.reconstruct(out["core"], out["factors"])
        assert metrics.fnorm(wl.x - xr) <= 1e-11 * metrics.fnorm(wl.x), om


def test_adaptive_extremes():
    wl = synth.config_small_fp64(mc=21, dims=(80, 70, 60), core=(5, 5, 5), p=3, q=4)
    a = rbki.rbki_tucker(wl.x, wl.ranks, wl.p, wl.q, wl.seed, q_tol=float("inf"))
    b = rbki.rbki_tucker(wl.x, wl.ranks, wl.p, wl.q, wl.seed, q_tol=-1.0)
    assert a["q_used"] == [1, 1, 1] and b["q_used"] == [wl.q] * 3
    f = rbki.rbki_tucker(wl.x, wl.ranks, wl.p, wl.q, wl.seed)
    for u, v in zip(b["factors"], f["factors"]):
        assert metrics.max_principal_sine(u, v) <= 1e-12


def test_power_and_sequential_exact_recovery():
    wl = _noiseless(mc=22)
    for out in (rbki.rbki_tucker(wl.x, wl.ranks, wl.p, 2, wl.seed, variant="power"),
                rbki.rbki_st_tucker(wl.x, wl.ranks, wl.p, 2, wl.seed),
                rbki.rbki_st_tucker(wl.x, wl.ranks, wl.p, 2, wl.seed, variant="power", omega=0.4)):
        xr = rbki.reconstruct(out["core"], out["factors"])
        assert metrics.fnorm(wl.x - xr) <= 1e-11 * metrics.fnorm(wl.x)
    p0 = rbki.rbki_tucker(wl.x, wl.ranks, wl.p, 0, wl.seed, variant="power")
    k0 = rbki.rbki_tucker(wl.x, wl.ranks, wl.p, 0, wl.seed)
    for u, v in zip(p0["factors"], k0["factors"]):
        np.testing.assert_allclose(u, v, atol=1e-13)


def test_divide_one_index_per_part():
    g = synth.rng(23)
    x = g.standard_normal((10, 12, 5))
    res = divide.divide_and_conquer(x, 2, 5, [[3, 4, 1]] * 5, 2, 1, 7)
    assert [r["core"].shape for r in res["parts"]] == [(3, 4, 1)] * 5
    err2 = metrics.fnorm(x - divide.reconstruct(res, 2)) ** 2
    assert abs(err2 - res["err2"]) <= 1e-10 * res["x_norm2"]
