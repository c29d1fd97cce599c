"""GPU edge cases of the variants, through the C ABI (FP64 path):
* column sampling and power iteration recover a noiseless tensor of multilinear rank R;
* adaptive depth with an infinite tolerance stops at q = 1 (the fixed q = 1 result);
* a one-item batch and a one-part divide-and-conquer equal the plain call bit for bit."""
import numpy as np
import pytest

import synth
from oracle import metrics, rbki

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def rb():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2211_14828_gb300 as rb
    rb.lib()
    return rb


def _recovers(out, x):
    g = out["core"].cpu().numpy()
    us = [u.cpu().numpy() for u in out["factors"]]
    return metrics.fnorm(x - rbki.reconstruct(g, us)) <= 1e-11 * metrics.fnorm(x)


def test_noiseless_recovery_sampled_and_power(rb):
    wl = synth.config_small_fp64(mc=20, dims=(48, 40, 36), core=(4, 3, 5), snr_db=None, p=3, q=1)
    x = torch.from_numpy(wl.x).cuda()
    for kw in (dict(omega=0.3), dict(flags=rb.FLAG_POWER), dict(flags=rb.FLAG_SEQUENTIAL, omega=0.5)):
        out = rb.rbki_tucker(x, wl.ranks, wl.p, 2, wl.seed, prec="fp64", **kw)
        torch.cuda.synchronize()
        assert _recovers(out, wl.x), kw


def test_adaptive_stops_at_first_check_with_infinite_tolerance(rb):
    """q_tol = inf: every Krylov-path mode stops at its first check, q = 1, and the result is
    the fixed-depth q = 1 decomposition.  (q_tol = 0 is not tested: converged fits that agree
    to the last bit make that decision a matter of rounding.)"""
    wl = synth.config_small_fp64(mc=21, dims=(80, 70, 60), core=(5, 5, 5), p=3, q=4)
    x = torch.from_numpy(wl.x).cuda()
    a = rb.rbki_tucker(x, wl.ranks, wl.p, wl.q, wl.seed, prec="fp64", flags=rb.FLAG_ADAPTIVE_Q,
                       q_tol=float("inf"))
    torch.cuda.synchronize()
    assert list(a["q_used"].cpu().numpy()) == [1, 1, 1]
    ref = rbki.rbki_tucker(wl.x, wl.ranks, wl.p, 1, wl.seed)
    for u, v in zip(a["factors"], ref["factors"]):
        assert metrics.max_principal_sine(v, u.cpu().numpy()) <= 1e-10


def test_single_item_batch_and_single_part(rb):
    wl = synth.config_small_fp64(mc=24, dims=(40, 36, 48), core=(5, 4, 6), p=3, q=2)
    x = torch.from_numpy(wl.x).cuda()
    one = rb.rbki_tucker(x, wl.ranks, wl.p, wl.q, wl.seed, prec="fp64")
    bat = rb.rbki_tucker_batch([x], [wl.ranks], wl.p, wl.q, [wl.seed], prec="fp64")[0]
    _, dc = rb.rbki_divide_and_conquer(x, 2, 1, [wl.ranks], wl.p, wl.q, wl.seed, prec="fp64")
    torch.cuda.synchronize()
    assert torch.equal(one["core"], bat["core"]) and torch.equal(one["core"], dc[0]["core"])
