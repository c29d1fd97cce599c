"""GPU parity of the power-iteration baseline (RBKI_FLAG_POWER) and the adaptive Krylov
depth (RBKI_FLAG_ADAPTIVE_Q) against the oracle (oracle.rbki variant="power", q_tol),
through the C ABI.

FP64 bar: principal-angle sines <= 1e-10, Ritz values to 1e-11, the reconstruction error to
1e-12 relative, and the adaptive depth per mode equal to the oracle's (both decide in FP64 on
the same fit formula; the cases are checked not to be borderline).  Mixed bar: the error
within 1% of the oracle's, a depth within the bound."""
import numpy as np
from parity_bars import err_matches
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


def _err(norms):
    n = norms.cpu().numpy()
    return float(np.sqrt(max(n[0] - n[1], 0.0)))


def _check(rb, x, ranks, p, q, seed, flags, ref, sequential=False):
    xt = torch.from_numpy(np.ascontiguousarray(x)).cuda()
    kw = dict(q_tol=ref.get("_q_tol", 0.0))
    out = rb.rbki_tucker(xt, ranks, p, q, seed, prec="fp64", flags=flags, **kw)
    torch.cuda.synchronize()
    N = x.ndim
    info = out["info"].cpu().numpy()
    assert list(info[:N]) == ref["kept"]
    assert list(info[N:2 * N]) == [1 if p_ == "gram" else 0 for p_ in ref["path"]]
    assert info[2 * N] == 0
    if "q_used" in ref:
        assert list(out["q_used"].cpu().numpy()) == ref["q_used"]
    for n in range(N):
        u = out["factors"][n].cpu().numpy()
        assert np.linalg.norm(u.T @ u - np.eye(u.shape[1])) <= 1e-12
        assert metrics.max_principal_sine(ref["factors"][n], u) <= 1e-10
        np.testing.assert_allclose(out["eigvals"][n].cpu().numpy(), ref["eigvals"][n], rtol=1e-11,
                                   atol=1e-12 * ref["eigvals"][n][0])
    e_ref = np.sqrt(max(ref["x_norm2"] - ref["core_norm2"], 0.0))
    assert err_matches(_err(out["norms"]), e_ref, ref["x_norm2"])
    return out


@pytest.mark.parametrize("case", [
    dict(mc=0, q=2),
    dict(mc=1, dims=(37, 23, 41), core=(5, 4, 6), p=3, q=3),
    dict(mc=2, dims=(12, 30, 9, 25), core=(3, 4, 2, 5), p=2, q=1),
    dict(mc=3, dims=(136, 40, 96), core=(6, 5, 4), p=4, q=0),
])
def test_power_fp64_matches_oracle(rb, case):
    q = case.pop("q")
    wl = synth.config_small_fp64(**case)
    ref = rbki.rbki_tucker(wl.x, wl.ranks, wl.p, q, wl.seed, variant="power")
    _check(rb, wl.x, wl.ranks, wl.p, q, wl.seed, rb.FLAG_POWER, ref)


def test_power_sequential_and_sampled(rb):
    wl = synth.config_small_fp64(mc=4, dims=(96, 80, 72), core=(6, 5, 4), p=3, q=2)
    ref = rbki.rbki_st_tucker(wl.x, wl.ranks, wl.p, wl.q, wl.seed, variant="power")
    _check(rb, wl.x, wl.ranks, wl.p, wl.q, wl.seed, rb.FLAG_POWER | rb.FLAG_SEQUENTIAL, ref)
    ref = rbki.rbki_tucker(wl.x, wl.ranks, wl.p, wl.q, wl.seed, variant="power", omega=0.4)
    xt = torch.from_numpy(wl.x).cuda()
    out = rb.rbki_tucker(xt, wl.ranks, wl.p, wl.q, wl.seed, prec="fp64", flags=rb.FLAG_POWER, omega=0.4)
    for n in range(3):
        assert metrics.max_principal_sine(ref["factors"][n], out["factors"][n].cpu().numpy()) <= 1e-10


def _adaptive_case(seed=21, size=80, snr=-5.0):
    g = synth.rng(seed)
    clean = synth.gaussian_tucker(g, 3, size, 6)
    return synth.add_noise_snr(clean, snr, g)


@pytest.mark.parametrize("tol", [1e-2, 1e-4, 1e-6])
def test_adaptive_q_fp64_matches_oracle(rb, tol):
    x = _adaptive_case()
    ranks, p, q_max, seed = [6, 6, 6], 3, 6, 4
    ref = rbki.rbki_tucker(x, ranks, p, q_max, seed, q_tol=tol)
    ref["_q_tol"] = tol
    # not borderline: every decision the oracle took is clear of the threshold
    from oracle.tensor import unfold
    from oracle import philox
    for n in range(3):
        xn = unfold(x, n)
        om = philox.omega_mode(seed, n, x.shape, ranks[n] + p)
        _, _, _, _, fits = rbki.krylov_adaptive(xn, om, ranks[n], q_max, tol)
        for j in range(1, len(fits)):
            assert abs(abs(fits[j] - fits[j - 1]) - tol) > 1e-9
    _check(rb, x, ranks, p, q_max, seed, rb.FLAG_ADAPTIVE_Q, ref)


def test_adaptive_q_mixed_and_host_io(rb):
    wl = synth.config_large(size=256)
    tol = 1e-4
    ref = rbki.rbki_tucker(wl.x, wl.ranks, wl.p, wl.q, wl.seed, q_tol=tol)
    e_ref = np.sqrt(max(ref["x_norm2"] - ref["core_norm2"], 0.0))
    x = torch.from_numpy(wl.x).cuda()
    out = rb.rbki_tucker(x, wl.ranks, wl.p, wl.q, wl.seed, prec="bf16", flags=rb.FLAG_ADAPTIVE_Q, q_tol=tol)
    torch.cuda.synchronize()
    qu = out["q_used"].cpu().numpy()
    assert np.all((qu >= 1) & (qu <= wl.q))
    assert abs(_err(out["norms"]) - e_ref) <= 0.01 * e_ref
    # FP64 through host buffers: same depths as the oracle
    host = rb.rbki_tucker(torch.from_numpy(wl.x).pin_memory(), wl.ranks, wl.p, wl.q, wl.seed, prec="fp64",
                          flags=rb.FLAG_ADAPTIVE_Q | rb.FLAG_HOST_IO, q_tol=tol)
    assert list(host["q_used"].numpy()) == ref["q_used"]
    assert err_matches(_err(host["norms"]), e_ref, ref["x_norm2"])


def test_variant_flag_validation(rb):
    x = torch.zeros((16, 16, 16), dtype=torch.float64, device="cuda")
    for flags, kw in ((rb.FLAG_ADAPTIVE_Q | rb.FLAG_POWER, {}), (rb.FLAG_ADAPTIVE_Q, dict(q_tol=-1.0)),
                      (rb.FLAG_ADAPTIVE_Q | rb.FLAG_SEQUENTIAL, {}), (rb.FLAG_ADAPTIVE_Q, dict(omega=0.5))):
        with pytest.raises(rb.RbkiError):
            rb.rbki_tucker(x, [2, 2, 2], 2, 1, 0, prec="fp64", flags=flags, **kw)
