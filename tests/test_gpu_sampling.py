"""GPU parity of partial column sampling (rbki_params.omega) against the oracle
(oracle.sampling, oracle.rbki with omega), through the C ABI.

* the kept units: bit-exact against the oracle's selection;
* FP64 decompositions: principal-angle sines <= 1e-10, Ritz values to 1e-11, the
  reconstruction error to 1e-12 relative (same units, same Omega on Y's columns);
* the mixed path: error within 1% of the oracle's sampled decomposition;
* sampling composes with the sequential reading, at 512^3 too."""
import numpy as np
from parity_bars import err_matches
import pytest

import synth
from oracle import metrics, rbki, sampling
from oracle.tensor import unfold

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


@pytest.mark.parametrize("nu,kept", [(1, 1), (7, 7), (40, 1), (40, 10), (313, 32), (2048, 1024),
                                     (24576, 2458), (100000, 77777)])
def test_sample_units_bit_exact(rb, nu, kept):
    for seed, mode in ((0, 0), (42, 1), (2**40 + 3, 5)):
        got = rb.rbki_sample_units(seed, mode, nu, kept).cpu().numpy()
        want = sampling.sample_units(seed, mode, nu, kept)
        np.testing.assert_array_equal(got, want)


def _check_fp64(rb, x, ranks, p, q, seed, omega, sequential=False):
    fn = rbki.rbki_st_tucker if sequential else rbki.rbki_tucker
    ref = fn(x, ranks, p, q, seed, omega=omega)
    flags = rb.FLAG_SEQUENTIAL if sequential else 0
    xt = torch.from_numpy(np.ascontiguousarray(x)).cuda()
    out = rb.rbki_tucker(xt, ranks, p, q, seed, prec="fp64", flags=flags, omega=omega)
    torch.cuda.synchronize()
    N = x.ndim
    info = out["info"].cpu().numpy()
    assert list(info[:N]) == ref["kept"]
    assert list(info[N:2 * N]) == [1 if p_ == "gram" else 0 for p_ in ref["path"]]
    assert info[2 * N] == 0
    for n in range(N):
        u = out["factors"][n].cpu().numpy()
        assert np.linalg.norm(u.T @ u - np.eye(u.shape[1])) <= 1e-12
        assert metrics.max_principal_sine(ref["factors"][n], u) <= 1e-10
        np.testing.assert_allclose(out["eigvals"][n].cpu().numpy(), ref["eigvals"][n], rtol=1e-11,
                                   atol=1e-12 * ref["eigvals"][n][0])
    e_ref = np.sqrt(max(ref["x_norm2"] - ref["core_norm2"], 0.0))
    assert err_matches(_err(out["norms"]), e_ref, ref["x_norm2"])
    return out, ref


@pytest.mark.parametrize("case", [
    dict(mc=0, omega=0.5),                                                   # 64^3: C>1 ragged units, C=1
    dict(mc=1, dims=(37, 23, 41), core=(5, 4, 6), p=3, q=1, omega=0.3),       # ragged everywhere
    dict(mc=2, dims=(12, 30, 9, 25), core=(3, 4, 2, 5), p=2, q=2, omega=0.2), # order 4, Gram modes unsampled
    dict(mc=3, dims=(136, 40, 300), core=(6, 5, 4), p=4, q=2, omega=0.05),    # one unit on some modes
])
def test_sampled_fp64_matches_oracle(rb, case):
    omega = case.pop("omega")
    wl = synth.config_small_fp64(**case)
    _check_fp64(rb, wl.x, wl.ranks, wl.p, wl.q, wl.seed, omega)


def test_sampled_sequential_fp64(rb):
    wl = synth.config_small_fp64(mc=4, dims=(96, 80, 72), core=(6, 5, 4), p=3, q=2)
    _check_fp64(rb, wl.x, wl.ranks, wl.p, wl.q, wl.seed, 0.4, sequential=True)


def test_sampled_mode_basis(rb):
    wl = synth.config_small_fp64(mc=5)
    x = torch.from_numpy(wl.x).cuda()
    for n in range(3):
        qg = rb.rbki_mode_basis(x, wl.ranks, wl.p, wl.q, wl.seed, n, prec="fp64", omega=0.3).cpu().numpy()
        y, _ = sampling.sampled_mode(wl.x, n, wl.seed, 0.3)
        from oracle import philox
        s = wl.ranks[n] + wl.p
        om = philox.omega(wl.seed, n, np.arange(y.shape[1], dtype=np.uint64), s)
        qr = np.concatenate(rbki.rbki(y, om, wl.q), axis=1)
        assert metrics.max_principal_sine(qr, qg) <= 1e-10 and metrics.max_principal_sine(qg, qr) <= 1e-10


def test_sampled_power_law_256_mixed(rb):
    wl = synth.config_large(size=256)
    _, ref = _check_fp64(rb, wl.x, wl.ranks, wl.p, wl.q, wl.seed, 0.25)
    e_ref = np.sqrt(max(ref["x_norm2"] - ref["core_norm2"], 0.0))
    x = torch.from_numpy(wl.x).cuda()
    for prec in ("bf16", "fp16"):
        out = rb.rbki_tucker(x, wl.ranks, wl.p, wl.q, wl.seed, prec=prec, omega=0.25)
        torch.cuda.synchronize()
        assert out["info"].cpu().numpy()[6] == 0
        assert abs(_err(out["norms"]) - e_ref) <= 0.01 * e_ref, prec


def test_sampled_512_full_size(rb):
    wl = synth.config_large(size=512)
    _, ref = _check_fp64(rb, wl.x, wl.ranks, wl.p, wl.q, wl.seed, 0.5)
    e_ref = np.sqrt(max(ref["x_norm2"] - ref["core_norm2"], 0.0))
    out = rb.rbki_tucker(torch.from_numpy(wl.x).cuda(), wl.ranks, wl.p, wl.q, wl.seed, prec="bf16", omega=0.5)
    assert abs(_err(out["norms"]) - e_ref) <= 0.01 * e_ref
    # sampled and sequential together, mixed precision
    st = rbki.rbki_st_tucker(wl.x, wl.ranks, wl.p, wl.q, wl.seed, omega=0.5)
    e_st = np.sqrt(max(st["x_norm2"] - st["core_norm2"], 0.0))
    o2 = rb.rbki_tucker(torch.from_numpy(wl.x).cuda(), wl.ranks, wl.p, wl.q, wl.seed, prec="bf16",
                        flags=rb.FLAG_SEQUENTIAL, omega=0.5)
    assert abs(_err(o2["norms"]) - e_st) <= 0.01 * e_st


def test_omega_validation(rb):
    x = torch.zeros((16, 16, 16), dtype=torch.float64, device="cuda")
    with pytest.raises(rb.RbkiError):
        rb.rbki_tucker(x, [2, 2, 2], 2, 1, 0, prec="fp64", omega=float("nan"))
    with pytest.raises(rb.RbkiError):
        rb.rbki_sample_units(0, 0, 10, 11)
