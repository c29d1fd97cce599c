"""GPU parity of the sequentially truncated reading of Algorithm 2 (RBKI_FLAG_SEQUENTIAL)
against the oracle's rbki_st_tucker, through the C ABI.

FP64 bar: principal-angle sines <= 1e-10, Ritz values to 1e-11, the core entry by entry
(both sides fix the factor signs the same way) to 1e-10 of its largest entry, the
reconstruction error to 1e-12 relative.  Mixed bar: error within 1% of the oracle's.
Also: the host-I/O call, the server and Algorithm 3 accept the flag and give the
device call's result."""
import time

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


def _check_fp64(rb, wl, sine_tol=1e-10):
    ref = rbki.rbki_st_tucker(wl.x, wl.ranks, wl.p, wl.q, wl.seed)
    x = torch.from_numpy(np.ascontiguousarray(wl.x)).cuda()
    out = rb.rbki_tucker(x, wl.ranks, wl.p, wl.q, wl.seed, prec="fp64", flags=rb.FLAG_SEQUENTIAL)
    torch.cuda.synchronize()
    N = x.dim()
    info = out["info"].cpu().numpy()
    assert list(info[:N]) == ref["kept"]
    assert list(info[N:2 * N]) == [1 if p == "gram" else 0 for p in ref["path"]]
    assert info[2 * N] == 0
    for n in range(N):
        u = out["factors"][n].cpu().numpy()
        assert np.linalg.norm(u.T @ u - np.eye(u.shape[1])) <= 1e-12
        assert metrics.max_principal_sine(ref["factors"][n], u) <= sine_tol
        np.testing.assert_allclose(out["eigvals"][n].cpu().numpy(), ref["eigvals"][n], rtol=1e-11,
                                   atol=1e-12 * ref["eigvals"][n][0])
    g = out["core"].cpu().numpy()
    np.testing.assert_allclose(g, ref["core"], rtol=0, atol=1e-10 * np.abs(ref["core"]).max())
    e_ref = np.sqrt(max(ref["x_norm2"] - ref["core_norm2"], 0.0))
    assert err_matches(_err(out["norms"]), e_ref, ref["x_norm2"])
    return out, ref


@pytest.mark.parametrize("case", [
    dict(mc=0),
    dict(mc=1, dims=(37, 23, 41), core=(5, 4, 6), p=3, q=1),          # ragged
    dict(mc=2, dims=(12, 30, 9, 25), core=(3, 4, 2, 5), p=2, q=2),     # order 4, Gram modes
    dict(mc=3, dims=(136, 40, 24), core=(6, 5, 4), p=4, q=2),         # Krylov, Krylov, Gram
])
def test_sequential_fp64_matches_oracle(rb, case):
    _check_fp64(rb, synth.config_small_fp64(**case))


def test_sequential_exact_recovery(rb):
    wl = synth.config_small_fp64(mc=4, snr_db=None)
    out, _ = _check_fp64(rb, wl)
    us = [f.cpu().numpy() for f in out["factors"]]
    x_hat = rbki.reconstruct(out["core"].cpu().numpy(), us)
    assert metrics.fnorm(wl.x - x_hat) <= 1e-12 * metrics.fnorm(wl.x)


def test_sequential_power_law_256(rb):
    """The 512^3 workload's spectrum at 256^3: FP64 at the FP64 bar; BF16 (tensor-core first
    product, FP32 intermediates) within 1% of the oracle's error."""
    wl = synth.config_large(size=256)
    _, ref = _check_fp64(rb, wl)
    e_ref = np.sqrt(max(ref["x_norm2"] - ref["core_norm2"], 0.0))
    x = torch.from_numpy(wl.x).cuda()
    for prec in ("bf16", "fp16"):
        out = rb.rbki_tucker(x, wl.ranks, wl.p, wl.q, wl.seed, prec=prec, flags=rb.FLAG_SEQUENTIAL)
        torch.cuda.synchronize()
        assert out["info"].cpu().numpy()[6] == 0
        e = _err(out["norms"])
        assert np.isfinite(e) and abs(e - e_ref) <= 0.01 * e_ref, (prec, e, e_ref)
        for u in out["factors"]:
            u = u.cpu().numpy()
            assert np.linalg.norm(u.T @ u - np.eye(u.shape[1])) <= 1e-12


def test_sequential_power_law_512_full_size(rb):
    wl = synth.config_large(size=512)
    _, ref = _check_fp64(rb, wl)
    e_ref = np.sqrt(max(ref["x_norm2"] - ref["core_norm2"], 0.0))
    out = rb.rbki_tucker(torch.from_numpy(wl.x).cuda(), wl.ranks, wl.p, wl.q, wl.seed, prec="bf16",
                         flags=rb.FLAG_SEQUENTIAL)
    assert abs(_err(out["norms"]) - e_ref) <= 0.01 * e_ref


def test_sequential_host_io_and_server_agree(rb):
    wl = synth.config_small_fp64(mc=5, dims=(48, 40, 56), core=(5, 4, 6), p=3, q=2)
    x = torch.from_numpy(wl.x).cuda()
    dev = rb.rbki_tucker(x, wl.ranks, wl.p, wl.q, wl.seed, prec="fp64", flags=rb.FLAG_SEQUENTIAL)
    torch.cuda.synchronize()
    host = rb.rbki_tucker(torch.from_numpy(wl.x).pin_memory(), wl.ranks, wl.p, wl.q, wl.seed, prec="fp64",
                          flags=rb.FLAG_SEQUENTIAL | rb.FLAG_HOST_IO)
    assert torch.equal(host["core"], dev["core"].cpu())
    for a, b in zip(host["factors"], dev["factors"]):
        assert torch.equal(a, b.cpu())
    with rb.RbkiServer(0, mem_budget=1 << 30, max_slots=2) as srv:
        tk, o = srv.submit(x, wl.ranks, wl.p, wl.q, wl.seed, prec="fp64", flags=rb.FLAG_SEQUENTIAL)
        t0 = time.time()
        while time.time() - t0 < 60:
            ok, st, _ = srv.poll(tk)
            if ok:
                break
            time.sleep(0.002)
        assert ok and st == 0
    assert torch.equal(o["core"], dev["core"])


def test_sequential_htr_tucker_stage(rb):
    """Algorithm 3 on the sequentially truncated Tucker result: its intermediate Tucker
    output equals the plain sequential call."""
    wl = synth.config_small_fp64(mc=6, dims=(24, 20, 28), core=(6, 5, 7), p=2, q=1)
    x = torch.from_numpy(wl.x).cuda()
    trr = (3, 2, 4)
    init = [torch.from_numpy(c).cuda() for c in synth.tr_init_cores(7, wl.ranks, trr)]
    got = rb.rbki_htr(x, wl.ranks, wl.p, wl.q, wl.seed, trr, init, maxit=3, tol=0.0, prec="fp64",
                      flags=rb.FLAG_SEQUENTIAL)
    ref = rb.rbki_tucker(x, wl.ranks, wl.p, wl.q, wl.seed, prec="fp64", flags=rb.FLAG_SEQUENTIAL)
    torch.cuda.synchronize()
    assert torch.equal(got["tucker"]["core"], ref["core"])
