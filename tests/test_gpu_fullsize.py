"""GPU parity at the workloads' full sizes, in the launch configuration the bench times.

* 512^3 power-law tensor (R = 20, p = 10, q = 3): the FP64 GPU path against the oracle's
  full decomposition (principal-angle sines <= 1e-10, eigenvalues, reconstruction error to
  1e-12 relative); the mixed path's error within 1% of the oracle's; one tensor-core Krylov
  step against the exact product on the BF16-rounded tensor.
* 1024 x 1024 x 3 x 256 video-shaped tensor (p = 10, q = 4; b = 250 on the two 1024
  modes, the Gram path on the colour mode): the same FP64 and mixed bars.
* the served stream's first requests at their real sizes, through the server.

The 64^3 and 16^6 workloads run at full size in test_gpu_parity.py and test_gpu_htr.py."""
import time

import numpy as np
from parity_bars import err_matches
import pytest

import synth
from oracle import metrics, rbki
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


def _sign_convention(u):
    """Algorithm 2 step 5 with reading c5: each column's largest-|.| entry (lowest row on
    ties) is positive."""
    i = np.argmax(np.abs(u), axis=0)
    return bool(np.all(u[i, np.arange(u.shape[1])] > 0))


def _mixed_leading_sines(ref, us, x_norm2):
    """Principal sines of the mixed factors' leading, well-separated subspaces against the
    oracle's.  Bound (Davis-Kahan sin-theta): the mixed path decomposes the BF16-rounded
    tensor, |dX|_F <= 2^-8 |X|_F, so |d(X X^T)|_2 <= 2 sigma_1 2^-8 |X|_F + 2^-16 |X|_F^2,
    and the leading-k subspace moves by at most that over the gap lambda_k - lambda_{k+1};
    a factor 2 covers the BF16 Omega and the FP32 accumulation.  Only k with a gap of at
    least 5% of lambda_1 are compared (the tail is noise-level and not unique)."""
    u8 = 2.0 ** -8
    xf = np.sqrt(x_norm2)
    worst = []
    for n, u in enumerate(us):
        lam = np.asarray(ref["eigvals"][n])
        sig1 = np.sqrt(lam[0])
        for k in range(1, len(lam)):
            gap = lam[k - 1] - lam[k]
            if gap < 0.05 * lam[0]:
                continue
            bound = 2.0 * (2.0 * sig1 * u8 * xf + u8 * u8 * x_norm2) / gap
            s = metrics.max_principal_sine(ref["factors"][n][:, :k], u[:, :k])
            assert s <= bound, (n, k, s, bound)
            worst.append((s, bound))
    return worst


def _fp64_and_mixed(rb, wl, mixed_prec="bf16"):
    ref = rbki.rbki_tucker(wl.x, wl.ranks, wl.p, wl.q, wl.seed)
    e_ref = np.sqrt(max(ref["x_norm2"] - ref["core_norm2"], 0.0))
    x = torch.from_numpy(np.ascontiguousarray(wl.x)).cuda()
    out = rb.rbki_tucker(x, wl.ranks, wl.p, wl.q, wl.seed, prec="fp64")
    torch.cuda.synchronize()
    N = x.dim()
    info = out["info"].cpu().numpy()
    assert list(info[:N]) == ref["kept"]
    assert list(info[N:2 * N]) == [1 if p == "gram" else 0 for p in ref["path"]]
    assert info[2 * N] == 0
    for n in range(N):
        u = out["factors"][n].cpu().numpy()
        assert np.linalg.norm(u.T @ u - np.eye(u.shape[1])) <= 1e-12
        assert metrics.max_principal_sine(ref["factors"][n], u) <= 1e-10
        assert _sign_convention(u)
        np.testing.assert_allclose(out["eigvals"][n].cpu().numpy(), ref["eigvals"][n], rtol=1e-11,
                                   atol=1e-12 * ref["eigvals"][n][0])
    e = _err(out["norms"])
    assert err_matches(e, e_ref, ref["x_norm2"])
    del out
    mixed = rb.rbki_tucker(x, wl.ranks, wl.p, wl.q, wl.seed, prec=mixed_prec)
    torch.cuda.synchronize()
    assert mixed["info"].cpu().numpy()[2 * N] == 0
    em = _err(mixed["norms"])
    assert abs(em - e_ref) <= 0.01 * e_ref
    us = [u.cpu().numpy() for u in mixed["factors"]]
    for u in us:
        assert np.linalg.norm(u.T @ u - np.eye(u.shape[1])) <= 1e-12
        assert _sign_convention(u)
    return ref, mixed, _mixed_leading_sines(ref, us, ref["x_norm2"])


def test_power_law_512_full_size(rb):
    wl = synth.config_large(size=512)
    _, _, compared = _fp64_and_mixed(rb, wl)
    # the power-law spectra (sigma_k ~ k^-1/2) have well-separated leading directions
    assert compared, "no well-separated leading subspace was compared"


def test_krylov_step_512_full_size(rb):
    """One BF16 tensor-core Krylov step per mode at 512^3 (the bench's launch shape,
    s = 30) against the exact product on the BF16-rounded tensor."""
    wl = synth.config_large(size=512)
    xt = torch.from_numpy(wl.x).cuda().bfloat16()
    xb = xt.double().cpu().numpy()
    g = np.random.default_rng(3)
    for mode in range(3):
        q, _ = np.linalg.qr(g.standard_normal((512, 30)))
        p = rb.rbki_krylov_product(xt, mode, torch.from_numpy(q).cuda(), prec="bf16").cpu().numpy()
        xn = unfold(xb, mode)
        want = xn @ (xn.T @ q)
        assert np.linalg.norm(p - want) <= 2e-3 * np.linalg.norm(want)


def test_video_full_size(rb):
    wl = synth.config_video()
    _, mixed, _ = _fp64_and_mixed(rb, wl)   # Gaussian-core spectra: gaps below 5% are skipped
    # denoising: the mixed result against the clean field, through the core identity
    # |X_clean - X^|^2 = |X_clean|^2 - 2 <X_clean, X^> + |G|^2 (factors orthonormal)
    g = mixed["core"].cpu().numpy()
    us = [u.cpu().numpy() for u in mixed["factors"]]
    proj = wl.clean                                   # FP32; the first contraction shrinks 1024 -> 40
    for n, u in enumerate(us):
        proj = np.moveaxis(np.tensordot(u.T.astype(proj.dtype), proj, axes=(1, n)), 0, n)
        proj = proj.astype(np.float64)
    c2 = sum(float(np.dot(s.ravel().astype(np.float64), s.ravel().astype(np.float64))) for s in wl.clean)
    d2 = c2 - 2.0 * float(np.sum(proj * g)) + float(np.sum(g * g))
    rel = np.sqrt(max(d2, 0.0) / c2)
    noise_rel = 10 ** (-5.0 / 20.0)          # the input's noise level at 5 dB
    assert rel < 0.2 * noise_rel              # a rank-(40,40,3,30) fit removes most of the noise


def test_served_stream_prefix_full_size(rb):
    reqs = synth.serve_stream(n_requests=8, seed=5000)
    wls = [synth.serve_request_tensor(r, dtype=np.float64) for r in reqs]
    with rb.RbkiServer(0, mem_budget=2 << 30, max_slots=4) as srv:
        subs = []
        for wl in wls:
            x = torch.from_numpy(wl.x).cuda()
            subs.append((srv.submit(x, wl.ranks, wl.p, wl.q, wl.seed, prec="fp64"),
                         srv.submit(x.bfloat16(), wl.ranks, wl.p, wl.q, wl.seed, prec="bf16")))
        tickets = [t for pair in subs for (t, _) in pair]
        t0, done = time.time(), {}
        while len(done) < len(tickets) and time.time() - t0 < 300:
            for t in tickets:
                if t not in done:
                    ok, st, lat = srv.poll(t)
                    if ok:
                        done[t] = st
            time.sleep(0.002)
        assert all(done[t] == 0 for t in tickets)
    for wl, ((_, o64), (_, omx)) in zip(wls, subs):
        ref = rbki.rbki_tucker(wl.x, wl.ranks, wl.p, wl.q, wl.seed)
        e_ref = np.sqrt(max(ref["x_norm2"] - ref["core_norm2"], 0.0))
        for n, u in enumerate(o64["factors"]):
            assert metrics.max_principal_sine(ref["factors"][n], u.cpu().numpy()) <= 1e-10
        assert err_matches(_err(o64["norms"]), e_ref, ref["x_norm2"])
        assert abs(_err(omx["norms"]) - e_ref) <= 0.01 * e_ref
