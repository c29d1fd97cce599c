"""GPU parity of the CUDA path (through the C ABI) against the FP64 CPU oracle.

FP64 path bar: principal-angle sines <= 1e-10 per mode and reconstruction error agreeing
to 1e-12 relative (same seeded Omega and input).  Mixed (BF16 products / FP32 accumulate,
FP64 orthonormalisation and eigensolve) bar: relative reconstruction error within 1% of
the oracle's."""
import numpy as np
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


def _err_from_norms(norms):
    n = norms.cpu().numpy()
    return float(np.sqrt(max(n[0] - n[1], 0.0)))


@pytest.mark.parametrize("dims", [(20, 30, 40), (37, 23, 41), (5, 130, 7), (64, 64, 64), (6, 5, 4, 7)])
@pytest.mark.parametrize("s", [1, 7, 16, 30])
def test_krylov_product_fp64(rb, dims, s):
    g = np.random.default_rng(sum(dims) + s)
    x = g.standard_normal(dims)
    xt = torch.from_numpy(x).cuda()
    for mode in range(len(dims)):
        q = g.standard_normal((dims[mode], s))
        p = rb.rbki_krylov_product(xt, mode, torch.from_numpy(q).cuda(), prec="fp64")
        xn = unfold(x, mode)
        want = xn @ (xn.T @ q)
        np.testing.assert_allclose(p.cpu().numpy(), want, rtol=1e-12, atol=1e-12 * np.abs(want).max())


@pytest.mark.parametrize("dims", [(21, 30, 37), (33, 17, 45)])
def test_krylov_product_bf16_cuda_cores(rb, dims):
    """Shapes the TMA path cannot take (contiguous extent not a multiple of 8) run the
    FP32-accumulate CUDA-core kernels."""
    g = np.random.default_rng(1)
    x = g.standard_normal(dims).astype(np.float32)
    q = g.standard_normal((dims[0], 12))
    xt = torch.from_numpy(x).cuda()
    xb = xt.bfloat16().double().cpu().numpy()          # the staged operand, exactly
    p = rb.rbki_krylov_product(xt, 0, torch.from_numpy(q).cuda(), prec="bf16").cpu().numpy()
    xn = unfold(xb, 0)
    want = xn @ (xn.T @ q)
    rel = np.linalg.norm(p - want) / np.linalg.norm(want)
    assert rel < 2e-5


@pytest.mark.parametrize("n", [1, 2, 5, 36, 48, 97, 120, 200, 250, 256])
def test_syev(rb, n):
    g = np.random.default_rng(n)
    a = g.standard_normal((n, n))
    a = a @ a.T + np.diag(np.linspace(0, 1, n))
    w, V = rb.rbki_syev(torch.from_numpy(a).cuda())
    w, V = w.cpu().numpy(), V.cpu().numpy()
    wr = np.sort(np.linalg.eigvalsh(a))[::-1]
    np.testing.assert_allclose(w, wr, rtol=1e-12, atol=1e-12 * wr[0])
    np.testing.assert_allclose(a @ V, V * w[None, :], atol=1e-11 * wr[0])
    np.testing.assert_allclose(V.T @ V, np.eye(n), atol=1e-13)


@pytest.mark.parametrize("n", [8, 20, 120])
@pytest.mark.parametrize("off", [0.0, 1e-20, 1e-16, 1e-13, 1e-6])
def test_syev_near_diagonal(rb, n, off):
    """A diagonal matrix plus a symmetric perturbation of size `off`: the shape of a Rayleigh
    quotient on vectors that are already Ritz vectors.  The FP32 tridiagonal then splits into
    blocks decoupled by negligible off-diagonal entries, where inverse iteration meets a pair
    of pivot candidates both below its tiny threshold."""
    g = np.random.default_rng(n)
    lam = np.sort(g.uniform(1, 100, n))[::-1]
    e = g.standard_normal((n, n)) * off
    a = np.diag(lam) + (e + e.T) / 2
    w, V = rb.rbki_syev(torch.from_numpy(a).cuda())
    w, V = w.cpu().numpy(), V.cpu().numpy()
    assert np.all(np.isfinite(w)) and np.all(np.isfinite(V))
    wr = np.sort(np.linalg.eigvalsh(a))[::-1]
    np.testing.assert_allclose(w, wr, rtol=1e-12, atol=1e-12 * wr[0])
    np.testing.assert_allclose(a @ V, V * w[None, :], atol=1e-11 * wr[0])
    np.testing.assert_allclose(V.T @ V, np.eye(n), atol=1e-13)


def _sym_with_spectrum(lam, seed):
    g = np.random.default_rng(seed)
    q, r = np.linalg.qr(g.standard_normal((len(lam), len(lam))))
    q *= np.sign(np.diag(r))[None, :]
    return (q * lam[None, :]) @ q.T, q


@pytest.mark.parametrize("kind", ["noise_cluster", "multiple", "eps32_spacing"])
def test_syev_clustered(rb, kind):
    """Spectra of Z on low-rank + noise data: a few separated leading eigenvalues above a
    cluster far narrower than FP32 resolution allows to split.  The separated pairs must
    come out to FP64 accuracy and the cluster as an orthonormal basis of its eigenspace."""
    n = 120
    if kind == "noise_cluster":       # the shape of Z for 512^3, R = 20, p = 10, q = 3
        top = 1.0 / np.arange(1, 21)
        rest = np.sort(np.random.default_rng(1).uniform(6.5e-4, 7.6e-4, n - 20))[::-1]
    elif kind == "multiple":          # an exactly repeated eigenvalue
        top = np.linspace(2.0, 1.0, 10)
        rest = np.full(n - 10, 1e-3)
    else:                             # spacing of a few FP32 ulps
        top = np.linspace(3.0, 2.0, 20)
        rest = 0.5 + 1e-7 * np.arange(n - 20)[::-1]
    lam = np.concatenate([top, rest])
    a, q = _sym_with_spectrum(lam, seed=len(kind))
    w, V = rb.rbki_syev(torch.from_numpy(a).cuda())
    w, V = w.cpu().numpy(), V.cpu().numpy()
    assert np.all(np.isfinite(w)) and np.all(np.isfinite(V))
    k = len(top)
    np.testing.assert_allclose(w[:k], top, rtol=1e-12, atol=1e-13 * lam[0])
    np.testing.assert_allclose(a @ V[:, :k], V[:, :k] * w[None, :k], atol=1e-11 * lam[0])
    np.testing.assert_allclose(V.T @ V, np.eye(n), atol=1e-12)
    width = rest.max() - rest.min()
    assert np.all(np.abs(w[k:] - rest) <= width + 1e-12 * lam[0])
    assert metrics.max_principal_sine(q[:, k:], V[:, k:]) <= 1e-9


def test_mode_basis_span_fp64(rb):
    wl = synth.config_small_fp64(mc=0)
    x = torch.from_numpy(wl.x).cuda()
    for n in range(3):
        q_gpu = rb.rbki_mode_basis(x, wl.ranks, wl.p, wl.q, wl.seed, n, prec="fp64").cpu().numpy()
        q_ref = rbki.krylov_basis(wl.x, n, wl.ranks[n] + wl.p, wl.q, wl.seed)
        assert np.linalg.norm(q_gpu.T @ q_gpu - np.eye(q_gpu.shape[1])) <= 1e-13
        assert metrics.max_principal_sine(q_ref, q_gpu) <= 1e-10
        assert metrics.max_principal_sine(q_gpu, q_ref) <= 1e-10


def _check_fp64(rb, wl, sine_tol=1e-10, err_rtol=1e-12):
    ref = rbki.rbki_tucker(wl.x, wl.ranks, wl.p, wl.q, wl.seed)
    x = torch.from_numpy(np.ascontiguousarray(wl.x)).cuda()
    out = rb.rbki_tucker(x, wl.ranks, wl.p, wl.q, wl.seed, prec="fp64")
    torch.cuda.synchronize()
    err_ref = metrics.fnorm(wl.x - rbki.reconstruct(ref["core"], ref["factors"]))
    for n in range(x.dim()):
        u = out["factors"][n].cpu().numpy()
        assert np.linalg.norm(u.T @ u - np.eye(u.shape[1])) <= 1e-12
        assert metrics.max_principal_sine(ref["factors"][n], u) <= sine_tol
        np.testing.assert_allclose(out["eigvals"][n].cpu().numpy(), ref["eigvals"][n], rtol=1e-11,
                                   atol=1e-12 * ref["eigvals"][n][0])
    info = out["info"].cpu().numpy()
    assert list(info[x.dim(): 2 * x.dim()]) == [1 if p == "gram" else 0 for p in ref["path"]]
    assert info[2 * x.dim()] == 0
    assert list(info[: x.dim()]) == ref["kept"]
    # reconstruction error: identity |X|^2 - |G|^2, and explicit from the returned factors
    g = out["core"].cpu().numpy()
    us = [f.cpu().numpy() for f in out["factors"]]
    err = metrics.fnorm(wl.x - rbki.reconstruct(g, us))
    assert abs(err - err_ref) <= err_rtol * max(err_ref, 1e-300) + 1e-13 * metrics.fnorm(wl.x)
    return out, ref


def test_tucker_fp64_small_config(rb):
    _check_fp64(rb, synth.config_small_fp64(mc=0))


def test_tucker_fp64_ragged_and_order4(rb):
    _check_fp64(rb, synth.config_small_fp64(mc=1, dims=(37, 23, 41), core=(5, 4, 6), p=3, q=1))
    _check_fp64(rb, synth.config_small_fp64(mc=2, dims=(12, 30, 9, 25), core=(3, 4, 2, 5), p=2, q=2))


def test_tucker_fp64_exact_recovery(rb):
    wl = synth.config_small_fp64(mc=3, snr_db=None)
    out, _ = _check_fp64(rb, wl)
    g = out["core"].cpu().numpy()
    us = [f.cpu().numpy() for f in out["factors"]]
    assert metrics.fnorm(wl.x - rbki.reconstruct(g, us)) / metrics.fnorm(wl.x) <= 1e-12


def test_tucker_power_law_256(rb):
    """512^3 workload's spectrum shape at 256^3 (R = 20, p = 10, q = 3: b = 120, 100 noise
    eigenvalues in a narrow cluster): FP64 path at the FP64 bar, mixed path within 1%."""
    wl = synth.config_large(size=256)
    _, ref = _check_fp64(rb, wl)
    e_ref = np.sqrt(max(ref["x_norm2"] - ref["core_norm2"], 0.0))
    x = torch.from_numpy(wl.x).cuda()
    out = rb.rbki_tucker(x, wl.ranks, wl.p, wl.q, wl.seed, prec="bf16")
    e = _err_from_norms(out["norms"])
    assert np.isfinite(e) and abs(e - e_ref) <= 0.01 * e_ref


def test_tucker_fp64_gram_path_equals_tsvd(rb):
    g = synth.rng(7)
    x = synth.gaussian_tucker(g, 3, 10, 3) + 0.3 * g.standard_normal((10, 10, 10))
    wl = synth.Workload("tiny", np.ascontiguousarray(x), None, [3, 3, 3], 2, 1, 11)
    out, ref = _check_fp64(rb, wl)
    ts = rbki.tsvd(x, [3, 3, 3])
    for n in range(3):
        assert metrics.max_principal_sine(ts["factors"][n], out["factors"][n].cpu().numpy()) <= 1e-12


def test_tucker_mixed_small_config(rb):
    wl = synth.config_small_fp64(mc=0)
    ref = rbki.rbki_tucker(wl.x, wl.ranks, wl.p, wl.q, wl.seed)
    x = torch.from_numpy(wl.x.astype(np.float32)).cuda()
    out = rb.rbki_tucker(x, wl.ranks, wl.p, wl.q, wl.seed, prec="bf16")
    torch.cuda.synchronize()
    err_ref = np.sqrt(ref["x_norm2"] - ref["core_norm2"])
    g = out["core"].cpu().numpy()
    us = [f.cpu().numpy() for f in out["factors"]]
    err = metrics.fnorm(wl.x - rbki.reconstruct(g, us))
    assert abs(err - err_ref) <= 0.01 * err_ref
    assert abs(_err_from_norms(out["norms"]) - err_ref) <= 0.01 * err_ref
    assert out["info"].cpu().numpy()[6] == 0


def _bf16(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).bfloat16().double().numpy()


@pytest.mark.parametrize("dims", [(200, 48, 40), (64, 64, 64), (512, 24, 136), (96, 136, 16), (8, 384, 24)])
@pytest.mark.parametrize("s", [12, 30])
def test_krylov_product_tensor_core(rb, dims, s):
    """tcgen05 Krylov step vs FP64 products of the BF16-exact operands.
    split: Q and Y carried as hi + lo BF16 pairs -> FP32-level agreement; plain BF16: the
    reference rounds Q and Y to BF16 the same way (a few elements may round the other way)."""
    g = np.random.default_rng(sum(dims) * 7 + s)
    x = g.standard_normal(dims).astype(np.float32)
    xt = torch.from_numpy(x).cuda()
    xb = _bf16(x)
    for mode in range(len(dims)):
        if dims[mode] > 512:
            continue
        q = g.standard_normal((dims[mode], s))
        qt = torch.from_numpy(q).cuda()
        xn = unfold(xb, mode)
        exact = xn @ (xn.T @ q)
        p_split = rb.rbki_krylov_product(xt, mode, qt, prec=-1).cpu().numpy()
        rel = np.linalg.norm(p_split - exact) / np.linalg.norm(exact)
        assert rel < 2e-5, (mode, rel)
        p = rb.rbki_krylov_product(xt, mode, qt, prec="bf16").cpu().numpy()
        yb = _bf16(xn.T @ _bf16(q))
        want = xn @ yb
        rel = np.linalg.norm(p - want) / np.linalg.norm(want)
        assert rel < 2e-3, (mode, rel)
        assert np.linalg.norm(p - exact) / np.linalg.norm(exact) < 1e-2


@pytest.mark.parametrize("dims,mode", [((1024, 96, 40), 0), ((40, 1024, 48), 1), ((48, 40, 1024), 2),
                                       ((1000, 64, 24), 0)])
@pytest.mark.parametrize("s", [12, 50])
def test_krylov_product_two_pass(rb, dims, mode, s):
    """I_n > 640: the fused tensor-core step does not fit, so the step runs in two passes
    (Y = X^T Q written as BF16 operand images, then P = X Y on the sketch kernel); same
    rounding as the fused plain-BF16 step."""
    g = np.random.default_rng(sum(dims) + s)
    x = g.standard_normal(dims).astype(np.float32)
    xt = torch.from_numpy(x).cuda()
    xb = _bf16(x)
    q = g.standard_normal((dims[mode], s))
    p = rb.rbki_krylov_product(xt, mode, torch.from_numpy(q).cuda(), prec="bf16").cpu().numpy()
    xn = unfold(xb, mode)
    want = xn @ _bf16(xn.T @ _bf16(q))
    assert np.linalg.norm(p - want) / np.linalg.norm(want) < 2e-3


@pytest.mark.parametrize("dims,core", [((3, 40, 50), (2, 5, 6)), ((40, 50, 5), (5, 6, 3)),
                                       ((30, 8, 20, 7), (4, 3, 4, 2)), ((16, 16, 16, 16), (8, 8, 8, 8))])
def test_tucker_short_gram_modes(rb, dims, core):
    """Gram-path modes with I_n <= 8 (<= 16 on the mixed path) run on the one-pass short-mode
    Gram kernel (both layouts: C > 1 and the last mode); FP64 bar, and the mixed path within 1%."""
    wl = synth.config_small_fp64(mc=12, dims=dims, core=core, p=3, q=1)
    _, ref = _check_fp64(rb, wl)
    e_ref = np.sqrt(max(ref["x_norm2"] - ref["core_norm2"], 0.0))
    out = rb.rbki_tucker(torch.from_numpy(wl.x.astype(np.float32)).cuda(), wl.ranks, wl.p, wl.q, wl.seed,
                         prec="bf16")
    assert abs(_err_from_norms(out["norms"]) - e_ref) <= 0.01 * e_ref


def test_host_io_async_in_flight(rb):
    """RBKI_FLAG_HOST_IO | RBKI_FLAG_ASYNC: calls on separate streams return at once and
    overlap; after a synchronisation every host output equals the synchronous call's."""
    wl = synth.config_small_fp64(mc=13, dims=(48, 40, 56), core=(5, 4, 6), p=3, q=2)
    xh = torch.from_numpy(wl.x).pin_memory()
    ref = rb.rbki_tucker(xh, wl.ranks, wl.p, wl.q, wl.seed, prec="fp64", flags=rb.FLAG_HOST_IO)
    streams = [torch.cuda.Stream() for _ in range(3)]
    outs = [rb.rbki_tucker(xh, wl.ranks, wl.p, wl.q, wl.seed, prec="fp64", flags=rb.FLAG_HOST_IO | rb.FLAG_ASYNC,
                           stream=s) for s in streams]
    torch.cuda.synchronize()
    for o in outs:
        assert torch.equal(o["core"], ref["core"])
        for a, b in zip(o["factors"], ref["factors"]):
            assert torch.equal(a, b)
        assert torch.equal(o["norms"], ref["norms"])


def test_first_core_product_rank_above_32(rb):
    """R = 40 on the first contracted mode: the split (hi + lo) factor no longer fits one
    tensor-core pass, so the product runs as two plain passes summed; the mixed result's
    error stays within 1% of the oracle's and within 1e-3 of the FP64 path's."""
    wl = synth.config_small_fp64(mc=14, dims=(256, 64, 48), core=(40, 16, 16), p=4, q=1)
    ref = rbki.rbki_tucker(wl.x, wl.ranks, wl.p, wl.q, wl.seed)
    e_ref = np.sqrt(max(ref["x_norm2"] - ref["core_norm2"], 0.0))
    x = torch.from_numpy(wl.x.astype(np.float32)).cuda()
    mixed = rb.rbki_tucker(x, wl.ranks, wl.p, wl.q, wl.seed, prec="bf16")
    f64 = rb.rbki_tucker(x, wl.ranks, wl.p, wl.q, wl.seed, prec="fp64")
    torch.cuda.synchronize()
    em, e64 = _err_from_norms(mixed["norms"]), _err_from_norms(f64["norms"])
    assert abs(em - e_ref) <= 0.01 * e_ref
    assert abs(em - e64) <= 1e-3 * e64
    assert mixed["info"].cpu().numpy()[6] == 0
