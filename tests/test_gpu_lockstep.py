"""GPU tests of the lockstep modes (the default for two or more Krylov-path modes with
b <= 192): every FP64 stage is one batched launch for all modes, and an orthonormalisation
pass is two launches (the chunk partials with the reduction, the Pythagorean Gram matrix and
the deflating Cholesky done by the CTA that finishes last, then the block update).

* Bit for bit the per-mode kernels' results (RBKI_FLAG_SERIAL_MODES): FP64 and mixed, with
  and without deflation (an exactly low-rank tensor whose Krylov blocks become dependent),
  order 3 and 4, and the 512^3 bench shape.
* Repeated calls on the same workspace give the same results (the tickets of the fused
  passes are left at 0).
* The 512^3 decomposition takes at most 100 launches."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def rb():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2211_14828_gb300 as rb
    rb.lib()
    return rb


def _same(a, b):
    for k in ("core", "norms", "info", "q_used"):
        assert torch.equal(a[k], b[k]), k
    for fa, fb in zip(a["factors"], b["factors"]):
        assert torch.equal(fa, fb)
    for ea, eb in zip(a["eigvals"], b["eigvals"]):
        assert torch.equal(ea, eb)


def _cases():
    yield "noisy64", synth.config_small_fp64(mc=3)
    yield "exact64", synth.config_small_fp64(mc=4, snr_db=None)     # rank 8 < b = 36: deflation
    yield "ragged", synth.config_small_fp64(mc=5, dims=(72, 40, 56), core=(6, 5, 7))
    yield "order4", synth.config_small_fp64(mc=6, dims=(24, 20, 28, 18), core=(3, 4, 3, 2), p=3, q=1)


@pytest.mark.parametrize("prec", ["fp64", "bf16"])
@pytest.mark.parametrize("case", [c for c, _ in _cases()])
def test_lockstep_equals_per_mode_kernels(rb, case, prec):
    wl = dict(_cases())[case]
    x = torch.from_numpy(wl.x).cuda()
    xin = x if prec == "fp64" else x.float()
    lock = rb.rbki_tucker(xin, wl.ranks, wl.p, wl.q, wl.seed, prec=prec)
    serial = rb.rbki_tucker(xin, wl.ranks, wl.p, wl.q, wl.seed, prec=prec, flags=rb.FLAG_SERIAL_MODES)
    torch.cuda.synchronize()
    _same(lock, serial)
    if case == "exact64" and prec == "fp64":
        # the dependent Krylov directions were dropped (in BF16 the rounding of the products
        # leaves components far above the deflation threshold)
        kept = lock["info"].cpu().numpy()[:3]
        assert (kept < 36).all(), kept
    # the same workspace again: the fused passes left their tickets at 0
    rb.rbki_tucker(xin, wl.ranks, wl.p, wl.q, wl.seed, prec=prec, workspace=lock["workspace"], out=lock)
    torch.cuda.synchronize()
    _same(lock, serial)


def test_lockstep_512_bitwise_and_launches(rb):
    wl = synth.config_large(size=512)
    x = torch.from_numpy(wl.x).cuda()
    lock = rb.rbki_tucker(x, wl.ranks, wl.p, wl.q, wl.seed, prec="bf16")
    torch.cuda.synchronize()
    l0 = rb.rbki_kernel_launches()
    rb.rbki_tucker(x, wl.ranks, wl.p, wl.q, wl.seed, prec="bf16", workspace=lock["workspace"], out=lock)
    launches = rb.rbki_kernel_launches() - l0
    serial = rb.rbki_tucker(x, wl.ranks, wl.p, wl.q, wl.seed, prec="bf16", flags=rb.FLAG_SERIAL_MODES)
    torch.cuda.synchronize()
    _same(lock, serial)
    assert launches <= 100, launches
