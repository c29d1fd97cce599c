"""GPU parity of the divide-and-conquer decomposition (Sec. 4.1.2) and of batches of
independent decompositions, through the C ABI.

* rbki_split_mode: bit-exact against NumPy slicing (every dtype, vector and scalar paths);
* rbki_tucker_batch: every item bit-identical to its own rbki_tucker call (mixed flags);
* divide-and-conquer against oracle.divide: FP64 bar per part and on the summed error,
  mixed path within 1%, on a video-shaped tensor split along the frame mode."""
import numpy as np
import pytest

import synth
from oracle import divide, metrics

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def rb():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2211_14828_gb300 as rb
    rb.lib()
    return rb


def _err2(norms):
    n = norms.cpu().numpy()
    return max(n[0] - n[1], 0.0)


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32, torch.bfloat16])
@pytest.mark.parametrize("shape,mode,parts", [((6, 5, 256), 2, 4), ((7, 33, 9), 1, 5), ((250, 3, 8), 0, 5),
                                              ((4, 6, 10, 3), 3, 3)])
def test_split_bit_exact(rb, dtype, shape, mode, parts):
    g = torch.Generator().manual_seed(1)
    x = torch.randn(shape, generator=g, dtype=torch.float64).to(dtype).cuda()
    got = rb.rbki_split_mode(x, mode, parts)
    torch.cuda.synchronize()
    for k, part in enumerate(got):
        lo, hi = k * shape[mode] // parts, (k + 1) * shape[mode] // parts
        assert torch.equal(part, x.narrow(mode, lo, hi - lo).contiguous())


def test_batch_items_equal_single_calls(rb):
    g = synth.rng(5)
    xs_np = [g.standard_normal(s) for s in ((40, 36, 48), (64, 64, 64), (30, 20, 50, 12))]
    ranks = [[5, 4, 6], [8, 8, 8], [3, 4, 5, 2]]
    xs = [torch.from_numpy(x).cuda() for x in xs_np]
    for prec, flags in (("fp64", 0), ("bf16", 0), ("fp64", 8)):
        outs = rb.rbki_tucker_batch(xs, ranks, 3, 2, [11, 12, 13], prec=prec, flags=flags)
        torch.cuda.synchronize()
        for k, x in enumerate(xs):
            one = rb.rbki_tucker(x, ranks[k], 3, 2, 11 + k, prec=prec, flags=flags)
            torch.cuda.synchronize()
            assert torch.equal(outs[k]["core"], one["core"]), (prec, flags, k)
            for a, b in zip(outs[k]["factors"], one["factors"]):
                assert torch.equal(a, b)


def test_divide_and_conquer_fp64_matches_oracle(rb):
    wl = synth.config_small_fp64(mc=11, dims=(48, 40, 96), core=(5, 4, 6), p=3, q=2)
    parts, ranks = 3, [[5, 4, 3]] * 3
    ref = divide.divide_and_conquer(wl.x, 2, parts, ranks, wl.p, wl.q, wl.seed)
    _, outs = rb.rbki_divide_and_conquer(torch.from_numpy(wl.x).cuda(), 2, parts, ranks, wl.p, wl.q, wl.seed,
                                         prec="fp64")
    torch.cuda.synchronize()
    err2 = 0.0
    for k in range(parts):
        r = ref["parts"][k]
        for n in range(3):
            assert metrics.max_principal_sine(r["factors"][n], outs[k]["factors"][n].cpu().numpy()) <= 1e-10
        err2 += _err2(outs[k]["norms"])
    assert abs(err2 - ref["err2"]) <= 1e-12 * ref["err2"] + 1e-13 * ref["x_norm2"]


def test_divide_and_conquer_video_shape_mixed(rb):
    """A 256 x 256 x 3 x 64 video-shaped tensor (DCT factors, 5 dB) split into 4 parts of 16
    frames along the frame mode; ranks 20 x 20 x 3 x 4 per part (the one-pass ratio 16/64)."""
    g = synth.rng(77)
    dims, core = (256, 256, 3, 64), (20, 20, 3, 16)
    c = g.standard_normal(core)
    facs = [synth.dct_factor(i, r) for i, r in zip(dims, core)]
    x = synth.add_noise_snr(synth.tucker_full(c, facs), 5.0, g, dtype=np.float32)
    parts, ranks = 4, [[20, 20, 3, 4]] * 4
    ref = divide.divide_and_conquer(x, 3, parts, ranks, 10, 2, 3)
    _, outs = rb.rbki_divide_and_conquer(torch.from_numpy(x).cuda(), 3, parts, ranks, 10, 2, 3, prec="bf16")
    torch.cuda.synchronize()
    err2 = sum(_err2(o["norms"]) for o in outs)
    assert abs(np.sqrt(err2) - np.sqrt(ref["err2"])) <= 0.01 * np.sqrt(ref["err2"])


def test_batch_validation(rb):
    x = torch.zeros((8, 8, 8), dtype=torch.float64, device="cuda")
    with pytest.raises(rb.RbkiError):
        rb.rbki_split_mode(x, 1, 9)
    with pytest.raises(rb.RbkiError):
        rb.rbki_tucker_batch([x], [[9, 2, 2]], 1, 1, [0], prec="fp64")
