"""The Krylov step without a workspace (rbki_krylov_product_noalloc), for callers that cannot
allocate device memory.  Its scratch is a fixed device array inside the library, shared by
every call, so two calls in a row must each match the regular entry point (which uses a
caller-provided workspace).  Collected last on purpose: it must pass both alone in a fresh
process and after every other test."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def rb():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2211_14828_gb300 as rb
    rb.lib()
    return rb


def _stored(x, prec):
    """X in the product precision the step streams (BF16 for "bf16" and the split variant)."""
    return x.half() if prec in ("fp16", -2) else x.bfloat16()


@pytest.mark.parametrize("prec", ["bf16", "fp16", -1])
def test_noalloc_matches_workspace_entry_point_twice(rb, prec):
    g = np.random.default_rng(2024)
    dims = (96, 64, 80)
    x = _stored(torch.from_numpy(g.standard_normal(dims).astype(np.float32)).cuda(), prec)
    for call, (mode, s) in enumerate([(0, 30), (2, 12)]):       # two calls in a row
        q = torch.from_numpy(g.standard_normal((dims[mode], s))).cuda()
        p_ws = rb.rbki_krylov_product(x, mode, q, prec=prec)
        p_na = rb.rbki_krylov_product_noalloc(x, mode, q, prec=prec)
        torch.cuda.synchronize()
        a, b = p_ws.cpu().numpy(), p_na.cpu().numpy()
        assert np.isfinite(b).all()
        np.testing.assert_array_equal(b, a, err_msg=f"call {call}")    # same kernels, same order


def test_noalloc_largest_scratch_shape_twice(rb):
    """The shape that comes closest to filling the static array: I_n = 512 with the split
    operand at s = 32 (N = 64): 152 x 512 x 64 FP32 partials + a 64 KB image on GB300."""
    g = np.random.default_rng(77)
    x = torch.from_numpy(g.standard_normal((512, 64, 64)).astype(np.float32)).cuda().bfloat16()
    for call in range(2):
        q = torch.from_numpy(g.standard_normal((512, 32))).cuda()
        p_ws = rb.rbki_krylov_product(x, 0, q, prec=-1)
        p_na = rb.rbki_krylov_product_noalloc(x, 0, q, prec=-1)
        torch.cuda.synchronize()
        a, b = p_ws.cpu().numpy(), p_na.cpu().numpy()
        assert np.isfinite(b).all()
        np.testing.assert_array_equal(b, a, err_msg=f"call {call}")


def test_noalloc_rejects_unsupported_and_wrong_dtype(rb):
    from paper_2211_14828_gb300 import _binding as B
    x = torch.zeros((8, 8, 8), dtype=torch.float32, device="cuda")
    q = torch.zeros((8, 4), dtype=torch.float64, device="cuda")
    with pytest.raises(rb.RbkiError) as e:
        rb.rbki_krylov_product_noalloc(x, 0, q, prec="bf16")          # X not stored in BF16
    assert e.value.status == B.E_INVAL
    tall = torch.zeros((600, 8, 16), dtype=torch.bfloat16, device="cuda")
    qt = torch.zeros((600, 32), dtype=torch.float64, device="cuda")
    with pytest.raises(rb.RbkiError) as e:
        rb.rbki_krylov_product_noalloc(tall, 0, qt, prec=-1)           # tile exceeds shared memory
    assert e.value.status == B.E_UNSUPPORTED
