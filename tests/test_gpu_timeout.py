"""Bounded device waits run out without a fault.  A planted stall (the MMA-issuing thread waits
on a barrier that nothing arrives at, for 2 ms) makes the tensor-core kernels
take their abort path: every role leaves its loop, the copies and MMAs already issued are
waited for, tensor memory is freed and the error word is set.  The call must report
RBKI_E_TIMEOUT with P all NaN, and the next regular call on the same context must succeed
and be correct (the context stays usable, no tensor memory leaks)."""
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


def _want(x, mode, q):
    xn = x.double().movedim(mode, 0).reshape(x.shape[mode], -1)
    return xn @ (xn.T @ q)


# (dims, mode, s): the pipelined fused kernel in both layouts (C-fast, I-fast), the
# split variant, and the two-pass step of a long mode (the first pass carries the stall)
CASES = [((96, 64, 80), 0, 30, "bf16"), ((96, 64, 80), 2, 12, "bf16"), ((64, 72, 48), 1, 20, -1),
         ((1024, 8, 16), 0, 24, "bf16")]


@pytest.mark.parametrize("dims,mode,s,prec", CASES)
def test_expired_wait_reports_timeout_and_next_call_succeeds(rb, dims, mode, s, prec):
    from paper_2211_14828_gb300 import _binding as B
    g = torch.Generator().manual_seed(7)
    x = torch.randn(dims, generator=g).cuda().bfloat16()
    q = torch.linalg.qr(torch.randn(dims[mode], s, generator=g, dtype=torch.float64))[0].cuda()
    status, p = rb.rbki_diag_krylov_stall(x, mode, q, prec=prec, wait_us=2000)
    assert status == B.E_TIMEOUT
    assert torch.isnan(p).all()
    # the context is still usable and the same step is correct right after
    for _ in range(2):
        p2 = rb.rbki_krylov_product(x, mode, q, prec=prec)
        torch.cuda.synchronize()
        want = _want(x, mode, q)
        assert not torch.isnan(p2).any()
        # Y = X^T Q is rounded to BF16 before the second product (unit roundoff 2^-8); the
        # split variant carries it as hi + lo (about 2^-16)
        assert float((p2 - want).norm() / want.norm()) <= (2.0 ** -8 if prec == "bf16" else 2e-5)


def test_batched_gram_pass_expired_wait_reports_timeout(rb):
    """The tensor-core Gram pass of rbki_tucker_batched: every CTA's planted wait runs out,
    the wave reports E_TIMEOUT with info[2N] set per item, and the next wave on the same
    context is correct and bitwise equal to a wave run before the stall."""
    import synth
    from paper_2211_14828_gb300 import _binding as B
    reqs = synth.serve_stream(n_requests=4, seed=808, dim_lo=24, dim_hi=96, rank_lo=3, rank_hi=10)
    xs = [synth.serve_request_device(r)[0] for r in reqs]           # BF16: the tensor-core pass
    ranks, qs, seeds = [r["ranks"] for r in reqs], [r["q"] for r in reqs], [r["seed"] for r in reqs]
    before = rb.rbki_tucker_batched(xs, ranks, 5, qs, seeds)
    torch.cuda.synchronize()
    status, outs = rb.rbki_diag_batched_stall(xs, ranks, 5, qs, seeds, wait_us=2000)
    assert status == B.E_TIMEOUT
    for o, x in zip(outs, xs):
        assert int(o["info"].cpu()[2 * x.dim()]) == 1
    for _ in range(2):
        after = rb.rbki_tucker_batched(xs, ranks, 5, qs, seeds)
        torch.cuda.synchronize()
        for a, b, x in zip(before, after, xs):
            assert int(b["info"].cpu()[2 * x.dim()]) == 0
            assert torch.equal(a["core"], b["core"]) and torch.equal(a["norms"], b["norms"])
            for fa, fb in zip(a["factors"], b["factors"]):
                assert torch.equal(fa, fb)
