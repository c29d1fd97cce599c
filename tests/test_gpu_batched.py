"""GPU tests of the batched small-decomposition path (rbki_tucker_batched): many rBKI-TK
requests of uneven shapes, ranks and depths as one wave of shared launches.

* Parity: every item's reconstruction error within 1% of the FP64 oracle's (the mixed-path
  bar), orthonormal factors with the sign rule, paths (Krylov / Gram) as the oracle's, Ritz
  values within the BF16 rounding of the products.
* Independence: an item's outputs are bitwise the same in a wave of many and alone.
* At the served stream's full sizes (I_n up to 256, R_n up to 32, q = 3): the error within
  1% of the single-call mixed path's, orthonormal factors.
* Launches: a wave's launch count does not grow with the number of requests.
* Unsupported requests are refused, not run some other way."""
import numpy as np
import pytest

import synth
from oracle import rbki

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def rb():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2211_14828_gb300 as rb
    rb.lib()
    return rb


def _reqs(n, seed, **kw):
    return synth.serve_stream(n_requests=n, seed=seed, **kw)


def _err(out):
    nr = out["norms"].cpu().numpy()
    return float(np.sqrt(max(nr[0] - nr[1], 0.0))), float(nr[0])


def _check_factor(u):
    u = u.cpu().numpy()
    assert np.linalg.norm(u.T @ u - np.eye(u.shape[1])) <= 1e-12
    for k in range(u.shape[1]):
        i = int(np.argmax(np.abs(u[:, k])))
        assert u[i, k] > 0.0


def _run(rb, xs, reqs):
    return rb.rbki_tucker_batched(xs, [r["ranks"] for r in reqs], reqs[0]["p"], [r["q"] for r in reqs],
                                  [r["seed"] + 17 for r in reqs], prec="bf16")


def test_batched_matches_oracle(rb):
    # small shapes so that the oracle finishes quickly; dims down to 8 put some modes on the
    # Gram path (b = (R + p)(q + 1) >= I_n); half the inputs are FP32 (rounded as read)
    reqs = _reqs(10, 314, dim_lo=8, dim_hi=72, rank_lo=2, rank_hi=10)
    wls = [synth.serve_request_tensor(r, dtype=np.float64) for r in reqs]
    xs = [torch.from_numpy(wl.x).cuda().float() if k % 2 else torch.from_numpy(wl.x).cuda().bfloat16()
          for k, wl in enumerate(wls)]
    outs = _run(rb, xs, reqs)
    torch.cuda.synchronize()
    n_gram = 0
    for wl, x, out, r in zip(wls, xs, outs, reqs):
        ref = rbki.rbki_tucker(np.asarray(x.double().cpu().numpy()), wl.ranks, wl.p, wl.q, wl.seed)
        e, x2 = _err(out)
        e_ref = float(np.sqrt(max(ref["x_norm2"] - ref["core_norm2"], 0.0)))
        assert abs(x2 - ref["x_norm2"]) <= 1e-12 * ref["x_norm2"]
        assert abs(e - e_ref) <= 0.01 * e_ref, (r, e, e_ref)
        info = out["info"].cpu().numpy()
        N = x.dim()
        for n in range(N):
            _check_factor(out["factors"][n])
            gram = ref["path"][n] == "gram"
            n_gram += int(gram)
            assert info[N + n] == int(gram)
            lam, lam_ref = out["eigvals"][n].cpu().numpy(), np.asarray(ref["eigvals"][n])
            assert np.max(np.abs(lam - lam_ref)) <= 1e-2 * lam_ref[0]
        assert info[2 * N] == 0
        assert out["q_used"].cpu().numpy().tolist() == [0 if ref["path"][n] == "gram" else r["q"] for n in range(N)]
    assert n_gram >= 1


def test_batched_item_independent_of_wave(rb):
    reqs = _reqs(12, 2718, dim_lo=16, dim_hi=96, rank_lo=3, rank_hi=16)
    xs = [synth.serve_request_device(r)[0] for r in reqs]
    wave = _run(rb, xs, reqs)
    alone = [_run(rb, [x], [r])[0] for x, r in zip(xs, reqs)]
    torch.cuda.synchronize()
    for a, b in zip(wave, alone):
        for k in ("core", "norms", "info", "q_used"):
            assert torch.equal(a[k], b[k]), k
        for fa, fb in zip(a["factors"], b["factors"]):
            assert torch.equal(fa, fb)
        for ea, eb in zip(a["eigvals"], b["eigvals"]):
            assert torch.equal(ea, eb)


def test_batched_fullsize_served_requests(rb):
    # the stream's largest shapes: I_n = 256, R_n = 32, q = 3 (eigenproblems of 148), next to
    # small ones in the same wave
    reqs = [dict(id=0, dims=[256, 256, 256], ranks=[32, 32, 32], p=5, q=3, snr_db=10.0, seed=4242),
            dict(id=1, dims=[256, 200, 48], ranks=[32, 7, 20], p=5, q=2, snr_db=5.0, seed=4243),
            dict(id=2, dims=[33, 256, 129], ranks=[4, 32, 13], p=5, q=1, snr_db=25.0, seed=4244)]
    xs = [synth.serve_request_device(r)[0] for r in reqs]
    outs = _run(rb, xs, reqs)
    for x, r, out in zip(xs, reqs, outs):
        single = rb.rbki_tucker(x, r["ranks"], r["p"], r["q"], r["seed"] + 17, prec="bf16")
        torch.cuda.synchronize()
        e, x2 = _err(out)
        e1, x21 = _err(single)
        assert abs(x2 - x21) <= 1e-12 * x21
        assert abs(e - e1) <= 0.01 * e1, (r["dims"], e, e1)
        for u in out["factors"]:
            _check_factor(u)


def test_batched_launches_do_not_grow_with_the_wave(rb):
    reqs = _reqs(40, 99, dim_lo=24, dim_hi=64, rank_lo=3, rank_hi=8)   # 120 mode items: one pack
    xs = [synth.serve_request_device(r)[0] for r in reqs]
    _run(rb, xs[:1], reqs[:1])      # one-time setup (shared-memory opt-in)
    torch.cuda.synchronize()
    l0 = rb.rbki_kernel_launches()
    _run(rb, xs[:4], reqs[:4])
    l1 = rb.rbki_kernel_launches()
    _run(rb, xs, reqs)
    l2 = rb.rbki_kernel_launches()
    torch.cuda.synchronize()
    small, big = l1 - l0, l2 - l1
    # a wave costs a fixed schedule of launches (plus a few per kernel variant its items
    # need): 40 requests cost about what 4 cost, against ~250 launches per single call
    assert big <= small + 30, (small, big)
    assert big / len(reqs) <= 5.0, big


def test_batched_refuses_unsupported(rb):
    from paper_2211_14828_gb300 import _binding as B
    r = _reqs(1, 5)[0]
    x = synth.serve_request_device(r)[0]
    for kw in (dict(prec="fp64"), dict(flags=rb.FLAG_SPLIT), dict(flags=rb.FLAG_SEQUENTIAL)):
        with pytest.raises(rb.RbkiError) as e:
            rb.rbki_tucker_batched([x.double() if kw.get("prec") == "fp64" else x], [r["ranks"]], 5, r["q"], [1],
                                   **kw)
        assert e.value.status == B.E_UNSUPPORTED
    big = torch.zeros((300, 8, 8), dtype=torch.bfloat16, device="cuda")
    with pytest.raises(rb.RbkiError) as e:
        rb.rbki_tucker_batched([big], [[4, 4, 4]], 2, 1, [1])
    assert e.value.status == B.E_UNSUPPORTED


def test_autotuned_table_keeps_parity_and_independence(rb, tmp_path):
    cand = {2, 4, 8, 16, 32, 64}
    try:
        rb.rbki_wave_autotune()
        t = rb.rbki_wave_tune_table()
        assert set(t["gram"]) <= cand and set(t["ttm"]) <= cand
        rb.rbki_wave_tune_save(tmp_path / "tune.txt")
        reqs = _reqs(6, 77, dim_lo=8, dim_hi=64, rank_lo=2, rank_hi=8)
        wls = [synth.serve_request_tensor(r, dtype=np.float64) for r in reqs]
        xs = [torch.from_numpy(wl.x).cuda().bfloat16() for wl in wls]
        wave = _run(rb, xs, reqs)
        alone = [_run(rb, [x], [r])[0] for x, r in zip(xs, reqs)]
        torch.cuda.synchronize()
        for wl, x, a, b in zip(wls, xs, wave, alone):
            assert torch.equal(a["core"], b["core"]) and torch.equal(a["norms"], b["norms"])
            ref = rbki.rbki_tucker(np.asarray(x.double().cpu().numpy()), wl.ranks, wl.p, wl.q, wl.seed)
            e, _ = _err(a)
            e_ref = float(np.sqrt(max(ref["x_norm2"] - ref["core_norm2"], 0.0)))
            assert abs(e - e_ref) <= 0.01 * e_ref
        # the saved table reproduces the tuned one
        rb.rbki_wave_tune_reset()
        rb.rbki_wave_tune_load(tmp_path / "tune.txt")
        assert rb.rbki_wave_tune_table() == t
    finally:
        rb.rbki_wave_tune_reset()


def test_captured_wave_replays(rb):
    reqs = _reqs(8, 55, dim_lo=16, dim_hi=80, rank_lo=3, rank_hi=10)
    xs = [synth.serve_request_device(r)[0] for r in reqs]
    ranks, qs, seeds = [r["ranks"] for r in reqs], [r["q"] for r in reqs], [r["seed"] + 17 for r in reqs]
    plan = rb.BatchedPlan(xs, ranks, 5, qs, seeds)
    try:
        for scale in (1.0, -0.5):
            with torch.no_grad():
                for x in xs:
                    x.mul_(scale)               # refilled in place: the plan reads the same buffers
            l0 = rb.rbki_kernel_launches()
            outs = plan.launch()
            l1 = rb.rbki_kernel_launches()
            ref = rb.rbki_tucker_batched(xs, ranks, 5, qs, seeds)
            torch.cuda.synchronize()
            assert 50 <= l1 - l0 <= 150          # one graph launch carries the whole wave
            for a, b in zip(outs, ref):
                for k in ("core", "norms", "info"):
                    assert torch.equal(a[k], b[k]), k
                for fa, fb in zip(a["factors"], b["factors"]):
                    assert torch.equal(fa, fb)
    finally:
        plan.close()
