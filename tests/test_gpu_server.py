"""GPU tests of the served stream (rbki_server_*): results in the mix equal the same
request run alone, bit for bit; memory admission under a small budget; cancellation;
requests refused at submission; and parity of served results with the oracle."""
import time

import numpy as np
from parity_bars import err_matches
import pytest

import synth
from oracle import rbki
from oracle.metrics import max_principal_sine

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def rb():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2211_14828_gb300 as rb
    rb.lib()
    return rb


def _requests(n=12, seed=77):
    """Small served-stream requests (shapes, ranks, q, SNR from the stream recipe)."""
    reqs = synth.serve_stream(n_requests=n, seed=seed, dim_lo=24, dim_hi=96, rank_lo=3, rank_hi=12)
    out = []
    for i, r in enumerate(reqs):
        wl = synth.serve_request_tensor(r, dtype=np.float64 if i % 3 == 0 else np.float32)
        prec = "fp64" if i % 3 == 0 else "bf16"
        out.append((wl, prec))
    return out


def _device_input(wl, prec):
    x = torch.from_numpy(np.ascontiguousarray(wl.x)).cuda()
    return x if prec == "fp64" else x.bfloat16()


def _wait(srv, tickets, timeout=120.0):
    done = {}
    t0 = time.time()
    while len(done) < len(tickets) and time.time() - t0 < timeout:
        for t in tickets:
            if t not in done:
                ok, st, lat = srv.poll(t)
                if ok:
                    done[t] = (st, lat)
        time.sleep(0.001)
    assert len(done) == len(tickets), "requests did not finish"
    return done


def _same(a, b):
    for k in ("core", "norms", "info"):
        assert torch.equal(a[k], b[k]), k
    for fa, fb in zip(a["factors"], b["factors"]):
        assert torch.equal(fa, fb)
    for ea, eb in zip(a["eigvals"], b["eigvals"]):
        assert torch.equal(ea, eb)


def _alone(rb, x, wl, prec, waves=True):
    """The request alone through the path the server gives it: the batched path (a wave of
    one) for BF16 requests when waves are on, rbki_tucker otherwise."""
    if waves and prec != "fp64":
        return rb.rbki_tucker_batched([x], [wl.ranks], wl.p, wl.q, [wl.seed], prec=prec)[0]
    return rb.rbki_tucker(x, wl.ranks, wl.p, wl.q, wl.seed, prec=prec)


@pytest.mark.parametrize("wave_threads", [2, 0])
def test_results_in_the_mix_equal_results_alone(rb, wave_threads):
    reqs = _requests()
    xs = [_device_input(wl, prec) for wl, prec in reqs]
    alone = [_alone(rb, x, wl, prec, wave_threads > 0) for x, (wl, prec) in zip(xs, reqs)]
    torch.cuda.synchronize()
    with rb.RbkiServer(0, mem_budget=1 << 30, max_slots=4, wave_threads=wave_threads) as srv:
        tickets, outs = [], []
        for x, (wl, prec) in zip(xs, reqs):
            t, o = srv.submit(x, wl.ranks, wl.p, wl.q, wl.seed, prec=prec)
            tickets.append(t)
            outs.append(o)
        done = _wait(srv, tickets)
        for t in tickets:
            assert done[t][0] == 0 and done[t][1] > 0
        srv.drain(10.0)
    for a, b in zip(alone, outs):
        _same(a, b)


def test_served_results_match_the_oracle(rb):
    reqs = _requests(n=6, seed=91)
    with rb.RbkiServer(0, mem_budget=1 << 30, max_slots=3) as srv:
        subs = [srv.submit(_device_input(wl, prec), wl.ranks, wl.p, wl.q, wl.seed, prec=prec) for wl, prec in reqs]
        done = _wait(srv, [t for t, _ in subs])
        assert all(v[0] == 0 for v in done.values())
    for (wl, prec), (_, out) in zip(reqs, subs):
        ref = rbki.rbki_tucker(np.asarray(wl.x, dtype=np.float64), wl.ranks, wl.p, wl.q, wl.seed)
        n = out["norms"].cpu().numpy()
        e = np.sqrt(max(n[0] - n[1], 0.0))
        e_ref = np.sqrt(max(ref["x_norm2"] - ref["core_norm2"], 0.0))
        if prec == "fp64":
            for k, u in enumerate(out["factors"]):
                assert max_principal_sine(ref["factors"][k], u.cpu().numpy()) <= 1e-10
            assert err_matches(e, e_ref, ref["x_norm2"])
        else:
            assert abs(e - e_ref) <= 0.01 * e_ref


def test_admission_under_a_small_budget(rb):
    """A budget that holds about one request at a time: every request still completes,
    in the mix, with the same results as alone; a request larger than the budget is
    refused at submission."""
    reqs = _requests(n=6, seed=5)
    xs = [_device_input(wl, prec) for wl, prec in reqs]
    need = [rb.rbki_tucker_workspace(x, wl.ranks, wl.p, wl.q, wl.seed, prec) if prec == "fp64" else
            rb.rbki_tucker_batched_workspace([x], [wl.ranks], wl.p, wl.q, [wl.seed], prec)
            for x, (wl, prec) in zip(xs, reqs)]
    budget = int(max(need) * 1.2)
    alone = [_alone(rb, x, wl, prec) for x, (wl, prec) in zip(xs, reqs)]
    torch.cuda.synchronize()
    with rb.RbkiServer(0, mem_budget=budget, max_slots=4) as srv:
        subs = [srv.submit(x, wl.ranks, wl.p, wl.q, wl.seed, prec=prec) for x, (wl, prec) in zip(xs, reqs)]
        done = _wait(srv, [t for t, _ in subs])
        assert all(v[0] == 0 for v in done.values())
        for a, (_, b) in zip(alone, subs):
            _same(a, b)
        big = torch.zeros((200, 200, 200), dtype=torch.bfloat16, device="cuda")
        with pytest.raises(rb.RbkiError) as ei:
            srv.submit(big, [20, 20, 20], 10, 3, 1, prec="bf16")
        assert ei.value.status == rb._binding.E_NOMEM


def test_cancel_invalid_and_unknown(rb):
    reqs = _requests(n=8, seed=13)
    with rb.RbkiServer(0, mem_budget=1 << 30, max_slots=1) as srv:
        subs = [srv.submit(_device_input(wl, prec), wl.ranks, wl.p, wl.q, wl.seed, prec=prec) for wl, prec in reqs]
        last = subs[-1][0]
        srv.cancel(last)                       # one slot: the last request is still queued
        # an invalid request (rank above the dimension) is refused at submission
        x = torch.zeros((8, 8, 8), dtype=torch.float64, device="cuda")
        with pytest.raises(rb.RbkiError) as ei:
            srv.submit(x, [9, 2, 2], 1, 1, 0, prec="fp64")
        assert ei.value.status == rb._binding.E_INVAL
        done = _wait(srv, [t for t, _ in subs])
        assert done[last][0] == rb._binding.E_CANCELLED
        assert all(done[t][0] == 0 for t, _ in subs[:-1])
        with pytest.raises(rb.RbkiError) as ei:
            srv.poll(last)                     # retired by its terminal poll
        assert ei.value.status == rb._binding.E_NOTFOUND
