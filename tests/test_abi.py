"""CPU checks of the C ABI: the library builds, loads and exports every symbol that
include/rbki.h declares; argument validation needs no GPU."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    from paper_2211_14828_gb300 import _build
    import paper_2211_14828_gb300 as rb
    if not os.path.exists(rb.LIB_PATH):
        _build.build()
    return rb.lib()


def _declared():
    txt = open(os.path.join(ROOT, "include", "rbki.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(rbki_[a-z_0-9]+)\s*\(", txt)))


def test_header_symbols_exported(L):
    names = _declared()
    assert len(names) >= 15
    for n in names:
        assert hasattr(L, n), n


def test_status_strings(L):
    assert L.rbki_status_str(0) == b"ok"
    assert L.rbki_status_str(-2).startswith(b"out of memory")


def test_validation_without_gpu(L):
    import torch
    import paper_2211_14828_gb300 as rb
    from paper_2211_14828_gb300 import _binding as B
    x = torch.zeros((8, 9, 10), dtype=torch.float32)
    assert rb.rbki_tucker_workspace(x, [2, 3, 4], 2, 1, prec="bf16") > 0
    with pytest.raises(rb.RbkiError) as e:
        rb.rbki_tucker_workspace(x, [2, 30, 4], 2, 1)        # R > I
    assert e.value.status == B.E_INVAL
    with pytest.raises(rb.RbkiError):
        rb.rbki_tucker_workspace(x, [2, 3, 4], -1, 1)        # p < 0
    t = B.make_tensor(x)
    t.order = 9
    n = ctypes.c_size_t(0)
    prm = B.make_params([1] * 8, 0, 0, 0, "fp64")
    assert L.rbki_tucker_workspace(ctypes.byref(t), ctypes.byref(prm), ctypes.byref(n)) == B.E_INVAL
    # a call with a too-small workspace is rejected before any device work
    t = B.make_tensor(x)
    prm = B.make_params([2, 3, 4], 2, 1, 0, "fp64")
    out = B.rbki_tucker_out()
    out.core = 16
    for i in range(3):
        out.factors[i] = 16
    st = L.rbki_tucker(ctypes.byref(t), ctypes.byref(prm), ctypes.c_void_p(16), ctypes.c_size_t(8),
                       ctypes.byref(out), None)
    assert st == B.E_NOMEM


def test_server_argument_checks_without_gpu(L):
    """Server entry points reject bad arguments before touching a device."""
    h = ctypes.c_void_p()
    assert L.rbki_server_create(0, ctypes.c_size_t(1 << 20), 0, ctypes.byref(h)) == -1      # max_slots < 1
    assert L.rbki_server_create(0, ctypes.c_size_t(16), 2, ctypes.byref(h)) == -1           # budget too small
    res = ctypes.c_int32(0)
    lat = ctypes.c_double(0)
    assert L.rbki_poll(None, ctypes.c_uint64(1), ctypes.byref(res), ctypes.byref(lat)) == -1
    assert L.rbki_cancel(None, ctypes.c_uint64(1)) == -1
    assert L.rbki_server_drain(None, ctypes.c_double(0.0)) == -1
    assert L.rbki_server_destroy(None) == -1


def test_sequential_flag_without_gpu(L):
    """The sequentially truncated reading adds two buffers of the largest Y_n to the
    workspace; the step-level basis call (defined on X) refuses the flag."""
    import torch
    import paper_2211_14828_gb300 as rb
    from paper_2211_14828_gb300 import _binding as B
    x = torch.zeros((64, 48, 40), dtype=torch.float64)
    ranks = [5, 6, 7]
    ws = rb.rbki_tucker_workspace(x, ranks, 2, 1, prec="fp64")
    ws_seq = rb.rbki_tucker_workspace(x, ranks, 2, 1, prec="fp64", flags=rb.FLAG_SEQUENTIAL)
    assert ws_seq >= 2 * 5 * 48 * 40 * 8
    assert ws_seq < ws + 2 * 5 * 48 * 40 * 8 + (1 << 20)
    t = B.make_tensor(x)
    prm = B.make_params(ranks, 2, 1, 0, "fp64", rb.FLAG_SEQUENTIAL)
    st = L.rbki_mode_basis(ctypes.byref(t), ctypes.byref(prm), 0, ctypes.c_void_p(16), ctypes.c_void_p(16),
                           ctypes.c_size_t(1 << 30), None)
    assert st == B.E_INVAL


def test_flag_and_argument_validation_without_gpu(L):
    """The option checks of rbki_params and the new entry points reject bad arguments on
    the host, before any device work."""
    import torch
    import paper_2211_14828_gb300 as rb
    from paper_2211_14828_gb300 import _binding as B
    x = torch.zeros((32, 24, 40), dtype=torch.float32)
    ranks = [4, 4, 4]
    bad = [
        dict(omega=float("nan")),                                   # E_INVAL
        dict(flags=rb.FLAG_ADAPTIVE_Q | rb.FLAG_POWER),            # E_INVAL
        dict(flags=rb.FLAG_ADAPTIVE_Q, q_tol=-1.0),                 # E_INVAL
        dict(flags=rb.FLAG_ADAPTIVE_Q | rb.FLAG_SEQUENTIAL),       # E_UNSUPPORTED
        dict(flags=rb.FLAG_ADAPTIVE_Q, omega=0.5),                  # E_UNSUPPORTED
    ]
    for kw in bad:
        with pytest.raises(rb.RbkiError) as e:
            rb.rbki_tucker_workspace(x, ranks, 2, 1, 0, "bf16", kw.get("flags", 0), kw.get("omega", 0.0),
                                     kw.get("q_tol", 0.0))
        assert e.value.status in (B.E_INVAL, B.E_UNSUPPORTED)
    # valid combinations size a workspace
    assert rb.rbki_tucker_workspace(x, ranks, 2, 1, 0, "bf16", rb.FLAG_POWER | rb.FLAG_SEQUENTIAL, 0.3) > 0
    assert rb.rbki_tucker_workspace(x, ranks, 2, 3, 0, "fp64", rb.FLAG_ADAPTIVE_Q, 0.0, 1e-3) > 0
    # sampling grows the workspace by the sample buffer only where a mode is sampled
    w0 = rb.rbki_tucker_workspace(x, ranks, 2, 1, 0, "fp64")
    w1 = rb.rbki_tucker_workspace(x, ranks, 2, 1, 0, "fp64", 0, 0.5)
    assert w1 > 0 and w0 > 0
    # the unit choice and the split refuse bad counts before launching anything
    assert L.rbki_sample_units(0, 0, 10, 11, ctypes.c_void_p(16), None) == B.E_INVAL
    assert L.rbki_sample_units(0, 0, 0, 0, ctypes.c_void_p(16), None) == B.E_INVAL
    t = B.make_tensor(x)
    dst = (ctypes.c_void_p * 4)(16, 16, 16, 16)
    assert L.rbki_split_mode(ctypes.byref(t), 1, 25, dst, None) == B.E_INVAL      # parts > I
    assert L.rbki_split_mode(ctypes.byref(t), 3, 2, dst, None) == B.E_INVAL       # mode out of range
    # batches refuse host buffers
    ts = (B.rbki_tensor * 1)(B.make_tensor(x))
    ps = (B.rbki_params * 1)(B.make_params(ranks, 2, 1, 0, "fp64", rb.FLAG_HOST_IO))
    n = ctypes.c_size_t(0)
    assert L.rbki_tucker_batch_workspace(1, ts, ps, ctypes.byref(n)) == B.E_UNSUPPORTED
