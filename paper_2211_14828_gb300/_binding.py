"""Thin ctypes binding of librbki.so (argument marshalling only).

Every computation runs in the library's CUDA kernels; PyTorch only provides device
memory and the current stream.  The functions keep the C entry points' names.
If the shared library has not been built, loading fails loudly: there is no CPU
fallback."""
from __future__ import annotations

import ctypes as C
import os
from typing import Dict, Optional, Sequence

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "librbki.so")
MAX_ORDER = 8

OK, PENDING, W_DEFLATED = 0, 1, 2
E_INVAL, E_NOMEM, E_CUDA, E_UNSUPPORTED, E_TIMEOUT, E_BUSY, E_CANCELLED, E_NOTFOUND = range(-1, -9, -1)
F64, F32, BF16, F16 = 0, 1, 2, 3
PREC_FP64, PREC_BF16, PREC_FP16 = 0, 1, 2
FLAG_HOST_IO, FLAG_SPLIT, FLAG_SERIAL_MODES, FLAG_SEQUENTIAL, FLAG_POWER, FLAG_ADAPTIVE_Q, FLAG_TR_SVD, FLAG_ASYNC = \
    1, 2, 4, 8, 16, 32, 64, 128
FLAG_REFINE_FP32 = 256
SERVER_WAVE_THREADS, SERVER_WAVE_MAX = 4, 32   # rbki_server_create's batched-path workers and wave size


class rbki_tensor(C.Structure):
    _fields_ = [("order", C.c_int32), ("dtype", C.c_int32), ("dims", C.c_int64 * MAX_ORDER),
                ("data", C.c_void_p)]


class rbki_params(C.Structure):
    _fields_ = [("ranks", C.c_int32 * MAX_ORDER), ("p", C.c_int32), ("q", C.c_int32),
                ("seed", C.c_uint64), ("prec", C.c_int32), ("flags", C.c_uint32), ("omega", C.c_double),
                ("q_tol", C.c_double)]


class rbki_tucker_out(C.Structure):
    _fields_ = [("core", C.c_void_p), ("factors", C.c_void_p * MAX_ORDER),
                ("eigvals", C.c_void_p * MAX_ORDER), ("norms", C.c_void_p), ("info", C.c_void_p),
                ("q_used", C.c_void_p)]


class RbkiError(RuntimeError):
    def __init__(self, status: int, what: str, detail: str):
        super().__init__(f"{what}: status {status} ({detail})")
        self.status = status


_lib = None


def lib():
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with __graft_entry__.build() "
                               "(there is no CPU fallback)")
        L = C.CDLL(LIB_PATH)
        st = C.c_int32
        vp = C.c_void_p
        sz = C.POINTER(C.c_size_t)
        sig = {
            "rbki_tucker_workspace": (st, [vp, vp, sz]),
            "rbki_tucker": (st, [vp, vp, vp, C.c_size_t, vp, vp]),
            "rbki_htr_workspace": (st, [vp, vp, vp, sz]),
            "rbki_htr": (st, [vp, vp, vp, vp, C.c_int32, C.c_double, vp, vp, vp, vp, C.c_size_t, vp]),
            "rbki_server_create": (st, [C.c_int32, C.c_size_t, C.c_int32, C.POINTER(vp)]),
            "rbki_server_create_ex": (st, [C.c_int32, C.c_size_t, C.c_int32, C.c_int32, C.c_int32, C.POINTER(vp)]),
            "rbki_submit": (st, [vp, vp, vp, vp, vp, C.POINTER(C.c_uint64)]),
            "rbki_poll": (st, [vp, C.c_uint64, C.POINTER(C.c_int32), C.POINTER(C.c_double)]),
            "rbki_cancel": (st, [vp, C.c_uint64]),
            "rbki_server_drain": (st, [vp, C.c_double]),
            "rbki_server_destroy": (st, [vp]),
            "rbki_krylov_product": (st, [vp, C.c_int32, C.c_int32, vp, C.c_int32, vp, vp, C.c_size_t, vp]),
            "rbki_krylov_product_workspace": (st, [vp, C.c_int32, C.c_int32, C.c_int32, sz]),
            "rbki_mode_basis": (st, [vp, vp, C.c_int32, vp, vp, C.c_size_t, vp]),
            "rbki_krylov_product_noalloc": (st, [vp, C.c_int32, C.c_int32, vp, C.c_int32, vp, vp]),
            "rbki_diag_krylov_stall": (st, [vp, C.c_int32, C.c_int32, vp, C.c_int32, vp, vp, C.c_size_t,
                                            C.c_uint32, vp]),
            "rbki_syev": (st, [vp, C.c_int32, vp, vp, vp, C.c_size_t, vp]),
            "rbki_syev_workspace": (st, [C.c_int32, sz]),
            "rbki_sample_units": (st, [C.c_uint64, C.c_int32, C.c_int64, C.c_int64, vp, vp]),
            "rbki_tucker_batch_workspace": (st, [C.c_int32, vp, vp, sz]),
            "rbki_tucker_batch": (st, [C.c_int32, vp, vp, vp, C.c_size_t, vp, vp]),
            "rbki_tucker_batched_workspace": (st, [C.c_int32, vp, vp, sz]),
            "rbki_wave_autotune": (st, [vp]),
            "rbki_diag_batched_stall": (st, [C.c_int32, vp, vp, vp, C.c_size_t, vp, C.c_uint32, vp]),
            "rbki_batched_plan_create": (st, [C.c_int32, vp, vp, vp, C.c_size_t, vp, vp, C.POINTER(vp)]),
            "rbki_batched_plan_launch": (st, [vp, vp]),
            "rbki_batched_plan_destroy": (st, [vp]),
            "rbki_wave_tune_get": (st, [C.c_int32, C.c_int32, C.POINTER(C.c_int32)]),
            "rbki_wave_tune_reset": (st, []),
            "rbki_wave_tune_save": (st, [C.c_char_p]),
            "rbki_wave_tune_load": (st, [C.c_char_p]),
            "rbki_tucker_batched": (st, [C.c_int32, vp, vp, vp, C.c_size_t, vp, vp]),
            "rbki_split_mode": (st, [vp, C.c_int32, C.c_int32, vp, vp]),
            "rbki_status_str": (C.c_char_p, [C.c_int32]),
            "rbki_last_error": (C.c_char_p, []),
            "rbki_kernel_launches": (C.c_uint64, []),
            "rbki_profile_enable": (None, [C.c_int32]),
            "rbki_profile_read": (st, [C.c_int32, C.POINTER(C.c_uint64), C.POINTER(C.c_double)]),
            "rbki_profile_reset": (None, []),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def check(status: int, what: str) -> int:
    if status < 0:
        L = lib()
        raise RbkiError(status, what, f"{L.rbki_status_str(status).decode()}: "
                                      f"{L.rbki_last_error().decode()}")
    return status


# ---------------- marshalling helpers (torch is used for memory and streams only) ----------------
def _torch():
    import torch
    return torch


def dtype_code(t) -> int:
    torch = _torch()
    return {torch.float64: F64, torch.float32: F32, torch.bfloat16: BF16, torch.float16: F16}[t.dtype]


def prec_code(prec) -> int:
    """'fp64' | 'bf16' | 'fp16', or the C code; a negative code selects the split variant."""
    if isinstance(prec, int):
        return prec
    return {"fp64": PREC_FP64, "bf16": PREC_BF16, "fp16": PREC_FP16}[prec]


def make_tensor(x, host: bool = False) -> rbki_tensor:
    if not x.is_contiguous():
        raise ValueError("X must be C-contiguous")
    t = rbki_tensor()
    t.order = x.dim()
    t.dtype = dtype_code(x)
    for i, d in enumerate(x.shape):
        t.dims[i] = int(d)
    t.data = x.data_ptr()
    return t


def make_params(ranks: Sequence[int], p: int, q: int, seed: int, prec, flags: int = 0,
                omega: float = 0.0, q_tol: float = 0.0) -> rbki_params:
    """omega: column sampling rate of the Krylov construction (0 < omega < 1), else none;
    q_tol: fit-change threshold of FLAG_ADAPTIVE_Q."""
    prm = rbki_params()
    for i, r in enumerate(ranks):
        prm.ranks[i] = int(r)
    prm.p, prm.q, prm.seed, prm.prec, prm.flags = int(p), int(q), int(seed), prec_code(prec), int(flags)
    prm.omega = float(omega)
    prm.q_tol = float(q_tol)
    return prm


def stream_ptr(stream=None):
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def alloc_outputs(dims, ranks, device, host=False) -> Dict:
    torch = _torch()
    kw = dict(dtype=torch.float64, device="cpu" if host else device)
    if host:
        kw["pin_memory"] = True
    out = dict(core=torch.zeros(tuple(ranks), **kw),
               factors=[torch.zeros((int(d), int(r)), **kw) for d, r in zip(dims, ranks)],
               eigvals=[torch.zeros(int(r), **kw) for r in ranks],
               norms=torch.zeros(2, **kw))
    ikw = dict(dtype=torch.int32, device="cpu" if host else device)
    if host:
        ikw["pin_memory"] = True
    out["info"] = torch.zeros(2 * len(dims) + 1, **ikw)
    out["q_used"] = torch.zeros(len(dims), **ikw)
    return out


def make_out(o: Dict) -> rbki_tucker_out:
    s = rbki_tucker_out()
    s.core = o["core"].data_ptr()
    for i, f in enumerate(o["factors"]):
        s.factors[i] = f.data_ptr()
    for i, e in enumerate(o.get("eigvals") or []):
        s.eigvals[i] = e.data_ptr() if e is not None else None
    s.norms = o["norms"].data_ptr() if o.get("norms") is not None else None
    s.info = o["info"].data_ptr() if o.get("info") is not None else None
    s.q_used = o["q_used"].data_ptr() if o.get("q_used") is not None else None
    return s


# ---------------- entry points ----------------
def rbki_tucker_workspace(x, ranks, p, q, seed=0, prec="bf16", flags=0, omega=0.0, q_tol=0.0) -> int:
    n = C.c_size_t(0)
    t, prm = make_tensor(x), make_params(ranks, p, q, seed, prec, flags, omega, q_tol)
    check(lib().rbki_tucker_workspace(C.byref(t), C.byref(prm), C.byref(n)), "rbki_tucker_workspace")
    return int(n.value)


def rbki_tucker(x, ranks, p, q, seed, prec="bf16", flags=0, workspace=None, out=None, stream=None, omega=0.0,
                q_tol=0.0):
    """rBKI-TK (Algorithm 2).  x: torch tensor (CUDA, or pinned CPU with FLAG_HOST_IO).
    omega: column sampling rate of the Krylov construction (0 < omega < 1), else none;
    q_tol: fit-change threshold with FLAG_ADAPTIVE_Q (q is then the bound)."""
    torch = _torch()
    host = bool(flags & FLAG_HOST_IO)
    t, prm = make_tensor(x), make_params(ranks, p, q, seed, prec, flags, omega, q_tol)
    need = C.c_size_t(0)
    check(lib().rbki_tucker_workspace(C.byref(t), C.byref(prm), C.byref(need)), "rbki_tucker_workspace")
    dev = torch.device("cuda", torch.cuda.current_device()) if host else x.device
    if workspace is None or workspace.numel() < need.value:
        workspace = torch.empty(int(need.value), dtype=torch.uint8, device=dev)
    if out is None:
        out = alloc_outputs(x.shape, ranks, dev, host=host)
    o = make_out(out)
    check(lib().rbki_tucker(C.byref(t), C.byref(prm), C.c_void_p(workspace.data_ptr()),
                            C.c_size_t(workspace.numel()), C.byref(o), stream_ptr(stream)), "rbki_tucker")
    out["workspace"] = workspace
    return out


def rbki_split_mode(x, mode, parts, stream=None):
    """Consecutive parts of x along `mode` (part k: [floor(k I / K), floor((k+1) I / K))) as
    dense device tensors, copied by the library's split kernel."""
    torch = _torch()
    size = x.shape[mode]
    outs = []
    for k in range(parts):
        shape = list(x.shape)
        shape[mode] = (k + 1) * size // parts - k * size // parts
        outs.append(torch.empty(shape, dtype=x.dtype, device=x.device))
    ptrs = (C.c_void_p * parts)(*[o.data_ptr() for o in outs])
    check(lib().rbki_split_mode(C.byref(make_tensor(x)), int(mode), int(parts), ptrs, stream_ptr(stream)),
          "rbki_split_mode")
    return outs


def rbki_tucker_batch(xs, ranks, p, q, seeds, prec="bf16", flags=0, omega=0.0, q_tol=0.0, workspace=None,
                      outs=None, stream=None):
    """Independent rBKI-TK decompositions run concurrently (one call).  ranks[k], seeds[k]
    per item; returns the list of output dicts (the first also holds the workspace)."""
    torch = _torch()
    n = len(xs)
    ts = (rbki_tensor * n)(*[make_tensor(x) for x in xs])
    ps = (rbki_params * n)(*[make_params(ranks[k], p, q, seeds[k], prec, flags, omega, q_tol) for k in range(n)])
    need = C.c_size_t(0)
    check(lib().rbki_tucker_batch_workspace(n, ts, ps, C.byref(need)), "rbki_tucker_batch_workspace")
    if workspace is None or workspace.numel() < need.value:
        workspace = torch.empty(int(need.value), dtype=torch.uint8, device=xs[0].device)
    if outs is None:
        outs = [alloc_outputs(x.shape, ranks[k], x.device) for k, x in enumerate(xs)]
    os_ = (rbki_tucker_out * n)(*[make_out(o) for o in outs])
    check(lib().rbki_tucker_batch(n, ts, ps, C.c_void_p(workspace.data_ptr()), C.c_size_t(workspace.numel()),
                                  os_, stream_ptr(stream)), "rbki_tucker_batch")
    outs[0]["workspace"] = workspace
    return outs


class BatchedPlan:
    """A wave captured as a CUDA graph (rbki_batched_plan_*): refill the inputs in place and
    call launch(); the outputs land in `outs`.  Holds references to the inputs, outputs and
    workspace it is bound to."""

    def __init__(self, xs, ranks, p, qs, seeds, prec="bf16", flags=0, stream=None):
        torch = _torch()
        n = len(xs)
        qv = [int(qs)] * n if isinstance(qs, int) else [int(v) for v in qs]
        self.xs = xs
        ts = (rbki_tensor * n)(*[make_tensor(x) for x in xs])
        ps = (rbki_params * n)(*[make_params(ranks[k], p, qv[k], seeds[k], prec, flags) for k in range(n)])
        need = C.c_size_t(0)
        check(lib().rbki_tucker_batched_workspace(n, ts, ps, C.byref(need)), "rbki_tucker_batched_workspace")
        self.workspace = torch.empty(max(int(need.value), 1), dtype=torch.uint8, device=xs[0].device)
        self.outs = [alloc_outputs(x.shape, ranks[k], x.device) for k, x in enumerate(xs)]
        os_ = (rbki_tucker_out * n)(*[make_out(o) for o in self.outs])
        h = C.c_void_p()
        check(lib().rbki_batched_plan_create(n, ts, ps, C.c_void_p(self.workspace.data_ptr()),
                                             C.c_size_t(self.workspace.numel()), os_, stream_ptr(stream),
                                             C.byref(h)), "rbki_batched_plan_create")
        self._h = h

    def launch(self, stream=None):
        check(lib().rbki_batched_plan_launch(self._h, stream_ptr(stream)), "rbki_batched_plan_launch")
        return self.outs

    def close(self):
        if self._h:
            lib().rbki_batched_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def rbki_wave_autotune(stream=None):
    """Measures the batched path's work granularity on the device and keeps the fastest."""
    check(lib().rbki_wave_autotune(stream_ptr(stream)), "rbki_wave_autotune")


def rbki_wave_tune_table():
    """The current table: {"gram": [steps per bucket], "ttm": [...]} (buckets of 32 rows)."""
    out = {}
    for kind, name in enumerate(("gram", "ttm")):
        row = []
        for b in range(8):
            v = C.c_int32(0)
            check(lib().rbki_wave_tune_get(kind, b, C.byref(v)), "rbki_wave_tune_get")
            row.append(int(v.value))
        out[name] = row
    return out


def rbki_wave_tune_save(path):
    check(lib().rbki_wave_tune_save(str(path).encode()), "rbki_wave_tune_save")


def rbki_wave_tune_load(path):
    check(lib().rbki_wave_tune_load(str(path).encode()), "rbki_wave_tune_load")


def rbki_wave_tune_reset():
    check(lib().rbki_wave_tune_reset(), "rbki_wave_tune_reset")


def rbki_tucker_batched_workspace(xs, ranks, p, qs, seeds, prec="bf16", flags=0) -> int:
    """Workspace bytes of rbki_tucker_batched for these items."""
    n = len(xs)
    qv = [int(qs)] * n if isinstance(qs, int) else [int(v) for v in qs]
    ts = (rbki_tensor * n)(*[make_tensor(x) for x in xs])
    ps = (rbki_params * n)(*[make_params(ranks[k], p, qv[k], seeds[k], prec, flags) for k in range(n)])
    need = C.c_size_t(0)
    check(lib().rbki_tucker_batched_workspace(n, ts, ps, C.byref(need)), "rbki_tucker_batched_workspace")
    return int(need.value)


def rbki_tucker_batched(xs, ranks, p, qs, seeds, prec="bf16", flags=0, workspace=None, outs=None,
                        stream=None):
    """Many small rBKI-TK decompositions as one wave (rbki_tucker_batched): ranks[k], qs[k]
    (an int applies to all), seeds[k] per item.  Returns the list of output dicts (the first
    also holds the workspace)."""
    torch = _torch()
    n = len(xs)
    qv = [int(qs)] * n if isinstance(qs, int) else [int(v) for v in qs]
    ts = (rbki_tensor * n)(*[make_tensor(x) for x in xs])
    ps = (rbki_params * n)(*[make_params(ranks[k], p, qv[k], seeds[k], prec, flags) for k in range(n)])
    need = C.c_size_t(0)
    check(lib().rbki_tucker_batched_workspace(n, ts, ps, C.byref(need)), "rbki_tucker_batched_workspace")
    if workspace is None or workspace.numel() < need.value:
        workspace = torch.empty(max(int(need.value), 1), dtype=torch.uint8, device=xs[0].device)
    if outs is None:
        outs = [alloc_outputs(x.shape, ranks[k], x.device) for k, x in enumerate(xs)]
    os_ = (rbki_tucker_out * n)(*[make_out(o) for o in outs])
    check(lib().rbki_tucker_batched(n, ts, ps, C.c_void_p(workspace.data_ptr()), C.c_size_t(workspace.numel()),
                                    os_, stream_ptr(stream)), "rbki_tucker_batched")
    outs[0]["workspace"] = workspace
    return outs


def rbki_divide_and_conquer(x, mode, parts, ranks, p, q, seed, prec="bf16", flags=0, stream=None):
    """Divide-and-conquer decomposition along `mode`: split into `parts` consecutive parts,
    decompose them as one batch (part k with ranks[k] and seed + k).  Returns (parts, outs)."""
    xs = rbki_split_mode(x, mode, parts, stream=stream)
    outs = rbki_tucker_batch(xs, ranks, p, q, [seed + k for k in range(parts)], prec=prec, flags=flags,
                             stream=stream)
    return xs, outs


def rbki_htr(x, tucker_ranks, p, q, seed, tr_ranks, tr_init, maxit=20, tol=1e-3, prec="fp64", flags=0,
             workspace=None, tucker_out=None, stream=None, omega=0.0):
    """rBKI-TK-TR (Algorithm 3).  tr_init: list of float64 CUDA tensors (r_{n-1}, R_n, r_n), or
    None with FLAG_TR_SVD (TR-SVD instead of TR-ALS).
    Returns dict(cores=[(r_{n-1}, I_n, r_n)], fits=(maxit,) NaN after the stop, tucker=...)."""
    torch = _torch()
    N = x.dim()
    t, prm = make_tensor(x), make_params(tucker_ranks, p, q, seed, prec, flags, omega)
    trr = (C.c_int32 * 8)(*[int(r) for r in tr_ranks])
    need = C.c_size_t(0)
    check(lib().rbki_htr_workspace(C.byref(t), C.byref(prm), trr, C.byref(need)), "rbki_htr_workspace")
    if workspace is None or workspace.numel() < need.value:
        workspace = torch.empty(int(need.value), dtype=torch.uint8, device=x.device)
    init = [z.contiguous() for z in tr_init] if tr_init is not None else []
    init_p = (C.c_void_p * 8)(*[z.data_ptr() for z in init]) if tr_init is not None else None
    cores = [torch.zeros((int(tr_ranks[(n + N - 1) % N]), int(x.shape[n]), int(tr_ranks[n])),
                         dtype=torch.float64, device=x.device) for n in range(N)]
    cores_p = (C.c_void_p * 8)(*[z.data_ptr() for z in cores])
    fits = torch.zeros(int(maxit), dtype=torch.float64, device=x.device)
    if tucker_out is None:
        tucker_out = alloc_outputs(x.shape, tucker_ranks, x.device)
    o = make_out(tucker_out)
    check(lib().rbki_htr(C.byref(t), C.byref(prm), trr, init_p, C.c_int32(int(maxit)), C.c_double(float(tol)),
                         cores_p, C.c_void_p(fits.data_ptr()), C.byref(o), C.c_void_p(workspace.data_ptr()),
                         C.c_size_t(workspace.numel()), stream_ptr(stream)), "rbki_htr")
    return dict(cores=cores, fits=fits, tucker=tucker_out, workspace=workspace)


def rbki_krylov_product(x, mode: int, q_mat, prec="fp64", workspace=None, stream=None):
    """P = X_(n) (X_(n)^T Q) (Algorithm 1 step 3), Q: (I_n, s) float64 CUDA tensor."""
    torch = _torch()
    t = make_tensor(x)
    s = int(q_mat.shape[1])
    need = C.c_size_t(0)
    check(lib().rbki_krylov_product_workspace(C.byref(t), mode, prec_code(prec), s, C.byref(need)),
          "rbki_krylov_product_workspace")
    if workspace is None or workspace.numel() < need.value:
        workspace = torch.empty(int(need.value), dtype=torch.uint8, device=x.device)
    P = torch.empty((x.shape[mode], s), dtype=torch.float64, device=x.device)
    q_c = q_mat.contiguous()
    check(lib().rbki_krylov_product(C.byref(t), mode, prec_code(prec), C.c_void_p(q_c.data_ptr()), s,
                                    C.c_void_p(P.data_ptr()), C.c_void_p(workspace.data_ptr()),
                                    C.c_size_t(workspace.numel()), stream_ptr(stream)), "rbki_krylov_product")
    return P


def rbki_diag_krylov_stall(x, mode: int, q_mat, prec="bf16", wait_us: int = 2000, stream=None):
    """The Krylov step with a planted stall that nothing releases (bounded by wait_us):
    exercises the kernels' abort path.  Returns (status, P); the expected status is E_TIMEOUT
    with P all NaN."""
    torch = _torch()
    t = make_tensor(x)
    s = int(q_mat.shape[1])
    need = C.c_size_t(0)
    check(lib().rbki_krylov_product_workspace(C.byref(t), mode, prec_code(prec), s, C.byref(need)),
          "rbki_krylov_product_workspace")
    workspace = torch.empty(int(need.value), dtype=torch.uint8, device=x.device)
    P = torch.empty((x.shape[mode], s), dtype=torch.float64, device=x.device)
    q_c = q_mat.contiguous()
    status = lib().rbki_diag_krylov_stall(C.byref(t), mode, prec_code(prec), C.c_void_p(q_c.data_ptr()), s,
                                          C.c_void_p(P.data_ptr()), C.c_void_p(workspace.data_ptr()),
                                          C.c_size_t(workspace.numel()), C.c_uint32(wait_us), stream_ptr(stream))
    return int(status), P


def rbki_diag_batched_stall(xs, ranks, p, qs, seeds, prec="bf16", wait_us: int = 2000, stream=None):
    """A wave with a planted stall in its tensor-core Gram pass (bounded by wait_us): exercises
    that kernel's abort path.  Returns (status, outs); the expected status is E_TIMEOUT with
    info[2N] set on the items that took the tensor-core pass."""
    torch = _torch()
    n = len(xs)
    qv = [int(qs)] * n if isinstance(qs, int) else [int(v) for v in qs]
    ts = (rbki_tensor * n)(*[make_tensor(x) for x in xs])
    ps = (rbki_params * n)(*[make_params(ranks[k], p, qv[k], seeds[k], prec, 0) for k in range(n)])
    need = C.c_size_t(0)
    check(lib().rbki_tucker_batched_workspace(n, ts, ps, C.byref(need)), "rbki_tucker_batched_workspace")
    workspace = torch.empty(max(int(need.value), 1), dtype=torch.uint8, device=xs[0].device)
    outs = [alloc_outputs(x.shape, ranks[k], x.device) for k, x in enumerate(xs)]
    os_ = (rbki_tucker_out * n)(*[make_out(o) for o in outs])
    status = lib().rbki_diag_batched_stall(n, ts, ps, C.c_void_p(workspace.data_ptr()),
                                           C.c_size_t(workspace.numel()), os_, C.c_uint32(wait_us),
                                           stream_ptr(stream))
    return int(status), outs


def rbki_krylov_product_noalloc(x, mode: int, q_mat, prec="bf16", stream=None):
    """Krylov step without a workspace (static device scratch inside the library).
    x must already be BF16 (prec 'bf16') or FP16 (prec 'fp16'); a negative prec code selects
    the split variant.  Returns P = X_(n) (X_(n)^T Q) as an (I_n, s) float64 CUDA tensor."""
    torch = _torch()
    t = make_tensor(x)
    s = int(q_mat.shape[1])
    P = torch.empty((x.shape[mode], s), dtype=torch.float64, device=x.device)
    q_c = q_mat.contiguous()
    check(lib().rbki_krylov_product_noalloc(C.byref(t), mode, prec_code(prec), C.c_void_p(q_c.data_ptr()), s,
                                            C.c_void_p(P.data_ptr()), stream_ptr(stream)),
          "rbki_krylov_product_noalloc")
    return P


def rbki_mode_basis(x, ranks, p, q, seed, mode, prec="fp64", stream=None, omega=0.0):
    """Algorithm 1 basis Q = [Q_0..Q_q] for one mode (I_n x S(q+1), zero deflated columns)."""
    torch = _torch()
    t, prm = make_tensor(x), make_params(ranks, p, q, seed, prec, 0, omega)
    need = C.c_size_t(0)
    check(lib().rbki_tucker_workspace(C.byref(t), C.byref(prm), C.byref(need)), "rbki_tucker_workspace")
    ws = torch.empty(int(need.value), dtype=torch.uint8, device=x.device)
    s = min(ranks[mode] + p, x.shape[mode])
    Q = torch.empty((x.shape[mode], s * (q + 1)), dtype=torch.float64, device=x.device)
    check(lib().rbki_mode_basis(C.byref(t), C.byref(prm), mode, C.c_void_p(Q.data_ptr()),
                                C.c_void_p(ws.data_ptr()), C.c_size_t(ws.numel()), stream_ptr(stream)),
          "rbki_mode_basis")
    return Q


def rbki_sample_units(seed, mode, n_units, kept, device=None, stream=None):
    """Kept units of partial column sampling (int32 device tensor, ascending)."""
    torch = _torch()
    units = torch.empty(int(kept), dtype=torch.int32, device=device or "cuda")
    check(lib().rbki_sample_units(int(seed), int(mode), int(n_units), int(kept), C.c_void_p(units.data_ptr()),
                                  stream_ptr(stream)), "rbki_sample_units")
    return units


def rbki_syev(a, stream=None):
    """Eigen-decomposition of a symmetric FP64 matrix: (w descending, V columns)."""
    torch = _torch()
    n = int(a.shape[0])
    need = C.c_size_t(0)
    check(lib().rbki_syev_workspace(n, C.byref(need)), "rbki_syev_workspace")
    ws = torch.empty(int(need.value), dtype=torch.uint8, device=a.device)
    w = torch.empty(n, dtype=torch.float64, device=a.device)
    V = torch.empty((n, n), dtype=torch.float64, device=a.device)
    a_c = a.contiguous()
    check(lib().rbki_syev(C.c_void_p(a_c.data_ptr()), n, C.c_void_p(w.data_ptr()), C.c_void_p(V.data_ptr()),
                          C.c_void_p(ws.data_ptr()), C.c_size_t(ws.numel()), stream_ptr(stream)), "rbki_syev")
    return w, V


PENDING, E_CANCELLED, E_NOTFOUND, E_NOMEM, E_INVAL = 1, -7, -8, -2, -1


class RbkiServer:
    """Served stream (rbki_server_*): continuous batching with device-memory admission.
    Holds references to each request's input and outputs until its terminal poll."""

    def __init__(self, device: int = 0, mem_budget: int = 1 << 30, max_slots: int = 4,
                 wave_threads: int = SERVER_WAVE_THREADS, wave_max: int = SERVER_WAVE_MAX):
        """wave_threads workers serve the requests rbki_tucker_batched supports in waves of up
        to wave_max (0 workers: every request on the max_slots slots, one rbki_tucker each)."""
        h = C.c_void_p()
        check(lib().rbki_server_create_ex(int(device), C.c_size_t(int(mem_budget)), int(max_slots), int(wave_threads),
                                          int(wave_max), C.byref(h)), "rbki_server_create_ex")
        self._h = h
        self._live = {}

    def submit(self, x, ranks, p, q, seed, prec="bf16", out=None, after_stream=None, flags=0, omega=0.0,
               q_tol=0.0):
        """Queues a request; its kernels wait for the work already queued on `after_stream`
        (default: torch's current stream, where x and out were made)."""
        torch = _torch()
        t, prm = make_tensor(x), make_params(ranks, p, q, seed, prec, flags, omega, q_tol)
        if out is None:
            out = alloc_outputs(x.shape, ranks, x.device)
        o = make_out(out)
        tk = C.c_uint64(0)
        st = after_stream if after_stream is not None else torch.cuda.current_stream()
        # the legacy default stream has handle 0, which the C ABI reads as "no stream to wait
        # for": pass its explicit handle (cudaStreamLegacy) instead
        handle = st.cuda_stream or 0x1
        check(lib().rbki_submit(self._h, C.byref(t), C.byref(prm), C.byref(o), C.c_void_p(handle), C.byref(tk)),
              "rbki_submit")
        self._live[tk.value] = (x, out)
        return tk.value, out

    def poll(self, ticket):
        """(done, status, latency_s): done False while the request is queued or running."""
        res = C.c_int32(0)
        lat = C.c_double(0.0)
        st = lib().rbki_poll(self._h, C.c_uint64(ticket), C.byref(res), C.byref(lat))
        if st == PENDING:
            return False, PENDING, None
        check(st, "rbki_poll")
        self._live.pop(ticket, None)
        return True, int(res.value), float(lat.value)

    def cancel(self, ticket):
        check(lib().rbki_cancel(self._h, C.c_uint64(ticket)), "rbki_cancel")

    def drain(self, timeout_s: float = -1.0):
        return check(lib().rbki_server_drain(self._h, C.c_double(timeout_s)), "rbki_server_drain")

    def close(self):
        if self._h is not None:
            check(lib().rbki_server_destroy(self._h), "rbki_server_destroy")
            self._h = None
            self._live.clear()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


PROF_KRYLOV, PROF_SKETCH, PROF_GRAM, PROF_TTM, PROF_STAGE, PROF_SAMPLE = range(6)


def rbki_profile_enable(on: bool = True) -> None:
    lib().rbki_profile_enable(1 if on else 0)


def rbki_profile_reset() -> None:
    lib().rbki_profile_reset()


def rbki_profile_read(cls: int):
    """(launch count, total ms) of kernel class `cls` since the last reset."""
    n = C.c_uint64(0)
    ms = C.c_double(0)
    check(lib().rbki_profile_read(cls, C.byref(n), C.byref(ms)), "rbki_profile_read")
    return int(n.value), float(ms.value)


def rbki_kernel_launches() -> int:
    return int(lib().rbki_kernel_launches())
