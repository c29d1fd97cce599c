"""Seeded synthetic inputs shared by the CUDA path's tests/bench and by the oracle.

This module only *makes data*: Tucker and tensor-ring test tensors, additive
Gaussian noise at a prescribed SNR, the power-functional tensor, and the random
initial tensor-ring cores that TR-ALS starts from.  It holds none of the
rBKI-TK arithmetic (no sketch, Krylov step, orthonormalisation, eigensolve or
TTM of the method), so that neither the CUDA path nor the oracle depends on
the other through it.

Workload recipes follow the paper's experiments:
  * Gaussian Tucker data, core and factors i.i.d. N(0,1)  (Sec. 4.1.1, "Gaussian random data")
  * power-functional data x = (sum_k i_k^p)^(-1/p), p = 10 (Sec. 4.1.1, Eq. "eq:function")
  * noise lambda*N scaled so 20 log10(|X|/|lambda N|) = SNR exactly (Eq. "eq:SNR")
  * video-shaped and TR-shaped stand-ins for the YUV / COIL-100 / CIFAR-10 data
    that are not available here (Sec. 4.1.2, Sec. 4.2).
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Sequence

import numpy as np

__all__ = [
    "rng", "haar_factor", "dct_factor", "tucker_full", "tr_full",
    "add_noise_snr", "power_functional", "gaussian_tucker",
    "Workload", "config_small_fp64", "config_large", "config_video",
    "config_htr", "serve_stream", "serve_request_tensor", "serve_request_device", "tr_init_cores",
]


def rng(seed: int) -> np.random.Generator:
    """PCG64 generator for a seed (all inputs in this project are seeded)."""
    return np.random.Generator(np.random.PCG64(int(seed)))


def haar_factor(g: np.random.Generator, rows: int, cols: int) -> np.ndarray:
    """Haar-distributed orthonormal rows x cols matrix: QR of a Gaussian with diag(R) > 0."""
    a = g.standard_normal((rows, cols))
    q, r = np.linalg.qr(a)
    s = np.sign(np.diag(r))
    s[s == 0] = 1.0
    return q * s[None, :]


def dct_factor(rows: int, cols: int) -> np.ndarray:
    """First `cols` orthonormal DCT-II basis vectors of length `rows` (smooth factors)."""
    i = np.arange(rows)[:, None] + 0.5
    k = np.arange(cols)[None, :]
    m = np.cos(np.pi * i * k / rows) * math.sqrt(2.0 / rows)
    m[:, 0] = 1.0 / math.sqrt(rows)
    return m


def tucker_full(core: np.ndarray, factors: Sequence[np.ndarray], dtype=np.float64) -> np.ndarray:
    """Dense tensor of the Tucker model core x_1 U1 x_2 U2 ... (data construction only)."""
    t = np.asarray(core, dtype=dtype)
    for n, u in enumerate(factors):
        t = np.moveaxis(np.tensordot(np.asarray(u, dtype=dtype), t, axes=(1, n)), 0, n)
    return np.ascontiguousarray(t)


def tr_full(cores: Sequence[np.ndarray]) -> np.ndarray:
    """Dense tensor of a tensor ring with cores (r_{k-1}, I_k, r_k), ring closed by r_0 = r_N."""
    t = cores[0]                                   # (r0, I1, r1)
    for c in cores[1:]:
        t = np.tensordot(t, c, axes=(t.ndim - 1, 0))  # (r0, I1..Ik, rk)
    # close the ring: trace over first and last rank index
    return np.ascontiguousarray(np.trace(t, axis1=0, axis2=t.ndim - 1))


def add_noise_snr(x: np.ndarray, snr_db: float, g: np.random.Generator,
                  dtype=None) -> np.ndarray:
    """x + lambda*N with N ~ N(0,1) i.i.d. and lambda fixed by the realised norms so that
    20*log10(|x|_F / |lambda N|_F) == snr_db  (Eq. "eq:SNR")."""
    dtype = dtype or x.dtype
    noise = g.standard_normal(x.shape, dtype=np.float32 if dtype == np.float32 else np.float64)
    nx = float(np.linalg.norm(x.ravel().astype(np.float64)))
    nn = float(np.linalg.norm(noise.ravel().astype(np.float64)))
    lam = nx / (nn * 10.0 ** (snr_db / 20.0))
    out = x.astype(dtype, copy=True)
    out += (lam * noise).astype(dtype, copy=False)
    return out


def power_functional(order: int, size: int, p: float = 10.0) -> np.ndarray:
    """x_{i1..iN} = (i1^p + ... + iN^p)^(-1/p), 1-based indices (Eq. "eq:function")."""
    idx = np.arange(1, size + 1, dtype=np.float64) ** p
    acc = np.zeros((size,) * order)
    for n in range(order):
        shape = [1] * order
        shape[n] = size
        acc = acc + idx.reshape(shape)
    return acc ** (-1.0 / p)


def gaussian_tucker(g: np.random.Generator, order: int, size: int, rank: int) -> np.ndarray:
    """Gaussian Tucker data: core and (non-orthonormal) factors i.i.d. N(0,1) (Sec. 4.1.1)."""
    core = g.standard_normal((rank,) * order)
    facs = [g.standard_normal((size, rank)) for _ in range(order)]
    return tucker_full(core, facs)


@dataclasses.dataclass
class Workload:
    """One decomposition problem: noisy input, clean tensor, and method parameters."""
    name: str
    x: np.ndarray                       # the (noisy) tensor to decompose, C-order
    clean: Optional[np.ndarray]         # noise-free tensor (reference for Fit / RErr), or None
    ranks: List[int]
    p: int
    q: int
    seed: int                           # seed of the sketching matrices Omega
    true_factors: Optional[List[np.ndarray]] = None
    tr_ranks: Optional[List[int]] = None
    tr_init: Optional[List[np.ndarray]] = None


def config_small_fp64(mc: int = 0, dims=(64, 64, 64), core=(8, 8, 8), snr_db: Optional[float] = 20.0,
                      p: int = 4, q: int = 2) -> Workload:
    """64^3 FP64: Gaussian 8^3 core x three Haar 64x8 factors + noise at 20 dB; R=(8,8,8), p=4, q=2."""
    g = rng(1001 + mc)
    c = g.standard_normal(core)
    facs = [haar_factor(g, i, r) for i, r in zip(dims, core)]
    clean = tucker_full(c, facs)
    x = clean if snr_db is None else add_noise_snr(clean, snr_db, g)
    return Workload("tucker64_fp64", np.ascontiguousarray(x), clean, list(core), p, q, 42 + mc, facs)


def config_large(mc: int = 0, size: int = 512, rank: int = 20, snr_db: Optional[float] = 10.0,
                 p: int = 10, q: int = 3, dtype=np.float32) -> Workload:
    """512^3 FP32: superdiagonal core g_kkk = k^-1/2 (power-law mode spectra) x Haar factors
    + noise at 10 dB; R=(20,20,20), p=10, q=3."""
    g = rng(1002 + mc)
    core = np.zeros((rank,) * 3)
    for k in range(rank):
        core[k, k, k] = (k + 1) ** -0.5
    facs = [haar_factor(g, size, rank) for _ in range(3)]
    clean = tucker_full(core, facs, dtype=np.float32 if dtype == np.float32 else np.float64)
    x = clean if snr_db is None else add_noise_snr(clean, snr_db, g, dtype=dtype)
    return Workload(f"tucker{size}_power", np.ascontiguousarray(x.astype(dtype, copy=False)),
                    clean, [rank] * 3, p, q, 42 + mc, facs)


def config_video(mc: int = 0, dims=(1024, 1024, 3, 256), ranks=(40, 40, 3, 30), snr_db: float = 5.0,
                 p: int = 10, q: int = 4) -> Workload:
    """Video-shaped (pixels x pixels x colour x frames) low-rank field: Gaussian core, DCT-II
    factors, noise at 5 dB.  Stand-in for the YUV sequences of Sec. 4.1.2."""
    g = rng(1003 + mc)
    c = g.standard_normal(ranks).astype(np.float32)
    facs = [dct_factor(i, r).astype(np.float32) for i, r in zip(dims, ranks)]
    clean = tucker_full(c, facs, dtype=np.float32)
    x = add_noise_snr(clean, snr_db, g, dtype=np.float32)
    return Workload("video_" + "x".join(map(str, dims)), x, clean, list(ranks), p, q, 42 + mc, facs)


def tr_init_cores(seed: int, dims: Sequence[int], ranks: Sequence[int]) -> List[np.ndarray]:
    """Initial TR cores for TR-ALS: N(0,1)/sqrt(r_{k-1} r_k), shape (r_{k-1}, dims[k], r_k), r_0 = r_N."""
    g = rng(seed)
    n = len(dims)
    out = []
    for k in range(n):
        r0, r1 = ranks[k - 1], ranks[k]
        out.append(g.standard_normal((r0, dims[k], r1)) / math.sqrt(r0 * r1))
    return out


def config_htr(mc: int = 0, order: int = 6, size: int = 16, tr_rank: int = 6, snr_db: float = 15.0,
               tucker_rank: int = 10, p: int = 5, q: int = 2, tr_seed: int = 7) -> Workload:
    """Random TR tensor (Gaussian 6x16x6 cores) + noise at 15 dB; Tucker rank 10 per mode, then
    TR of the 10^6 core with all TR ranks 6.  Stand-in for COIL-100 / CIFAR-10 (Sec. 4.2)."""
    g = rng(1004 + mc)
    cores = [g.standard_normal((tr_rank, size, tr_rank)) for _ in range(order)]
    clean = tr_full(cores).astype(np.float32)
    x = add_noise_snr(clean, snr_db, g, dtype=np.float32)
    ranks = [tucker_rank] * order
    return Workload(f"htr{size}^{order}", x, clean, ranks, p, q, 42 + mc,
                    tr_ranks=[tr_rank] * order,
                    tr_init=tr_init_cores(tr_seed, ranks, [tr_rank] * order))


def serve_stream(n_requests: int = 4096, seed: int = 5000, dim_lo: int = 32, dim_hi: int = 256,
                 rank_lo: int = 4, rank_hi: int = 32, p: int = 5, qs=(1, 2, 3),
                 snr_lo: float = 5.0, snr_hi: float = 25.0):
    """Request descriptors of the served stream (shapes, ranks, q, SNR, per-request seed).
    Tensors are made on demand with `serve_request_tensor` to bound host memory."""
    g = rng(seed)
    reqs = []
    for i in range(n_requests):
        dims = [int(v) for v in g.integers(dim_lo, dim_hi + 1, size=3)]
        ranks = [min(int(v), d) for v, d in zip(g.integers(rank_lo, rank_hi + 1, size=3), dims)]
        q = int(g.choice(qs))
        snr = float(g.uniform(snr_lo, snr_hi))
        reqs.append(dict(id=i, dims=dims, ranks=ranks, p=p, q=q, snr_db=snr, seed=seed * 10 + i))
    return reqs


def serve_request_device(req, device="cuda", dtype=None):
    """Device-side version of `serve_request_tensor` for large streams: the same recipe
    (Gaussian core and Haar factors drawn with NumPy from the request's seed; the dense
    tensor formed on the device; Gaussian noise from torch's generator seeded with the
    request's seed, scaled to the request's SNR by the realised norms).  The noise draws
    differ from the NumPy version's, so values are not identical to it.  Returns
    (x on `device` in `dtype` (default bfloat16), ranks, p, q, omega_seed)."""
    import torch
    g = rng(req["seed"])
    c = torch.from_numpy(g.standard_normal(req["ranks"]).astype(np.float32)).to(device)
    facs = [torch.from_numpy(haar_factor(g, i, r).astype(np.float32)).to(device)
            for i, r in zip(req["dims"], req["ranks"])]
    clean = torch.einsum("abc,ia,jb,kc->ijk", c, facs[0], facs[1], facs[2])
    gen = torch.Generator(device=device)
    gen.manual_seed(int(req["seed"]))
    noise = torch.randn(clean.shape, generator=gen, device=device, dtype=torch.float32)
    lam = torch.linalg.vector_norm(clean) / (torch.linalg.vector_norm(noise) * 10.0 ** (req["snr_db"] / 20.0))
    x = (clean + lam * noise).to(dtype or torch.bfloat16).contiguous()
    return x, list(req["ranks"]), req["p"], req["q"], req["seed"] + 17


def serve_request_tensor(req, dtype=np.float32) -> Workload:
    """Exactly multilinear-rank-`ranks` tensor (Gaussian core, Haar factors) + noise at the request's SNR."""
    g = rng(req["seed"])
    c = g.standard_normal(req["ranks"])
    facs = [haar_factor(g, i, r) for i, r in zip(req["dims"], req["ranks"])]
    clean = tucker_full(c, facs)
    x = add_noise_snr(clean, req["snr_db"], g, dtype=dtype)
    return Workload(f"req{req['id']}", x, clean, list(req["ranks"]), req["p"], req["q"],
                    req["seed"] + 17, facs)
