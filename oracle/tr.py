"""TR-ALS on the Tucker core and rBKI-TK-TR (Algorithm 3), oracle side, FP64.

Algorithm 3: (1) rBKI-TK compresses X to [[G; U^(1..N)]]; (3) TR-ALS fits a tensor
ring to the small core G; (4) each TR core is contracted with its factor over the
physical mode: X_n = G_n x_2 U^(n) in R^{R_{n-1} x I_n x R_n}.

Readings (where the paper is silent):
  c9   TR-ALS runs once on G and yields all N cores; ring closed by r_0 = r_N.
  c10  the initial cores are inputs (seeded, from `synth.tr_init_cores`); a sweep
       updates cores 1..N in order; each update is the exact least-squares solution of
       Eq. unTR for that core with the others fixed; stop after `maxit` sweeps or when
       |Fit_t - Fit_{t-1}| <= tol, Fit measured as a fraction against G (Sec. 4 stopping
       rule, max 20 iterations, tol 1e-3).

TR-SVD (`tr_svd`, reading c32) is pinned by exact recovery of a TR tensor whose unfolding
ranks match, by the exact split of its error into the steps' truncation errors, and, for
N = 2 with r_1 = 1, by the Eckart-Young truncated SVD.

Parity: the LS update is pinned by monotone non-increasing residual (exact ALS) and by
exact recovery of a noiseless TR tensor's ring from a nearby start; the contraction
identity R[[Z_n x_2 U_n]] = R[[Z_n]] x_1 U_1 ... x_N U_N is pinned exactly.  Agreement
of ALS iterates with another implementation is otherwise "parity unpinned" (ALS is
non-convex; the GPU path must follow the same iterates from the same start).
"""
from __future__ import annotations

from typing import List, Sequence

import numpy as np

from .rbki import rbki_tucker, sign_fix
from .tensor import tr


def subchain(cores: Sequence[np.ndarray], k: int) -> np.ndarray:
    """B_{!=k}: rows = indices of modes k+1..N-1,0..k-1 (C-order in that cyclic order),
    columns (a, b) for core k's entry Z_k[a, i, b]; B[row, a*r_k + b] = M(row)[b, a] with
    M = Z_{k+1}(i_{k+1}) ... Z_{k-1}(i_{k-1}) in R^{r_k x r_{k-1}}  (Eq. unTR)."""
    n = len(cores)
    order = [(k + j) % n for j in range(1, n)]
    t = cores[order[0]]                                   # (r_k, I, r)
    for m in order[1:]:
        t = np.tensordot(t, cores[m], axes=(t.ndim - 1, 0))
    # t: (r_k, I_{k+1}, ..., I_{k-1}, r_{k-1}) -> (I..., r_{k-1}, r_k)
    t = np.moveaxis(t, 0, -1)
    rows = int(np.prod(t.shape[:-2]))
    return t.reshape(rows, t.shape[-2] * t.shape[-1])


def unfold_cyclic(g: np.ndarray, k: int) -> np.ndarray:
    """G_(k) with columns in the cyclic order k+1..N-1,0..k-1 used by `subchain`."""
    n = g.ndim
    perm = [k] + [(k + j) % n for j in range(1, n)]
    return np.transpose(g, perm).reshape(g.shape[k], -1)


def tr_fit(g: np.ndarray, cores: Sequence[np.ndarray]) -> float:
    """Fit as a fraction: 1 - |G - R[[cores]]| / |G|."""
    return 1.0 - float(np.linalg.norm((g - tr(cores)).ravel()) / np.linalg.norm(g.ravel()))


def tr_als(g: np.ndarray, init: Sequence[np.ndarray], maxit: int = 20, tol: float = 1e-3):
    """TR-ALS (reading c10).  Returns (cores, fits per sweep)."""
    cores: List[np.ndarray] = [np.array(c, dtype=np.float64, copy=True) for c in init]
    g = np.asarray(g, dtype=np.float64)
    n = g.ndim
    fits = []
    prev = None
    for _ in range(maxit):
        for k in range(n):
            b = subchain(cores, k)                        # (prod_{j!=k} I_j, r_{k-1} r_k)
            gk = unfold_cyclic(g, k)                      # (I_k, prod_{j!=k} I_j)
            sol, *_ = np.linalg.lstsq(b, gk.T, rcond=None)  # min |G_(k) - Z_k(2) B^T|
            r0, r1 = cores[k].shape[0], cores[k].shape[2]
            cores[k] = sol.T.reshape(g.shape[k], r0, r1).transpose(1, 0, 2).copy()
        f = tr_fit(g, cores)
        fits.append(f)
        if prev is not None and abs(f - prev) <= tol:
            break
        prev = f
    return cores, fits


def tr_svd(g: np.ndarray, ranks: Sequence[int]):
    """TR-SVD (Zhao, Zhou, Xie, Zhang, Cichocki 2016), the alternative Algorithm 3 step 3
    names, with fixed TR ranks (reading c32): core n has shape (r_{n-1}, S_n, r_n), r_{-1} =
    r_{N-1}.
      step 0:  C = G as S_1 x prod(rest); truncated SVD of rank r_{N-1} r_0; core 0 [a, i, b]
               = U[i, a r_0 + b]; the remainder Sigma V^T, indexed (a, b, rest), is reordered
               to (b, rest, a) and read as (r_0 S_2) x (prod(rest) r_{N-1} / S_2);
      step n:  truncated SVD of rank r_n of C ((r_{n-1} S_n) x ...); core n = U as
               (r_{n-1}, S_n, r_n); C <- Sigma V^T read as (r_n S_{n+1}) x ...;
      last:    core N-1 = C as (r_{N-2}, S_N, r_{N-1}).
    Each U is sign-normalised (largest-|.| entry of every column positive, reading c5) before
    use: the split of step 0 mixes bond indices, so the result depends on the signs.
    Returns (cores, squared truncation error of every step)."""
    g = np.asarray(g, dtype=np.float64)
    n = g.ndim
    r = list(ranks)
    cores = []
    errs = []
    c = g.reshape(g.shape[0], -1)
    for k in range(n - 1):
        rk = r[n - 1] * r[0] if k == 0 else r[k]
        u, sv, _ = np.linalg.svd(c, full_matrices=False)
        errs.append(float(np.sum(sv[rk:] ** 2)))
        u = sign_fix(u[:, :rk])
        w = u.T @ c                                                        # Sigma V^T, signs of u
        if k == 0:
            cores.append(u.reshape(g.shape[0], r[n - 1], r[0]).transpose(1, 0, 2).copy())
            w = w.reshape(r[n - 1], r[0], -1).transpose(1, 2, 0)          # (b, rest, a)
            c = w.reshape(r[0] * g.shape[1], -1)
        else:
            cores.append(u.reshape(r[k - 1], g.shape[k], r[k]).copy())
            c = w.reshape(r[k] * g.shape[k + 1], -1)
    cores.append(c.reshape(r[n - 2], g.shape[n - 1], r[n - 1]).copy())
    return cores, errs


def contract_factor(core: np.ndarray, u: np.ndarray) -> np.ndarray:
    """Algorithm 3 step 4: X_n = G_n x_2 U^(n):  X_n[a, i, b] = sum_s U[i, s] G_n[a, s, b]."""
    return np.einsum("is,asb->aib", u, core)


def rbki_tk_tr(x: np.ndarray, tucker_ranks: Sequence[int], p: int, q: int, seed: int,
               tr_init: Sequence[np.ndarray], maxit: int = 20, tol: float = 1e-3, tr_ranks=None):
    """Algorithm 3 (rBKI-TK-TR).  tr_init None: TR-SVD with ranks tr_ranks instead of TR-ALS."""
    tk = rbki_tucker(x, tucker_ranks, p, q, seed)
    if tr_init is None:
        cores, _ = tr_svd(tk["core"], tr_ranks)
        fits = [tr_fit(tk["core"], cores)]
    else:
        cores, fits = tr_als(tk["core"], tr_init, maxit, tol)
    tr_cores = [contract_factor(c, u) for c, u in zip(cores, tk["factors"])]
    return dict(tucker=tk, small_cores=cores, fits=fits, cores=tr_cores)
