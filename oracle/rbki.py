"""rBKI tensor sketching (Algorithm 1) and rBKI-TK (Algorithm 2), oracle side, FP64.

Steps follow the paper's order and notation:

  Algorithm 1 (per mode n, X_(n) in R^{I_n x d_n}):
    step 1  Omega^(n) in R^{d_n x S_n}, Gaussian (oracle.philox, reading c6)
    step 2  W = X_(n) Omega^(n)
    step 3  K = [W, (X X^T) W, ..., (X X^T)^q W]        (Eq. BKspace)
    ENSURE  Q = orth(K)                                 (economical QR)
  Algorithm 2 (per mode n):
    step 2  Q^(n) = rBKI(X_(n), S_n)
    step 3  Z^(n) = Q^T X_(n) X_(n)^T Q                 (Remark 1)
    step 4  U~ = leading eigenvectors of Z (Z symmetric PSD: svd(Z) = evd(Z), reading c5)
    step 5  U^(n) = Q U~(:, 1:R_n)
    step 6  G = X x_1 U^(1)T ... x_N U^(N)T            (HOSVD reading c1, Eq. tensorsketch)

Readings (where the paper is silent):
  c2  K is orthonormalised block by block: block j+1 = orth((X X^T) Q_j) against all
      earlier blocks.  In exact arithmetic this spans exactly the space of Eq. BKspace.
  c3  deflation: a new direction is dropped when the norm of its component orthogonal
      to every accepted direction is <= TAU_DEFLATE x its norm before projection.
      If fewer than R_n directions survive, U is completed with an orthonormal
      complement (whose core slices are exactly zero).
  c4  S_n = min(R_n + p, I_n); K has q+1 blocks, width b_n = S_n (q+1).
  c5  eigenvalues descending; each factor column's largest-|.| entry made positive
      (ties -> lowest row index).
  c7  when b_n >= I_n the Krylov space is all of R^{I_n}: Z = X_(n) X_(n)^T, Q = I
      ("Gram path"), which is exactly truncated HOSVD for that mode.

Parity pins (tests/test_oracle_rbki.py): q = 0 equals the randomized range finder
computed by LAPACK QR + SVD; b_n >= I_n equals T-SVD; exact recovery of noiseless
low-rank tensors; Theorem 1 (optimality within span Q); Remark 1's energy identity;
eigenvalue interlacing; Eq. Pythagorean and Theorem 2 bounds; nesting in q and p;
paper Tables 3-4 (statistical).
"""
from __future__ import annotations

from typing import Dict, List, Sequence

import numpy as np

from . import philox, sampling
from .tensor import ttm, unfold

TAU_DEFLATE = 1e-6


def sketch_plan(dims: Sequence[int], ranks: Sequence[int], p: int, q: int, variant: str = "krylov"):
    """Per mode: (S_n, b_n, path) with path 'krylov' or 'gram' (readings c4, c7).  The
    power-iteration variant keeps one block of width S_n (b_n = S_n)."""
    plan = []
    for i_n, r_n in zip(dims, ranks):
        s = min(r_n + p, i_n)
        b = s if variant == "power" else s * (q + 1)
        plan.append((s, b, "gram" if b >= i_n else "krylov"))
    return plan


def orth_block(v: np.ndarray, prev: np.ndarray, tau: float = TAU_DEFLATE) -> np.ndarray:
    """Orthonormal basis of the part of span(v) orthogonal to span(prev) (reading c2, c3).

    Column by column: classical Gram-Schmidt applied twice against every accepted
    direction (earlier blocks and earlier columns of this block); a column is kept iff
    the remaining norm exceeds tau x its norm before projection."""
    basis = [prev[:, k] for k in range(prev.shape[1])] if prev.size else []
    kept = []
    for k in range(v.shape[1]):
        col = v[:, k].astype(np.float64, copy=True)
        nu = float(np.linalg.norm(col))
        if nu == 0.0:
            continue
        if basis:
            b = np.stack(basis, axis=1)
            for _ in range(2):
                col = col - b @ (b.T @ col)
        rem = float(np.linalg.norm(col))
        if rem > tau * nu:
            col = col / rem
            basis.append(col)
            kept.append(col)
    if not kept:
        return np.zeros((v.shape[0], 0))
    return np.stack(kept, axis=1)


def rbki(xn: np.ndarray, om: np.ndarray, q: int, tau: float = TAU_DEFLATE) -> List[np.ndarray]:
    """Algorithm 1 with block orthonormalisation: returns the blocks Q_0..Q_q."""
    w = xn @ om                                          # step 2: W = X Omega
    blocks = [orth_block(w, np.zeros((xn.shape[0], 0)), tau)]
    for _ in range(q):                                   # step 3: K = [W, AW, ..., A^q W]
        prev = np.concatenate(blocks, axis=1)
        v = xn @ (xn.T @ blocks[-1])                     # (X X^T) Q_j
        blocks.append(orth_block(v, prev, tau))
    return blocks


def power_basis(xn: np.ndarray, om: np.ndarray, q: int, tau: float = TAU_DEFLATE) -> np.ndarray:
    """Power-iteration baseline (the "P-iter" / GRpi comparison of Sec. 3.1: K = (X X^T)^q W
    instead of Eq. BKspace): Q_0 = orth(X Omega), Q_{j+1} = orth((X X^T) Q_j), and the
    basis is the last block Q_q alone (width S)."""
    qb = orth_block(xn @ om, np.zeros((xn.shape[0], 0)), tau)
    for _ in range(q):
        qb = orth_block(xn @ (xn.T @ qb), np.zeros((xn.shape[0], 0)), tau)
    return qb


def mode_fit(lam: np.ndarray, x_norm2: float) -> float:
    """Fit (as a fraction, 1 - |X - X^|/|X|) of the rank-R projection U U^T X_(n) whose
    Rayleigh-Ritz values are lam: |X - U U^T X|^2 = |X|^2 - sum(lam) (reading c27)."""
    return 1.0 - np.sqrt(max(x_norm2 - float(np.sum(lam)), 0.0) / x_norm2)


def krylov_adaptive(xn: np.ndarray, om: np.ndarray, r: int, q_max: int, q_tol: float,
                    tau: float = TAU_DEFLATE):
    """Adaptive depth (reading c26): after block j the Rayleigh-Ritz step runs on Q_0..Q_j;
    stop at the first j >= 1 with |Fit_j - Fit_{j-1}| <= q_tol, or at j = q_max.
    Returns (U, lambda, kept width, q used, fits)."""
    x_norm2 = float(np.sum(xn * xn))
    blocks = [orth_block(xn @ om, np.zeros((xn.shape[0], 0)), tau)]
    fits = []
    for j in range(q_max + 1):
        qb = np.concatenate(blocks, axis=1)
        u, lam, _ = rayleigh_ritz(xn, qb, r)
        fits.append(mode_fit(lam, x_norm2))
        if j == q_max or (j >= 1 and abs(fits[j] - fits[j - 1]) <= q_tol):
            return u, lam, qb.shape[1], j, fits
        blocks.append(orth_block(xn @ (xn.T @ blocks[-1]), qb, tau))
    raise AssertionError("unreachable")


def complete_basis(u: np.ndarray, r: int) -> np.ndarray:
    """Extend orthonormal columns u (I x k, k < r) to r columns with e_1, e_2, ... projected
    out of the current span (reading c3)."""
    cols = [u[:, k] for k in range(u.shape[1])]
    e = 0
    while len(cols) < r:
        c = np.zeros(u.shape[0])
        c[e] = 1.0
        e += 1
        b = np.stack(cols, axis=1) if cols else np.zeros((u.shape[0], 0))
        for _ in range(2):
            c = c - b @ (b.T @ c)
        nc = np.linalg.norm(c)
        if nc > 1e-8:
            cols.append(c / nc)
    return np.stack(cols, axis=1)


def sign_fix(u: np.ndarray) -> np.ndarray:
    """Make the largest-magnitude entry of each column positive (first index on ties)."""
    u = u.copy()
    for k in range(u.shape[1]):
        i = int(np.argmax(np.abs(u[:, k])))
        if u[i, k] < 0:
            u[:, k] = -u[:, k]
    return u


def rayleigh_ritz(xn: np.ndarray, q_basis: np.ndarray, r: int):
    """Algorithm 2 steps 3-5: Z = Q^T X X^T Q, leading eigenvectors, U = Q U~(:, 1:R)."""
    y = q_basis.T @ xn                                   # Q^T X_(n)
    z = y @ y.T                                          # Remark 1
    lam, vec = np.linalg.eigh(z)
    order = np.argsort(-lam, kind="stable")
    lam, vec = lam[order], vec[:, order]
    k = min(r, q_basis.shape[1])
    u = q_basis @ vec[:, :k]
    if k < r:
        u = complete_basis(u, r)
        lam = np.concatenate([lam[:k], np.zeros(r - k)])
    return sign_fix(u), lam[:r], z


def refine_rr(a: np.ndarray, u: np.ndarray):
    """Rayleigh-Ritz refinement of a factor (the precision pattern's final step, reading c17):
    Z_r = U^T A A^T U from a fresh product with the unfolding A, its eigenvectors W
    (descending), U' = U W with the sign rule, and the Ritz values lambda'.  U' spans the
    same space as U, so the projector U U^T (and the reconstruction error) is unchanged; in
    exact arithmetic, when U already holds eigenvectors of the mode's Rayleigh quotient, Z_r
    is diagonal and U' = U.  A path whose Z carries product rounding gets its Ritz values
    and vectors recomputed from accurate products."""
    y = u.T @ a
    zr = y @ y.T
    lam, vec = np.linalg.eigh(zr)
    order = np.argsort(-lam, kind="stable")
    return sign_fix(u @ vec[:, order]), lam[order]


def krylov_mode(xn: np.ndarray, x: np.ndarray, n: int, s: int, r: int, q: int, seed: int, omega: float,
                tau: float = TAU_DEFLATE, variant: str = "krylov", q_tol=None, refine: bool = False):
    """Algorithms 1-2 for a Krylov-path mode of tensor x (unfolding xn): (U, lambda, kept, q used).
    0 < omega < 1: the Krylov space and Z come from the sampled Y (oracle.sampling).
    variant "power": the power-iteration basis; q_tol: adaptive depth with q as the bound;
    refine: the Rayleigh-Ritz refinement of U on the same data (refine_rr)."""
    if 0.0 < omega < 1.0:
        if q_tol is not None:
            raise ValueError("adaptive q with column sampling is not defined")
        y, _ = sampling.sampled_mode(x, n, seed, omega)
        om = philox.omega(seed, n, np.arange(y.shape[1], dtype=np.uint64), s)
        a = y
    else:
        om = philox.omega_mode(seed, n, x.shape, s)
        a = xn
    if q_tol is not None:
        if variant != "krylov":
            raise ValueError("adaptive q applies to the block Krylov space")
        u, lam, k, qu, _ = krylov_adaptive(a, om, r, q, q_tol, tau)
        return u, lam, k, qu
    qb = power_basis(a, om, q, tau) if variant == "power" else np.concatenate(rbki(a, om, q, tau), axis=1)
    u, lam, _ = rayleigh_ritz(a, qb, r)
    if refine:
        u, lam = refine_rr(a, u)
    return u, lam, qb.shape[1], q


def rbki_tucker(x: np.ndarray, ranks: Sequence[int], p: int, q: int, seed: int,
                tau: float = TAU_DEFLATE, omega: float = 1.0, variant: str = "krylov", q_tol=None,
                refine: bool = False) -> Dict:
    """Algorithm 2 (rBKI-TK), HOSVD reading: every mode sketches the original X.
    0 < omega < 1: partial column sampling of the Krylov construction (oracle.sampling).
    variant "power": the power-iteration baseline; q_tol: adaptive depth, q the bound;
    refine: Rayleigh-Ritz refinement of each Krylov-path factor (refine_rr)."""
    x = np.asarray(x, dtype=np.float64)
    plan = sketch_plan(x.shape, ranks, p, q, variant)
    factors, eigvals, kept, paths, q_used = [], [], [], [], []
    for n, (s, b, path) in enumerate(plan):
        xn = unfold(x, n)
        if path == "gram":
            lam, vec = np.linalg.eigh(xn @ xn.T)
            order = np.argsort(-lam, kind="stable")
            u = sign_fix(vec[:, order[: ranks[n]]])
            lam = lam[order[: ranks[n]]]
            kept.append(x.shape[n])
            q_used.append(0)
        else:
            u, lam, k, qu = krylov_mode(xn, x, n, s, ranks[n], q, seed, omega, tau, variant, q_tol, refine)
            kept.append(k)
            q_used.append(qu)
        factors.append(u)
        eigvals.append(lam)
        paths.append(path)
    core = x
    for n, u in enumerate(factors):
        core = ttm(core, u.T, n)                         # step 6
    return dict(core=core, factors=factors, eigvals=eigvals, kept=kept, path=paths, q_used=q_used,
                x_norm2=float(np.sum(x * x)), core_norm2=float(np.sum(core * core)))


def rbki_st_tucker(x: np.ndarray, ranks: Sequence[int], p: int, q: int, seed: int,
                   tau: float = TAU_DEFLATE, omega: float = 1.0, variant: str = "krylov") -> Dict:
    """Algorithm 2 read literally (sequential truncation, the other reading of step 6): the
    modes are taken in order n = 1..N, and mode n is sketched from the tensor already
    contracted by the earlier factors, Y_n = X x_1 U^(1)T ... x_{n-1} U^(n-1)T; after U^(n)
    the tensor is contracted once more, and the last contraction is the core.  Omega^(n) is
    keyed by the column index of Y_n's mode-n unfolding (reading c6 applied to Y_n).
    Returns the same fields as rbki_tucker, plus `step_res2[n]` = |Y_n - Y_n x_n U U^T|^2."""
    y = np.asarray(x, dtype=np.float64)
    x_norm2 = float(np.sum(y * y))
    factors, eigvals, kept, paths, res2 = [], [], [], [], []
    for n in range(y.ndim):
        s, b, path = sketch_plan(y.shape, ranks, p, q, variant)[n]
        yn = unfold(y, n)
        if path == "gram":
            lam, vec = np.linalg.eigh(yn @ yn.T)
            order = np.argsort(-lam, kind="stable")
            u = sign_fix(vec[:, order[: ranks[n]]])
            lam = lam[order[: ranks[n]]]
            kept.append(y.shape[n])
        else:
            u, lam, k, _ = krylov_mode(yn, y, n, s, ranks[n], q, seed, omega, tau, variant)
            kept.append(k)
        factors.append(u)
        eigvals.append(lam)
        paths.append(path)
        nxt = ttm(y, u.T, n)                              # step 6, inside the mode loop
        res2.append(float(np.sum(y * y) - np.sum(nxt * nxt)))
        y = nxt
    return dict(core=y, factors=factors, eigvals=eigvals, kept=kept, path=paths, step_res2=res2,
                x_norm2=x_norm2, core_norm2=float(np.sum(y * y)))


def krylov_basis(x: np.ndarray, n: int, s: int, q: int, seed: int, tau: float = TAU_DEFLATE):
    """Q^(n) of Algorithm 1 for mode n (all blocks concatenated)."""
    x = np.asarray(x, dtype=np.float64)
    xn = unfold(x, n)
    om = philox.omega_mode(seed, n, x.shape, s)
    return np.concatenate(rbki(xn, om, q, tau), axis=1)


def tsvd(x: np.ndarray, ranks: Sequence[int]) -> Dict:
    """Truncated HOSVD (the T-SVD benchmark of Sec. 4): U^(n) = leading left singular
    vectors of X_(n) (Lemma 1, Eckart-Young), G = X x_n U^(n)T."""
    x = np.asarray(x, dtype=np.float64)
    factors = []
    for n, r in enumerate(ranks):
        u, _, _ = np.linalg.svd(unfold(x, n), full_matrices=False)
        factors.append(sign_fix(u[:, :r]))
    core = x
    for n, u in enumerate(factors):
        core = ttm(core, u.T, n)
    return dict(core=core, factors=factors)


def reconstruct(core: np.ndarray, factors: Sequence[np.ndarray]) -> np.ndarray:
    t = core
    for n, u in enumerate(factors):
        t = ttm(t, u, n)
    return t
