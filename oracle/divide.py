"""Divide-and-conquer decomposition along one mode (Sec. 4.1.2, the "divide and conquer"
processing of the flower video), oracle side.  Test infrastructure: only tests/, the smoke
check and the CPU baseline of bench.py use it.

The paper splits the frame mode of a video into consecutive subsets (250 frames into five
of 50) and decomposes each subset with the same rank-to-size ratio (rank 50 of 250 frames
one-pass, 10 of 50 per subset).

Readings (where the paper is silent):
  c29 part k of K along mode n covers indices [floor(k I_n / K), floor((k+1) I_n / K)), so
      every part is non-empty when K <= I_n and sizes differ by at most one.
  c30 part k is decomposed by rBKI-TK (Algorithm 2) with seed + k, so the parts draw
      different sketches; the ranks are the caller's, per part.
  c31 the approximation of X is the concatenation of the parts' Tucker approximations
      along mode n; its squared error is the sum of the parts' squared errors,
      sum_k (|X_k|^2 - |G_k|^2).

Pins (tests/test_oracle_divide.py): K = 1 is the one-pass decomposition; the parts
tile X exactly (brute-force reassembly); the error identity of c31 against the explicit
concatenated reconstruction.
"""
from __future__ import annotations

from typing import Dict, List, Sequence

import numpy as np

from . import rbki


def part_bounds(size: int, parts: int) -> List[tuple]:
    """Reading c29: [floor(k I / K), floor((k+1) I / K)) for k = 0..K-1."""
    if not 1 <= parts <= size:
        raise ValueError("need 1 <= parts <= size")
    return [(k * size // parts, (k + 1) * size // parts) for k in range(parts)]


def split(x: np.ndarray, mode: int, parts: int) -> List[np.ndarray]:
    out = []
    for lo, hi in part_bounds(x.shape[mode], parts):
        idx = [slice(None)] * x.ndim
        idx[mode] = slice(lo, hi)
        out.append(np.ascontiguousarray(x[tuple(idx)]))
    return out


def divide_and_conquer(x: np.ndarray, mode: int, parts: int, ranks: Sequence[Sequence[int]], p: int, q: int,
                       seed: int, **kw) -> Dict:
    """Readings c29-c31: rBKI-TK of every part (ranks[k] for part k, seed + k)."""
    x = np.asarray(x, dtype=np.float64)
    res = [rbki.rbki_tucker(xk, ranks[k], p, q, seed + k, **kw) for k, xk in enumerate(split(x, mode, parts))]
    err2 = sum(max(r["x_norm2"] - r["core_norm2"], 0.0) for r in res)
    return dict(parts=res, err2=err2, x_norm2=float(np.sum(x * x)))


def reconstruct(res: Dict, mode: int) -> np.ndarray:
    return np.concatenate([rbki.reconstruct(r["core"], r["factors"]) for r in res["parts"]], axis=mode)
