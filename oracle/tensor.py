"""Tensor algebra of Sec. 2.1 (oracle side): unfolding, mode-n product, Tucker and TR models.

Parity: pinned by tests/test_oracle_tensor.py against brute-force index loops on
tiny tensors (unfold / ttm / tucker / tr) - independent of the vectorised code here.
"""
from __future__ import annotations

from typing import Sequence

import numpy as np


def unfold(x: np.ndarray, n: int) -> np.ndarray:
    """Mode-n matricization X_(n) in R^{I_n x prod_{p!=n} I_p} (Table 1, Eq. unTKD).
    Column index = C-order linear index of the remaining indices (reading c8)."""
    return np.moveaxis(x, n, 0).reshape(x.shape[n], -1)


def fold(m: np.ndarray, n: int, shape: Sequence[int]) -> np.ndarray:
    """Inverse of `unfold` for a tensor of `shape` (mode n of size m.shape[0])."""
    rest = [s for k, s in enumerate(shape) if k != n]
    return np.moveaxis(m.reshape([m.shape[0]] + rest), 0, n)


def ttm(x: np.ndarray, m: np.ndarray, n: int) -> np.ndarray:
    """Mode-n product X x_n M: (X x_n M)_(n) = M X_(n)  (Table 1, Eq. TKD)."""
    shape = list(x.shape)
    shape[n] = m.shape[0]
    return fold(m @ unfold(x, n), n, shape)


def tucker(core: np.ndarray, factors: Sequence[np.ndarray]) -> np.ndarray:
    """[[G; U^(1),...,U^(N)]] = G x_1 U^(1) ... x_N U^(N)  (Eq. TKD)."""
    t = core
    for n, u in enumerate(factors):
        t = ttm(t, u, n)
    return t


def tr(cores: Sequence[np.ndarray]) -> np.ndarray:
    """TR model X(i_1..i_N) = trace(X_1(i_1) X_2(i_2) ... X_N(i_N)), cores (r_{n-1}, I_n, r_n),
    ring closed by r_0 = r_N (Eq. TR; reading c9)."""
    t = cores[0]
    for c in cores[1:]:
        t = np.tensordot(t, c, axes=(t.ndim - 1, 0))
    return np.trace(t, axis1=0, axis2=t.ndim - 1)
