"""Partial column sampling for the Krylov construction (Sec. 3.2, after Table 2), oracle side.

Test infrastructure: only tests/, the smoke check and the CPU baseline of bench.py use it.

The paper shortens X_(n) (I_n x d_n, d_n large) to Y (I_n x m, m = omega d_n) by uniform
column sampling and builds the block Krylov space from Y instead of X_(n); omega is the
sampling rate (Fig. 5 sweeps omega = 0.1 .. 1; the hall video uses omega = 0.5).

Readings (where the paper is silent):
  c20 Algorithm 2 steps 3-5 use the products of the sampled construction (Remark 1 on Y):
      Z = Q^T Y Y^T Q, U = Q * leading eigenvectors of Z.  The core (step 6) uses all of X.
  c21 the sampling unit is a tile of 128 unfolding columns, not a single column:
        C_n > 1:  unit u = (a, c-block) with a = u // nb, columns c in [128 (u % nb), +128),
                  nb = ceil(C_n / 128);
        C_n = 1:  unit u = the 128 columns a in [128 u, +128);
      where X is viewed as [A_n][I_n][C_n] (A_n = prod_{k<n} I_k, C_n = prod_{k>n} I_k).
      A unit is all or nothing, so a sampled pass reads whole contiguous rows.  U_n units in
      all; m_u = clamp(ceil(omega U_n), 1, U_n) of them are kept.
  c22 which units: the m_u units with the smallest key
        key(u) = word 0 of Philox4x32-10(counter = (u mod 2^32, u >> 32, n, 0x53414D50),
                                          key = (seed mod 2^32, seed >> 32)),
      ties by the lower unit index; kept units are taken in ascending order.  Every subset
      of size m_u is equally likely (the keys are i.i.d. uniform words).
  c23 Y's column j*128 + t is the t-th column of the j-th kept unit, or a zero column where
      the unit is ragged (past C_n or A_n).  Omega for the sampled mode is indexed by Y's
      columns (reading c6 with Y in place of X_(n)).  Zero columns change neither Y Y^T nor
      the span.
  c24 only Krylov-path modes are sampled; a Gram-path mode (b_n >= I_n) stays the exact
      T-SVD mode.

Pins (tests/test_oracle_sampling.py): brute-force column extraction; with omega = 1 on tile-
aligned shapes the method is exactly the unsampled rBKI-TK; selection size, order and
uniform inclusion frequencies; Fig. 5's fit at omega = 0.1 on the [3, 200, 10], -5 dB
Gaussian tensor.
"""
from __future__ import annotations

import math
from typing import Tuple

import numpy as np

from . import philox
from .tensor import unfold

UNIT = 128
SAMPLE_TAG = 0x53414D50


def view_dims(shape, n: int) -> Tuple[int, int, int]:
    a = int(np.prod(shape[:n], dtype=np.int64))
    c = int(np.prod(shape[n + 1:], dtype=np.int64))
    return a, int(shape[n]), c


def unit_count(shape, n: int) -> int:
    a, _, c = view_dims(shape, n)
    if c > 1:
        return a * -(-c // UNIT)
    return -(-a // UNIT)


def kept_units(omega: float, n_units: int) -> int:
    return int(min(max(math.ceil(omega * n_units), 1), n_units))


def unit_keys(seed: int, n: int, n_units: int) -> np.ndarray:
    u = np.arange(n_units, dtype=np.uint64)
    key = (seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF)
    r0, _, _, _ = philox.philox4x32_10(
        (u & philox.MASK, u >> np.uint64(32), np.full(n_units, n, np.uint64),
         np.full(n_units, SAMPLE_TAG, np.uint64)), key)
    return r0


def sample_units(seed: int, n: int, n_units: int, m_u: int) -> np.ndarray:
    """Reading c22: the m_u smallest keys (ties -> lower index), in ascending unit order."""
    keys = unit_keys(seed, n, n_units)
    order = np.lexsort((np.arange(n_units), keys))      # by key, then by index
    return np.sort(order[:m_u]).astype(np.int64)


def sampled_unfolding(x: np.ndarray, n: int, units: np.ndarray) -> np.ndarray:
    """Y (I_n x 128 m_u) of reading c23, built from X_(n)'s columns."""
    a_n, i_n, c_n = view_dims(x.shape, n)
    xn = unfold(x, n)                                   # column index a * C_n + c
    y = np.zeros((i_n, UNIT * len(units)), dtype=xn.dtype)
    for j, u in enumerate(units):
        if c_n > 1:
            nb = -(-c_n // UNIT)
            a, c0 = int(u) // nb, (int(u) % nb) * UNIT
            w = min(UNIT, c_n - c0)
            y[:, j * UNIT: j * UNIT + w] = xn[:, a * c_n + c0: a * c_n + c0 + w]
        else:
            a0 = int(u) * UNIT
            w = min(UNIT, a_n - a0)
            y[:, j * UNIT: j * UNIT + w] = xn[:, a0: a0 + w]
    return y


def sampled_mode(x: np.ndarray, n: int, seed: int, omega: float):
    """(Y, units) for mode n at sampling rate omega."""
    nu = unit_count(x.shape, n)
    units = sample_units(seed, n, nu, kept_units(omega, nu))
    return sampled_unfolding(x, n, units), units
