"""Counter-based Gaussian sketching matrix Omega (oracle side).

The paper draws Omega^(n) in R^{prod_{p!=n} I_p x S_n} as "a randomized sketching
matrix" (Algorithm 1, step 1); its comparison methods make clear the Gaussian
family is meant (Sec. 4.1, GR-SVD etc.).  To let two independent implementations
draw the *same* Omega, each entry is defined by a published counter-based
generator:

  Philox4x32-10 (J. Salmon, M. Moraes, R. Dror, D. Shaw, "Parallel random numbers:
  as easy as 1, 2, 3", SC'11):  key (k0, k1) = (seed mod 2^32, seed >> 32);
  counter (c0, c1, c2, c3) = (s >> 1, n, col mod 2^32, col >> 32)
  where n is the mode, col the C-order linear index of the unfolding column and s
  the sketch column.  Ten rounds, key bumped by the Weyl constants between rounds.

  Box-Muller on two 53-bit uniforms built from the four output words r0..r3:
     u1 = ((r0 >> 5) * 2^26 + (r1 >> 6) + 1) * 2^-53   in (0, 1]
     u2 = ((r2 >> 5) * 2^26 + (r3 >> 6))     * 2^-53   in [0, 1)
     rho = sqrt(-2 ln u1);  Omega[col, s] = rho cos(2 pi u2) for even s,
                                            rho sin(2 pi u2) for odd s.

Pins (tests/test_oracle_philox.py): the published Philox4x32-10 known-answer
vectors (tests/golden/philox4x32_10_kat.txt), the moments of N(0,1), and
prefix nesting in s.
"""
from __future__ import annotations

import numpy as np

M0 = np.uint64(0xD2511F53)
M1 = np.uint64(0xCD9E8D57)
W0 = np.uint64(0x9E3779B9)
W1 = np.uint64(0xBB67AE85)
MASK = np.uint64(0xFFFFFFFF)


def philox4x32_10(ctr, key):
    """Philox4x32 with 10 rounds.  ctr: 4 arrays of uint32-valued ints; key: 2 ints.
    Returns 4 uint64 arrays holding 32-bit words (SC'11, Sec. 4 / Figure 2)."""
    x0, x1, x2, x3 = (np.asarray(c, dtype=np.uint64) & MASK for c in ctr)
    k0 = np.uint64(int(key[0]) & 0xFFFFFFFF)
    k1 = np.uint64(int(key[1]) & 0xFFFFFFFF)
    for rnd in range(10):
        if rnd:
            k0 = (k0 + W0) & MASK
            k1 = (k1 + W1) & MASK
        p0 = M0 * x0
        p1 = M1 * x2
        hi0, lo0 = p0 >> np.uint64(32), p0 & MASK
        hi1, lo1 = p1 >> np.uint64(32), p1 & MASK
        x0, x1, x2, x3 = hi1 ^ x1 ^ k0, lo1, hi0 ^ x3 ^ k1, lo0
    return x0, x1, x2, x3


def omega(seed: int, mode: int, cols, n_sketch: int) -> np.ndarray:
    """Omega^(mode)[cols, 0:n_sketch] in FP64 (rows = unfolding columns)."""
    cols = np.asarray(cols, dtype=np.uint64).reshape(-1)
    out = np.empty((cols.size, n_sketch), dtype=np.float64)
    key = (seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF)
    for pair in range((n_sketch + 1) // 2):
        r0, r1, r2, r3 = philox4x32_10(
            (np.full(cols.size, pair, np.uint64), np.full(cols.size, mode, np.uint64),
             cols & MASK, cols >> np.uint64(32)), key)
        u1 = ((r0 >> np.uint64(5)).astype(np.float64) * 67108864.0
              + (r1 >> np.uint64(6)).astype(np.float64) + 1.0) * 2.0 ** -53
        u2 = ((r2 >> np.uint64(5)).astype(np.float64) * 67108864.0
              + (r3 >> np.uint64(6)).astype(np.float64)) * 2.0 ** -53
        rho = np.sqrt(-2.0 * np.log(u1))
        out[:, 2 * pair] = rho * np.cos(2.0 * np.pi * u2)
        if 2 * pair + 1 < n_sketch:
            out[:, 2 * pair + 1] = rho * np.sin(2.0 * np.pi * u2)
    return out


def omega_mode(seed: int, mode: int, dims, n_sketch: int) -> np.ndarray:
    """The full d_n x S_n sketching matrix of mode `mode` for a tensor of shape `dims`."""
    d = int(np.prod([v for k, v in enumerate(dims) if k != mode], dtype=np.int64))
    return omega(seed, mode, np.arange(d, dtype=np.uint64), n_sketch)
