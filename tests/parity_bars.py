"""Shared FP64 bar on the reconstruction error.

The error is sqrt(|X|^2 - |G|^2) (Eq. Pythagorean).  Rounding in the two norms is about
1e-16 |X|^2, so where the fit is exact (|X|^2 - |G|^2 near 0) the square root turns it into
about 1e-8 |X|; there the squared errors are compared instead."""
import math


def err_matches(e: float, e_ref: float, x_norm2: float) -> bool:
    if abs(e - e_ref) <= 1e-12 * e_ref + 1e-13 * math.sqrt(x_norm2):
        return True
    return abs(e * e - e_ref * e_ref) <= 1e-13 * x_norm2
