"""Accuracy metrics of Sec. 4 (oracle side) and subspace comparison helpers.

Fit(%) = (1 - |X - X~|_F / |X|_F) * 100; X is the clean tensor (reading c11).
RErr   = |X - X~|_F / |X - X_k|_F with X_k the truncated-HOSVD approximation.
PSNR   = 10 log10(peak^2 / MSE), MSE = |X - X~|_F^2 / num(X) (reading c12: the
         printed formula omits the square).
Parity: closed forms on hand-made inputs in tests/test_oracle_metrics.py.
"""
from __future__ import annotations

import numpy as np


def fnorm(x) -> float:
    return float(np.linalg.norm(np.asarray(x, dtype=np.float64).ravel()))


def fit(ref, approx) -> float:
    return (1.0 - fnorm(np.asarray(ref, np.float64) - approx) / fnorm(ref)) * 100.0


def rerr(ref, approx, best) -> float:
    return fnorm(np.asarray(ref, np.float64) - approx) / fnorm(np.asarray(ref, np.float64) - best)


def psnr(ref, approx, peak=None) -> float:
    ref = np.asarray(ref, np.float64)
    peak = float(np.max(np.abs(ref))) if peak is None else float(peak)
    mse = fnorm(ref - approx) ** 2 / ref.size
    return 10.0 * np.log10(peak ** 2 / mse)


def snr_db(signal, noise) -> float:
    """Eq. SNR: 20 log10(|X|_F / |lambda N|_F)."""
    return 20.0 * np.log10(fnorm(signal) / fnorm(noise))


def max_principal_sine(a: np.ndarray, b: np.ndarray) -> float:
    """Largest principal-angle sine between span(a) and span(b) (orthonormal columns):
    |(I - a a^T) b|_2."""
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    r = b - a @ (a.T @ b)
    return float(np.linalg.norm(r, 2)) if r.size else 0.0
