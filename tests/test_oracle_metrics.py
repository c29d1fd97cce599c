"""Pins for the oracle metrics (Sec. 4) and the SNR generator (Eq. SNR)."""
import numpy as np

import synth
from oracle import metrics


def test_fit_rerr_psnr_closed_forms():
    ref = np.ones((4, 4))
    approx = ref * 0.9                                   # |ref - approx| = 0.1 |ref|
    assert abs(metrics.fit(ref, approx) - 90.0) < 1e-12
    assert abs(metrics.rerr(ref, approx, ref * 0.95) - 2.0) < 1e-12
    # MSE = 0.01, peak 1 -> 20 dB
    assert abs(metrics.psnr(ref, approx, peak=1.0) - 20.0) < 1e-12


def test_snr_generator_exact():
    g = synth.rng(3)
    x = g.standard_normal((10, 11, 12))
    for snr in (-10.0, 0.0, 5.0, 25.0):
        y = synth.add_noise_snr(x, snr, synth.rng(4))
        assert abs(metrics.snr_db(x, y - x) - snr) < 1e-10


def test_principal_sine():
    a = np.eye(5)[:, :2]
    th = 0.3
    b = np.zeros((5, 2))
    b[0, 0] = np.cos(th); b[2, 0] = np.sin(th); b[1, 1] = 1.0
    assert abs(metrics.max_principal_sine(a, b) - np.sin(th)) < 1e-14
