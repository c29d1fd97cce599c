"""Pins for partial column sampling (oracle.sampling, Sec. 3.2 after Table 2, Fig. 5).

* Y is exactly the chosen columns of X_(n) (brute-force loops over the tensor's entries).
* omega = 1 on tile-aligned shapes: Y = X_(n) and the sampled method is the unsampled one.
* selection: m_u distinct units in ascending order; over many seeds each unit is kept with
  frequency m_u / U (binomial bound); modes draw independent subsets.
* Fig. 5: on the (N=3, I=200, R=10, SNR=-5 dB) Gaussian tensor the fit at omega = 0.1 is
  about 85% (q = 2, p = 5) and grows with omega toward the unsampled method's."""
import numpy as np
import pytest

import synth
from oracle import metrics, philox, rbki, sampling
from oracle.tensor import unfold


def _brute_y(x, n, units):
    shape = x.shape
    a_n = int(np.prod(shape[:n]))
    c_n = int(np.prod(shape[n + 1:]))
    rest = [k for k in range(x.ndim) if k != n]
    y = np.zeros((shape[n], 128 * len(units)))
    for j, u in enumerate(units):
        for t in range(128):
            if c_n > 1:
                nb = -(-c_n // 128)
                a, c = u // nb, (u % nb) * 128 + t
                if c >= c_n:
                    continue
                col = a * c_n + c
            else:
                col = u * 128 + t
                if col >= a_n:
                    continue
            idx = np.unravel_index(col, [shape[k] for k in rest])    # C-order column index
            for i in range(shape[n]):
                full = [0] * x.ndim
                full[n] = i
                for k, v in zip(rest, idx):
                    full[k] = v
                y[i, j * 128 + t] = x[tuple(full)]
    return y


@pytest.mark.parametrize("shape", [(5, 6, 300), (7, 20, 19), (300, 4, 1), (3, 5, 7, 40)])
def test_sampled_unfolding_brute_force(shape):
    g = synth.rng(3)
    x = g.standard_normal(shape)
    for n in range(x.ndim):
        nu = sampling.unit_count(shape, n)
        units = sampling.sample_units(11, n, nu, sampling.kept_units(0.5, nu))
        np.testing.assert_array_equal(sampling.sampled_unfolding(x, n, units), _brute_y(x, n, units))


def test_full_rate_on_aligned_shape_is_the_unsampled_method():
    g = synth.rng(5)
    x = synth.gaussian_tucker(g, 3, 128, 4) + 0.1 * g.standard_normal((128, 128, 128))
    for n in range(3):
        y, units = sampling.sampled_mode(x, n, 9, 1.0)
        np.testing.assert_array_equal(units, np.arange(sampling.unit_count(x.shape, n)))
        np.testing.assert_array_equal(y, unfold(x, n))
    # omega just below 1 keeps every unit here (ceil), so the sampled path runs and must
    # equal the unsampled decomposition
    a = rbki.rbki_tucker(x, [4, 4, 4], 3, 1, 9, omega=0.9999)
    b = rbki.rbki_tucker(x, [4, 4, 4], 3, 1, 9)
    for u, v in zip(a["factors"], b["factors"]):
        np.testing.assert_allclose(u, v, atol=1e-12)
    np.testing.assert_allclose(a["core"], b["core"], atol=1e-10)


def test_selection_size_order_and_uniformity():
    nu, m_u = 40, 10
    counts = np.zeros(nu)
    for seed in range(2000):
        s = sampling.sample_units(seed, 1, nu, m_u)
        assert len(s) == m_u and len(set(s.tolist())) == m_u and np.all(np.diff(s) > 0)
        assert s.min() >= 0 and s.max() < nu
        counts[s] += 1
    p = m_u / nu
    sd = np.sqrt(2000 * p * (1 - p))
    assert np.all(np.abs(counts - 2000 * p) <= 5 * sd)
    keys = sampling.unit_keys(5, 1, nu)
    s = sampling.sample_units(5, 1, nu, m_u)
    rest = np.setdiff1d(np.arange(nu), s)
    assert keys[s].max() <= keys[rest].min()      # the kept units hold the smallest keys
    # modes and seeds draw different subsets; the keys are the Philox words of reading c22
    assert not np.array_equal(sampling.sample_units(1, 0, nu, m_u), sampling.sample_units(1, 1, nu, m_u))
    k = sampling.unit_keys(77, 2, 5)
    r0, _, _, _ = philox.philox4x32_10(([3], [0], [2], [0x53414D50]), (77, 0))
    assert int(k[3]) == int(r0[0])
    assert sampling.kept_units(0.1, 313) == 32 and sampling.kept_units(1e-9, 5) == 1


def test_fig5_fit_at_low_sampling_rate():
    g = synth.rng(100)
    clean = synth.gaussian_tucker(g, 3, 200, 10)
    x = synth.add_noise_snr(clean, -5.0, g)
    fits = {}
    for om in (0.1, 0.5, 1.0):
        out = rbki.rbki_tucker(x, [10] * 3, 5, 2, 42, omega=om)
        fits[om] = metrics.fit(clean, rbki.reconstruct(out["core"], out["factors"]))
    assert 80.0 <= fits[0.1] <= 90.0            # Fig. 5: about 85% at omega = 0.1
    assert fits[0.1] < fits[0.5] < fits[1.0] + 0.05
