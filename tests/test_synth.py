"""Pins for the seeded input generators (synth), which hold no arithmetic of the method:
DCT-II factors against SciPy's orthonormal DCT, Haar factors orthonormal with a positive
R diagonal, Tucker data of the stated multilinear rank, tensor rings equal to the oracle's
independent ring contraction, and the served stream within its stated ranges."""
import numpy as np
import pytest

import synth
from oracle.tensor import tr as oracle_tr
from oracle.tensor import unfold


def test_dct_factor_is_the_orthonormal_dct2_basis():
    scipy_fft = pytest.importorskip("scipy.fft")
    for rows, cols in ((16, 5), (64, 64), (37, 9)):
        u = synth.dct_factor(rows, cols)
        full = scipy_fft.dct(np.eye(rows), type=2, norm="ortho", axis=0)   # rows: frequencies
        np.testing.assert_allclose(u, full[:cols].T, atol=1e-12)
        np.testing.assert_allclose(u.T @ u, np.eye(cols), atol=1e-12)


def test_haar_factor_orthonormal_positive_r():
    g = synth.rng(3)
    u = synth.haar_factor(g, 50, 7)
    np.testing.assert_allclose(u.T @ u, np.eye(7), atol=1e-13)
    _, r = np.linalg.qr(u)
    assert np.all(np.abs(np.abs(np.diag(r)) - 1.0) < 1e-12)


def test_tucker_data_has_the_stated_multilinear_rank():
    g = synth.rng(4)
    core = g.standard_normal((3, 4, 2))
    facs = [synth.haar_factor(g, n, r) for n, r in ((20, 3), (15, 4), (10, 2))]
    x = synth.tucker_full(core, facs)
    for n, r in enumerate((3, 4, 2)):
        s = np.linalg.svd(unfold(x, n), compute_uv=False)
        assert s[r - 1] > 1e-8 * s[0] and (len(s) == r or s[r] < 1e-12 * s[0])


def test_tensor_ring_matches_oracle_contraction():
    g = synth.rng(5)
    ranks = (2, 3, 4)
    dims = (5, 6, 7)
    cores = [g.standard_normal((ranks[k - 1], dims[k], ranks[k])) for k in range(3)]
    np.testing.assert_allclose(synth.tr_full(cores), oracle_tr(cores), atol=1e-12)


def test_served_stream_ranges():
    reqs = synth.serve_stream(n_requests=64, seed=11)
    assert len(reqs) == 64
    for r in reqs:
        d = r["dims"] if isinstance(r, dict) else r.dims
        rk = r["ranks"] if isinstance(r, dict) else r.ranks
        q = r["q"] if isinstance(r, dict) else r.q
        assert all(32 <= v <= 256 for v in d)
        assert all(1 <= a <= b for a, b in zip(rk, d))
        assert q in (1, 2, 3)
