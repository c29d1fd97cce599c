"""GPU parity of rBKI-TK-TR (Algorithm 3) through the C ABI against the FP64 oracle.

Both sides start TR-ALS from the same seeded cores (`synth.tr_init_cores`) on the Tucker
core each computed, so they follow the same ALS iterates.  Bar: the same number of sweeps,
per-sweep fits within 1e-9, the contracted TR cores within 1e-7 of their largest entry, and
the full TR reconstructions within 1e-8 relative."""
import numpy as np
import pytest

import synth
from oracle import tr as otr
from oracle.tensor import tr as tr_full

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def rb():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2211_14828_gb300 as rb
    rb.lib()
    return rb


def _tr_tensor(dims, tr_rank, snr_db, seed):
    g = np.random.default_rng(seed)
    n = len(dims)
    rr = [tr_rank] * n if np.isscalar(tr_rank) else list(tr_rank)
    cores = [g.standard_normal((rr[k - 1], dims[k], rr[k])) for k in range(n)]
    clean = synth.tr_full(cores)
    return synth.add_noise_snr(clean, snr_db, g, dtype=np.float64)


def _run_both(rb, x, tucker_ranks, p, q, seed, tr_ranks, maxit=20, tol=1e-3, init_seed=7):
    init = synth.tr_init_cores(init_seed, tucker_ranks, tr_ranks)
    want = otr.rbki_tk_tr(x, tucker_ranks, p, q, seed, init, maxit, tol)
    got = rb.rbki_htr(torch.from_numpy(x).cuda(), tucker_ranks, p, q, seed, tr_ranks,
                      [torch.from_numpy(c).cuda() for c in init], maxit=maxit, tol=tol, prec="fp64")
    torch.cuda.synchronize()
    return want, got


def _check(want, got, maxit, unique=True):
    """unique=False: some ALS update is underdetermined (prod_{j!=k} R_j < r_{k-1} r_k), so
    the cores are not unique; then only the fits and the reconstruction are compared, and
    the fits to 1e-7: the GPU solves the singular normal equations with a diagonal shift of
    1e-12 trace/S, which leaves a residual of about 1e-9 |G| where the oracle's
    minimum-norm least squares leaves rounding."""
    fits = got["fits"].cpu().numpy()
    nsweeps = int(np.sum(~np.isnan(fits)))
    assert nsweeps == len(want["fits"]), (fits, want["fits"])
    assert np.all(np.isnan(fits[nsweeps:]))
    np.testing.assert_allclose(fits[:nsweeps], want["fits"], rtol=0, atol=1e-9 if unique else 1e-7)
    cores = [c.cpu().numpy() for c in got["cores"]]
    for c, w in zip(cores, want["cores"]):
        assert c.shape == w.shape
        if unique:
            np.testing.assert_allclose(c, w, rtol=0, atol=1e-7 * np.abs(w).max())
    a, b = tr_full(cores), tr_full(want["cores"])
    assert np.linalg.norm(a - b) <= 1e-8 * np.linalg.norm(b)


@pytest.mark.parametrize("case", [
    # dims, tucker ranks, p, q, TR ranks
    ((24, 24, 24, 24), (6, 6, 6, 6), 2, 1, (3, 3, 3, 3)),          # Krylov path, uniform ring
    ((20, 25, 30), (5, 6, 7), 2, 1, (2, 3, 4)),                    # ragged TR and Tucker ranks
    ((40, 36), (6, 5), 3, 1, (2, 3)),                              # order 2: 5 < 2*3, cores not unique
    ((30, 26, 22), (9, 9, 9), 3, 1, (8, 8, 8)),                    # largest supported TR rank
    ((8, 8, 8, 8, 8, 8), (5, 5, 5, 5, 5, 5), 2, 1, (4,) * 6),      # order 6, Gram path per mode
])
def test_htr_matches_oracle(rb, case):
    dims, tk, p, q, trr = case
    x = _tr_tensor(dims, max(trr), 15.0, seed=sum(dims))
    want, got = _run_both(rb, x, tk, p, q, seed=42, tr_ranks=trr)
    n = len(dims)
    unique = all(np.prod(tk) // tk[k] >= trr[k - 1] * trr[k] for k in range(n))
    _check(want, got, 20, unique)


def test_htr_maxit_and_tucker_out(rb):
    """tr_maxit = 2 stops after two sweeps; the intermediate Tucker result is returned."""
    dims, tk, trr = (24, 20, 28), (6, 5, 7), (3, 2, 4)
    x = _tr_tensor(dims, trr, 10.0, seed=3)
    want, got = _run_both(rb, x, tk, 2, 1, seed=5, tr_ranks=trr, maxit=2, tol=0.0)
    _check(want, got, 2)
    core = got["tucker"]["core"].cpu().numpy()
    np.testing.assert_allclose(core, want["tucker"]["core"], rtol=0, atol=1e-10 * np.abs(core).max())


def test_htr_workload_16_6(rb):
    """The 6th-order 16^6 workload (TR rank 6 + noise at 15 dB, Tucker rank 10, p = 5, q = 2):
    every mode takes the Gram path; TR-ALS on the 10^6 core."""
    wl = synth.config_htr()
    x = wl.x.astype(np.float64)
    init = wl.tr_init
    want = otr.rbki_tk_tr(x, wl.ranks, wl.p, wl.q, wl.seed, init, 20, 1e-3)
    got = rb.rbki_htr(torch.from_numpy(wl.x).cuda(), wl.ranks, wl.p, wl.q, wl.seed, wl.tr_ranks,
                      [torch.from_numpy(c).cuda() for c in init], maxit=20, tol=1e-3, prec="fp64")
    torch.cuda.synchronize()
    _check(want, got, 20)


def test_htr_rejects_bad_ranks(rb):
    x = torch.zeros((8, 8, 8), dtype=torch.float64, device="cuda")
    init = [torch.zeros((9, 4, 9), dtype=torch.float64, device="cuda") for _ in range(3)]
    with pytest.raises(rb.RbkiError):
        rb.rbki_htr(x, (4, 4, 4), 1, 1, 0, (9, 9, 9), init)


@pytest.mark.parametrize("case", [
    # dims, tucker ranks, p, q, TR ranks
    ((24, 24, 24, 24), (6, 6, 6, 6), 2, 1, (2, 3, 3, 2)),
    ((20, 25, 30), (8, 6, 7), 2, 1, (2, 3, 4)),
    ((16,) * 6, (10,) * 6, 5, 2, (3, 3, 3, 3, 3, 3)),
])
def test_htr_tr_svd_matches_oracle(rb, case):
    """TR-SVD instead of TR-ALS (RBKI_FLAG_TR_SVD): the ring's fit and its full
    reconstruction against the oracle's TR-SVD of the oracle's Tucker core (the cores
    themselves are fixed only up to rotations of each bond)."""
    dims, tk, p, q, trr = case
    x = _tr_tensor(dims, max(trr), 15.0, seed=sum(dims) + 1)
    want = otr.rbki_tk_tr(x, tk, p, q, 42, None, tr_ranks=trr)
    got = rb.rbki_htr(torch.from_numpy(x).cuda(), tk, p, q, 42, trr, None, maxit=4, prec="fp64",
                      flags=rb.FLAG_TR_SVD)
    torch.cuda.synchronize()
    fits = got["fits"].cpu().numpy()
    assert abs(fits[0] - want["fits"][0]) <= 1e-9 and np.all(np.isnan(fits[1:]))
    cores = [c.cpu().numpy() for c in got["cores"]]
    for c, w in zip(cores, want["cores"]):
        assert c.shape == w.shape
    a, b = tr_full(cores), tr_full(want["cores"])
    assert np.linalg.norm(a - b) <= 1e-8 * np.linalg.norm(b)
