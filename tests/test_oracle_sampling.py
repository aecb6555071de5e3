"""Pins of the oracle's gain and correlated-noise steps (readings of paper
the gain and n_corr conditionals of Eq. `gibbsstart` and Sect. 5 CG gap
filling)."""
import math

import numpy as np
import pytest
from scipy import stats

import oracle

FS = 32.5


def _setup(n, seed, flag_slices=()):
    rng = np.random.default_rng(seed)
    s = rng.standard_normal(n) * 1e-4
    mask = np.ones(n)
    for a, b in flag_slices:
        mask[a:b] = 0
    return rng, s, mask


def test_gain_zero_noise_returns_true_gain():
    """With d = g s exactly, mean b/a = g whatever the weights."""
    rng, s, mask = _setup(4096, 0, [(100, 300), (2000, 2050)])
    P = oracle.noise_psd(4096, FS, 1e-3, 0.1, -1.7)
    for g in (0.97, 1.0, 1.013):
        gg, mu, sig = oracle.sample_gain(s, g * s, mask, P, 0.0, oracle.MODE_MEAN)
        assert mu == pytest.approx(g, rel=1e-12) and gg == mu


def test_gain_mean_variance_matches_conditional():
    """No flags, noise drawn from the model PSD P: the estimator b/a is
    unbiased with variance 1/a.  A wrong weighting (1/P^2, dropping 1/P,
    keeping mode 0) fails this."""
    n = 2048
    rng, s, mask = _setup(n, 1)
    s = s + 3e-4 * np.cos(np.arange(n) / 40.0)          # some low-frequency signal
    P = oracle.noise_psd(n, FS, 1e-3, 0.2, -1.5)
    g = 1.01
    mus = []
    for i in range(1500):
        nk = rng.standard_normal(n) * np.sqrt(np.where(np.isinf(P), 1.0, P))
        nk[0] = rng.standard_normal() * 10.0               # arbitrary offset: must not matter
        d = g * s + oracle.idct(nk)
        _, mu, sig = oracle.sample_gain(s, d, mask, P, 0.0)
        mus.append(mu)
    mus = np.array(mus)
    assert abs(mus.mean() - g) < 4 * sig / math.sqrt(len(mus))
    assert mus.var() == pytest.approx(sig ** 2, rel=0.12)


def test_gain_draw_standardised_is_normal():
    rng, s, mask = _setup(512, 2, [(10, 40)])
    d = 1.02 * s + 1e-3 * rng.standard_normal(512)
    P = oracle.noise_psd(512, FS, 1e-3, 0.1, -1.0)
    zs = []
    for q in range(4000):
        z = oracle.gain_normal(17, 0, q, 0)
        g, mu, sig = oracle.sample_gain(s, d, mask, P, z)
        zs.append((g - mu) / sig)
    assert stats.kstest(zs, "norm").pvalue > 1e-3


@pytest.mark.parametrize("flags", [(), ((5, 9),), ((0, 3), (20, 31), (60, 64))])
def test_ncorr_pcg_matches_dense_bruteforce(flags):
    """n <= 64: PCG (and the diagonal solve when gap-free) equals a dense
    Cholesky solve of the explicit A = C^T diag(phi) C + M/sigma0^2."""
    n = 64
    rng, s, mask = _setup(n, 3, flags)
    phi = oracle.corr_inv_psd(n, FS, 1e-3, 0.15, -1.6)
    b = rng.standard_normal(n) * 1e3
    xd = oracle.ncorr_solve_dense(b, mask, 1e-3, phi)
    xp, it = oracle.ncorr_solve_pcg(b, mask, 1e-3, phi)
    assert it > 0 or not flags
    assert np.allclose(xp, xd, rtol=0, atol=1e-9 * np.abs(xd).max())
    if not flags:
        xg = oracle.ncorr_solve_gapfree(b, 1e-3, phi)
        assert np.allclose(xg, xd, rtol=0, atol=1e-10 * np.abs(xd).max())


def test_ncorr_all_flagged_is_minimum_norm_dense_solution():
    """Every sample flagged: A = C^T diag(phi) C is singular (phi_0 = 0, the
    offset).  The draw equals the minimum-norm solution of the explicit
    dense system (pseudo-inverse), and has no offset component."""
    n = 60
    rng = np.random.default_rng(8)
    phi = oracle.corr_inv_psd(n, FS, 1e-3, 0.12, -1.4)
    w2 = rng.standard_normal(n)
    r = rng.standard_normal(n) * 1e-3
    mask = np.zeros(n)
    b = oracle.ncorr_rhs(r, mask, 1e-3, phi, rng.standard_normal(n), w2)
    A = oracle.ncorr_dense_A(n, mask, 1e-3, phi)
    xref = np.linalg.pinv(A, rcond=1e-12) @ b
    x, it = oracle.sample_ncorr(r, np.zeros(n), 1.0, mask, 1e-3, 0.12, -1.4, FS, rng.standard_normal(n), w2)
    assert it == 0
    assert np.allclose(x, xref, rtol=0, atol=1e-9 * np.abs(xref).max())
    assert abs(x.sum()) <= 1e-9 * np.abs(x).sum()


def test_ncorr_mean_is_wiener_interpolation():
    """MODE_MEAN: A^{-1} M r / sigma^2 equals the textbook Gaussian
    conditional mean F_{.o} (F_oo + sigma^2 I)^{-1} r_o of the correlated
    noise given the unflagged residual (F = C^T diag(1/phi) C).  Checked with
    phi_0 > 0 so that F exists."""
    n = 48
    sigma = 1e-3
    rng, _, mask = _setup(n, 4, [(10, 17), (30, 33)])
    phi = oracle.corr_inv_psd(n, FS, sigma, 0.3, -1.3)
    phi[0] = phi[1]
    C = np.stack([oracle.dct(e) for e in np.eye(n)], axis=1)
    F = C.T @ np.diag(1.0 / phi) @ C
    r = rng.standard_normal(n) * 1e-3
    o = mask > 0
    wiener = F[:, o] @ np.linalg.solve(F[np.ix_(o, o)] + sigma ** 2 * np.eye(o.sum()), r[o])
    b = oracle.ncorr_rhs(r, mask, sigma, phi, np.zeros(n), np.zeros(n))
    x, _ = oracle.ncorr_solve_pcg(b, mask, sigma, phi)
    assert np.allclose(x, wiener, atol=1e-10 * np.abs(wiener).max())


def test_ncorr_draw_has_posterior_covariance():
    """x - x_mean ~ N(0, A^{-1}): whitening by L^T (A = L L^T) gives iid
    N(0,1).  Pins the two noise terms of the right-hand side."""
    n = 32
    sigma = 1e-3
    rng, _, mask = _setup(n, 5, [(4, 9)])
    fs, fk, al = FS, 0.2, -1.4
    phi = oracle.corr_inv_psd(n, fs, sigma, fk, al)
    A = oracle.ncorr_dense_A(n, mask, sigma, phi)
    L = np.linalg.cholesky(A)
    d = rng.standard_normal(n) * 1e-3
    s = np.zeros(n)
    xm, _ = oracle.sample_ncorr(d, s, 1.0, mask, sigma, fk, al, fs, np.zeros(n), np.zeros(n))
    ws = []
    for q in range(600):
        w1 = oracle.stream_normals(9, 0, q, oracle.PURPOSE_NC_W1, 0, n)
        w2 = oracle.stream_normals(9, 0, q, oracle.PURPOSE_NC_W2, 0, n)
        x, _ = oracle.sample_ncorr(d, s, 1.0, mask, sigma, fk, al, fs, w1, w2)
        ws.append(L.T @ (x - xm))
    ws = np.concatenate(ws)
    assert abs(ws.std() - 1) < 0.03
    assert stats.kstest(ws, "norm").pvalue > 1e-3


def test_ncorr_pcg_converges_on_lfi_like_detscan():
    n = oracle.fft_length(20000)
    rng = np.random.default_rng(6)
    mask = np.ones(n)
    mask[1000:1400] = 0
    mask[9000:9050] = 0
    phi = oracle.corr_inv_psd(n, FS, 1e-3, 0.2, -2.0)
    b = rng.standard_normal(n) * 1e6
    x, it = oracle.ncorr_solve_pcg(b, mask, 1e-3, phi)
    assert 0 < it < 500
    res = oracle.ncorr_apply_A(x, mask, 1e-3, phi) - b
    assert np.linalg.norm(res) <= 1e-11 * np.linalg.norm(b)
