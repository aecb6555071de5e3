"""Pins of the oracle's joint gain draw under the smooth prior across scans
(row A12; the per-detscan gain conditional of Eq. `gibbsstart` times a
Gaussian prior diagonal in the DCT basis of the scan index): the flat-prior
limit (independent per-scan draws), the constant-noise case (a diagonal
Wiener filter in the DCT basis), brute-force posterior moments for two
scans, the draw's covariance, and its normals."""
import math

import numpy as np
import pytest
import scipy.fft as sfft
from scipy import stats

import oracle


def _inputs(S, seed=0, sig_lo=0.8e-3, sig_hi=1.5e-3):
    rng = np.random.default_rng(seed)
    mu = 1.0 + 0.01 * np.cumsum(rng.standard_normal(S)) / math.sqrt(S) + 1e-3 * rng.standard_normal(S)
    sigma = rng.uniform(sig_lo, sig_hi, S)
    return mu, sigma


def test_flat_prior_gives_independent_draws():
    mu, sigma = _inputs(50)
    w1, w2 = oracle.gain_smooth_normals(7, 1, 2, 3, 50)
    g = oracle.sample_gain_smooth(mu, sigma, 1e9, -2.0, w1, w2)
    np.testing.assert_allclose(g, mu + sigma * w1, rtol=0, atol=1e-12)
    gm = oracle.sample_gain_smooth(mu, sigma, 1e9, -2.0, w1, w2, mode=oracle.MODE_MEAN)
    np.testing.assert_allclose(gm, mu, rtol=0, atol=1e-12)


@pytest.mark.parametrize("S,alpha", [(64, -2.0), (1000, -1.0), (37, -3.0)])
def test_constant_noise_is_a_dct_wiener_filter(S, alpha):
    mu, _ = _inputs(S, 1)
    sig, sg = 1e-3, 2e-3
    a = 1.0 / sig ** 2
    k = np.arange(S, dtype=np.float64)
    lam = np.zeros(S)
    lam[1:] = 1.0 / (sg ** 2 * k[1:] ** alpha)
    want = sfft.idct(sfft.dct(mu, norm="ortho") * a / (a + lam), norm="ortho")
    got = oracle.sample_gain_smooth(mu, np.full(S, sig), sg, alpha, None, None, mode=oracle.MODE_MEAN)
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-12)
    # the mean gain passes unchanged (lambda_0 = 0)
    assert got.mean() == pytest.approx(mu.mean(), abs=1e-11)


def test_two_scans_brute_force_posterior():
    """S = 2: the prior says g0 - g1 ~ N(0, 2 sigma_g^2) and nothing about
    g0 + g1; posterior moments by direct integration on a grid."""
    mu = np.array([1.003, 0.998])
    sigma = np.array([2e-3, 1e-3])
    sg = 1.5e-3
    grid = np.linspace(-0.02, 0.02, 1601)
    g0, g1 = np.meshgrid(mu[0] + grid, mu[1] + grid, indexing="ij")
    logp = (-0.5 * ((g0 - mu[0]) / sigma[0]) ** 2 - 0.5 * ((g1 - mu[1]) / sigma[1]) ** 2
            - (g0 - g1) ** 2 / (4 * sg ** 2))
    p = np.exp(logp - logp.max())
    p /= p.sum()
    m = np.array([(p * g0).sum(), (p * g1).sum()])
    cov = np.array([[(p * (g0 - m[0]) ** 2).sum(), (p * (g0 - m[0]) * (g1 - m[1])).sum()],
                    [0, (p * (g1 - m[1]) ** 2).sum()]])
    cov[1, 0] = cov[0, 1]
    got = oracle.sample_gain_smooth(mu, sigma, sg, -2.0, None, None, mode=oracle.MODE_MEAN)
    np.testing.assert_allclose(got, m, rtol=0, atol=1e-8)
    # draws: sample covariance of many draws against the grid covariance
    draws = np.array([oracle.sample_gain_smooth(mu, sigma, sg, -2.0, *oracle.gain_smooth_normals(5, 0, 0, it, 2))
                      for it in range(4000)])
    np.testing.assert_allclose(np.cov(draws.T), cov, rtol=0.1, atol=0.05 * cov[1, 1])


def test_draw_covariance_is_the_posterior_covariance():
    S = 8
    mu, sigma = _inputs(S, 2)
    sg, alpha = 1e-3, -2.0
    # the posterior precision written from the DCT's cosine definition
    q = np.arange(S)
    Cd = np.sqrt(2.0 / S) * np.cos(np.pi * np.outer(q, 2 * q + 1) / (2 * S))
    Cd[0] /= math.sqrt(2.0)
    lam = np.zeros(S)
    lam[1:] = 1.0 / (sg ** 2 * np.arange(1, S) ** alpha)
    A = np.diag(1.0 / sigma ** 2) + Cd.T @ np.diag(lam) @ Cd
    L = np.linalg.cholesky(A)
    mean = oracle.sample_gain_smooth(mu, sigma, sg, alpha, None, None, mode=oracle.MODE_MEAN)
    z = []
    for it in range(600):
        g = oracle.sample_gain_smooth(mu, sigma, sg, alpha, *oracle.gain_smooth_normals(9, 2, 1, it, S))
        z.append(L.T @ (g - mean))                 # N(0, I) if g ~ N(mean, A^-1)
    z = np.concatenate(z)
    assert stats.kstest(z, "norm").pvalue > 1e-3
    assert abs(z.std() - 1.0) < 0.05


def test_normals_are_standard_and_independent():
    w1, w2 = oracle.gain_smooth_normals(3, 4, 1, 9, 3000)
    assert stats.kstest(w1, "norm").pvalue > 1e-3 and stats.kstest(w2, "norm").pvalue > 1e-3
    assert abs(np.corrcoef(w1, w2)[0, 1]) < 0.06
    v1, _ = oracle.gain_smooth_normals(3, 4, 2, 9, 10)          # another detector: another stream
    assert not np.allclose(v1, w1[:10])
