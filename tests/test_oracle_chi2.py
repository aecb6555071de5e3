"""Pins of the oracle's TOD chi^2 and its gradients: central finite
differences in FP64 (relative 1e-4 or better), and the closed form of the
white-noise limit."""
import numpy as np
import pytest

import oracle


def _case(seed=0, n=96):
    rng = np.random.default_rng(seed)
    npix = 40
    pix = rng.integers(0, npix, n)
    psi = rng.integers(0, 4096, n)
    m = rng.standard_normal((3, npix)) * 1e-4
    s = oracle.project(m, pix, psi)
    mask = np.ones(n)
    mask[10:14] = 0
    d = 1.01 * s + 1e-3 * rng.standard_normal(n)
    return rng, npix, pix, psi, m, d, mask


def test_chi2_gradient_gain_and_psd_fd():
    _, _, pix, psi, m, d, mask = _case()
    s = oracle.project(m, pix, psi)
    th = (1.1e-3, 0.12, -1.4)
    g = 1.02
    r = oracle.chi2_detscan(d, s, g, mask, *th, 32.5)
    h = 1e-6
    num_g = (oracle.chi2_detscan(d, s, g + h, mask, *th, 32.5)["L"]
             - oracle.chi2_detscan(d, s, g - h, mask, *th, 32.5)["L"]) / (2 * h)
    assert r["dg"] == pytest.approx(num_g, rel=1e-5)
    for i in range(3):
        tp, tm = list(th), list(th)
        step = 1e-6 * abs(th[i])
        tp[i] += step
        tm[i] -= step
        num = (oracle.chi2_detscan(d, s, g, mask, *tp, 32.5)["L"]
               - oracle.chi2_detscan(d, s, g, mask, *tm, 32.5)["L"]) / (2 * step)
        assert r["dpsd"][i] == pytest.approx(num, rel=1e-4)


def test_chi2_gradient_map_fd():
    _, npix, pix, psi, m, d, mask = _case(1)
    off = np.array([0, 48, 96])
    gains = np.array([1.01, 0.99])
    psd = np.array([[1e-3, 0.1, -1.5], [1.2e-3, 0.05, -1.2]])
    res = oracle.chi2_band(m, pix, psi, d, gains, mask, psd, off, 2, 32.5)
    rng = np.random.default_rng(2)
    for _ in range(6):
        i, p = rng.integers(0, 3), rng.integers(0, npix)
        h = 1e-9
        mp, mm = m.copy(), m.copy()
        mp[i, p] += h
        mm[i, p] -= h
        num = (oracle.chi2_band(mp, pix, psi, d, gains, mask, psd, off, 2, 32.5)["L"]
               - oracle.chi2_band(mm, pix, psi, d, gains, mask, psd, off, 2, 32.5)["L"]) / (2 * h)
        assert res["dm"][i, p] == pytest.approx(num, rel=1e-4, abs=1e-6 * np.abs(res["dm"]).max())


def test_chi2_white_noise_limit():
    """alpha -> very negative, fknee -> 0: P -> sigma0^2 for k >= 1, so
    L = 1/2 (|M r|^2 - rhat_0^2)/sigma0^2 + (n-1) ln sigma0 (Parseval)."""
    n = 64
    rng = np.random.default_rng(3)
    d = rng.standard_normal(n)
    s = np.zeros(n)
    mask = np.ones(n)
    r = oracle.chi2_detscan(d, s, 1.0, mask, 2.0, 1e-12, -1.0, 32.5)
    rh0 = oracle.dct(d)[0]
    want = 0.5 * (np.dot(d, d) - rh0 ** 2) / 4.0 + (n - 1) * np.log(2.0)
    assert r["L"] == pytest.approx(want, rel=1e-9)
