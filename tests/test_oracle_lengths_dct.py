"""Pins of the FFT-length rule (paper Sect. 4.2) and the DCT-II
(mirror-equivalent FFT, paper Sect. 4.2)."""
import math

import numpy as np
import pytest

import oracle


def _smooth_even(k):
    if k < 2 or k % 2:
        return False
    for p in (2, 3, 5):
        while k % p == 0:
            k //= p
    return k == 1


def test_fft_length_brute_force():
    for n in list(range(0, 3000)) + [90000, 115321, 140000, 299999]:
        got = oracle.fft_length(n)
        want = max([k for k in range(2, n + 1) if _smooth_even(k)], default=0) if n < 3000 else None
        if want is not None:
            assert got == want
        else:
            assert _smooth_even(got) and got <= n
            assert not any(_smooth_even(k) for k in range(got + 1, n + 1))


@pytest.mark.parametrize("n", [1, 2, 3, 8, 30, 64, 100])
def test_dct_matches_definition(n):
    x = np.random.default_rng(n).standard_normal(n)
    assert np.allclose(oracle.dct(x), oracle.dct_direct(x), rtol=0, atol=1e-12)


@pytest.mark.parametrize("n", [8, 60, 250])
def test_dct_is_mirrored_fft(n):
    """Paper Sect. 4.2: double the array with its mirror image, FFT.  The
    half-sample-symmetric extension's FFT equals 2 e^{i pi k/2n} times the
    unnormalised DCT-II, and its bin n is exactly zero."""
    x = np.random.default_rng(n + 1).standard_normal(n)
    y = np.concatenate([x, x[::-1]])
    F = np.fft.fft(y)
    k = np.arange(n)
    unnorm = np.real(F[:n] * np.exp(-1j * np.pi * k / (2 * n))) / 2
    w = np.full(n, math.sqrt(2.0 / n))
    w[0] = math.sqrt(1.0 / n)
    assert np.allclose(w * unnorm, oracle.dct(x), atol=1e-12)
    assert abs(F[n]) < 1e-9


def test_dct_orthonormal_and_inverse():
    rng = np.random.default_rng(5)
    x = rng.standard_normal(1200)
    X = oracle.dct(x)
    assert np.isclose(np.dot(x, x), np.dot(X, X), rtol=1e-13)
    assert np.allclose(oracle.idct(X), x, atol=1e-12)
    y = rng.standard_normal(1200)
    assert np.isclose(np.dot(oracle.dct(x), y), np.dot(x, oracle.idct(y)), rtol=1e-12)
