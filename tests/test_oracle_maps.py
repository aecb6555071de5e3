"""Pins of projection, binning and the per-pixel solve (paper Eq. `todmodel`
g P m term; Sect. 5 table rows "TOD binning" and "Map solution")."""
import numpy as np
import pytest

import oracle
import synth


def test_projection_binning_adjoint():
    """<P m, y> = <m, P^T y> with P^T the binning of y (unit weights)."""
    rng = np.random.default_rng(0)
    npix, n = 500, 20000
    pix = rng.integers(0, npix, n)
    psi = rng.integers(0, 4096, n)
    m = rng.standard_normal((3, npix))
    y = rng.standard_normal(n)
    lhs = np.dot(oracle.project(m, pix, psi), y)
    _, b = oracle.bin_maps(npix, pix, psi, y, (np.ones(n), np.ones(n)))
    rhs = np.sum(m.T * b)
    assert lhs == pytest.approx(rhs, rel=1e-12)


def test_trig_table_definition():
    c, s = oracle.psi_trig_table()
    b = np.array([0, 1, 1023, 2048, 4095])
    psi = (b + 0.5) * 2 * np.pi / 4096
    assert np.allclose(c[b], np.cos(2 * psi), atol=1e-7)
    assert np.allclose(s[b], np.sin(2 * psi), atol=1e-7)
    assert np.all(c.astype(np.float32) == c)        # FP32-representable


def test_noiseless_round_trip_returns_map(tiny_band, tiny_ingest):
    """d = g P m with no noise, correct gains: binning then solving returns
    m on every valid pixel to 1e-10 relative, and nearly all pixels are valid."""
    ing, band = tiny_ingest, tiny_band
    off = ing["offsets"]
    pix = oracle.decode_band(ing["pix_streams"], off, 1)
    psi = oracle.decode_band(ing["psi_streams"], off, 1)
    g = oracle.per_sample(band.gain, off)
    d = oracle.project(band.map_tqu, pix, psi, g)
    sigma0 = 1e-3
    w = g ** 2 / sigma0 ** 2
    v = g / sigma0 ** 2
    A, b = oracle.bin_maps(band.npix, pix, psi, d, (w, v))
    hits = np.bincount(pix, minlength=band.npix)
    m, had, valid = oracle.solve_maps(A, b, hits)
    ok = valid > 0
    assert ok.sum() >= band.npix - 3
    err = np.abs(m[:, ok] - band.map_tqu[:, ok]).max(axis=1) / np.abs(band.map_tqu).max(axis=1)
    assert np.all(err < 1e-10)


def test_solve_exact_on_constructed_spd():
    rng = np.random.default_rng(1)
    npix = 200
    Ms = []
    A6 = np.empty((npix, 6))
    for p in range(npix):
        B = rng.standard_normal((3, 3))
        M = B @ B.T + 0.5 * np.eye(3)
        Ms.append(M)
        A6[p] = (M[0, 0], M[0, 1], M[0, 2], M[1, 1], M[1, 2], M[2, 2])
    x = rng.standard_normal((npix, 3))
    b = np.stack([Ms[p] @ x[p] for p in range(npix)])
    m, had, valid = oracle.solve_maps(A6, b, np.full(npix, 10), rcond_min=0.0)
    assert valid.all()
    assert np.allclose(m.T, x, rtol=1e-12, atol=1e-12)
    dets = np.array([np.linalg.det(M) / (M[0, 0] * M[1, 1] * M[2, 2]) for M in Ms])
    assert np.allclose(had, dets, rtol=1e-12)


def test_solve_validity_rule_edges():
    M = np.diag([4.0, 1.0, 1.0])
    M[1, 2] = M[2, 1] = np.sqrt(1 - 1e-6)         # Hadamard ratio exactly ~1e-6
    A6 = np.tile([M[0, 0], 0, 0, M[1, 1], M[1, 2], M[2, 2]], (4, 1)).astype(float)
    had = np.linalg.det(M) / 4.0
    b = np.ones((4, 3))
    m, h, valid = oracle.solve_maps(A6, b, np.array([3, 2, 3, 3]), rcond_min=had * (1 - 1e-9))
    assert list(valid[:3]) == [1, 0, 1]
    m2, _, valid2 = oracle.solve_maps(A6, b, np.array([3, 3, 3, 3]), rcond_min=had * (1 + 1e-6))
    assert not valid2.any() and not m2.any()
    assert not m[:, 1].any()
