"""HEALPix RING-scheme pixelisation (Gorski et al. 2005, ApJ 622, 759).

Used only to turn the synthetic continuous pointing into pixel indices, the
pre-pixelised pointing stream of paper Sect. 4.1.  Written from the published
equal-area construction: 12 Nside^2 pixels; polar caps |z| > 2/3 with 4i
pixels on ring i; an equatorial belt of 4 Nside pixels per ring.
Vectorised numpy, FP64.
"""
from __future__ import annotations

import numpy as np


def nside2npix(nside: int) -> int:
    return 12 * nside * nside


def ang2pix_ring(nside: int, theta: np.ndarray, phi: np.ndarray) -> np.ndarray:
    """Pixel index (int64) of colatitude theta, longitude phi (radians)."""
    theta = np.asarray(theta, dtype=np.float64)
    phi = np.asarray(phi, dtype=np.float64)
    z = np.cos(theta)
    za = np.abs(z)
    tt = np.mod(phi, 2 * np.pi) * (2.0 / np.pi)          # in [0, 4)
    tt = np.where(tt >= 4.0, tt - 4.0, tt)
    ncap = 2 * nside * (nside - 1)
    npix = 12 * nside * nside
    out = np.empty(z.shape, dtype=np.int64)

    eq = za <= 2.0 / 3.0
    # equatorial belt
    if np.any(eq):
        zq, tq = z[eq], tt[eq]
        t1 = nside * (0.5 + tq)
        t2 = nside * zq * 0.75
        jp = np.floor(t1 - t2).astype(np.int64)      # ascending edge line index
        jm = np.floor(t1 + t2).astype(np.int64)      # descending edge line index
        ir = nside + 1 + jp - jm                     # ring in {1 .. 2nside+1}
        kshift = 1 - (ir & 1)
        ip = (jp + jm - nside + kshift + 1) // 2
        ip = np.mod(ip, 4 * nside)
        out[eq] = ncap + (ir - 1) * 4 * nside + ip
    pol = ~eq
    if np.any(pol):
        zp, tp_all = z[pol], tt[pol]
        tp = tp_all - np.floor(tp_all)
        tmp = nside * np.sqrt(3.0 * (1.0 - np.abs(zp)))
        jp = np.floor(tp * tmp).astype(np.int64)
        jm = np.floor((1.0 - tp) * tmp).astype(np.int64)
        ir = jp + jm + 1                             # ring counted from the nearest pole
        ip = np.floor(tp_all * ir).astype(np.int64)
        ip = np.mod(ip, 4 * ir)
        north = zp > 0
        out_p = np.where(north, 2 * ir * (ir - 1) + ip, npix - 2 * ir * (ir + 1) + ip)
        out[pol] = out_p
    return out


def pix2ang_ring(nside: int, pix: np.ndarray):
    """Centre (theta, phi) of RING pixels."""
    pix = np.asarray(pix, dtype=np.int64)
    npix = 12 * nside * nside
    ncap = 2 * nside * (nside - 1)
    theta = np.empty(pix.shape)
    phi = np.empty(pix.shape)
    fact2 = 4.0 / npix

    n_cap = pix < ncap
    if np.any(n_cap):
        p = pix[n_cap]
        iring = (1 + np.floor(np.sqrt(1 + 2 * p)).astype(np.int64)) >> 1
        # guard float rounding of sqrt
        iring = np.where(2 * iring * (iring - 1) > p, iring - 1, iring)
        iring = np.where(2 * (iring + 1) * iring <= p, iring + 1, iring)
        iphi = p + 1 - 2 * iring * (iring - 1)
        z = 1.0 - iring * iring * fact2
        theta[n_cap] = np.arccos(z)
        phi[n_cap] = (iphi - 0.5) * (np.pi / 2) / iring
    s_cap = pix >= npix - ncap
    if np.any(s_cap):
        p = npix - pix[s_cap]
        iring = (1 + np.floor(np.sqrt(2 * p - 1)).astype(np.int64)) >> 1
        iring = np.where(2 * iring * (iring - 1) >= p, iring - 1, iring)
        iring = np.where(2 * (iring + 1) * iring < p, iring + 1, iring)
        iphi = 4 * iring + 1 - (p - 2 * iring * (iring - 1))
        z = -1.0 + iring * iring * fact2
        theta[s_cap] = np.arccos(z)
        phi[s_cap] = (iphi - 0.5) * (np.pi / 2) / iring
    belt = ~(n_cap | s_cap)
    if np.any(belt):
        ip = pix[belt] - ncap
        iring = ip // (4 * nside) + nside
        iphi = np.mod(ip, 4 * nside) + 1
        fodd = np.where(((iring + nside) & 1) == 1, 1.0, 0.5)
        z = (2 * nside - iring) * (2.0 / (3.0 * nside))
        theta[belt] = np.arccos(z)
        phi[belt] = (iphi - fodd) * np.pi / (2.0 * nside)
    return theta, phi
