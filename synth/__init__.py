"""Seeded synthetic inputs shaped like Planck LFI time-ordered data.

This module is the ONLY code shared by the FP64 oracle (``oracle/``) and the
GPU library (``paper_2201_03509_gb300``).  It holds none of the Gibbs TOD
step's arithmetic: it draws a sky map, a scan strategy, detector pointing,
gains, noise parameters, flags and the raw detector timelines.  Everything the
method computes (length rule, compression, projection, transforms, sampling,
binning, solving) lives on each side separately.

The workloads stand in for the Planck LFI 30/44/70 GHz data (sample rates,
hour-long pointing periods, HEALPix Nside 512/1024, n_psi = 4096; paper
Sect. 4.1), which are not available here.

Randomness: every array is drawn from ``numpy.random.Generator(Philox)``
streams keyed by ``(seed, purpose)``.  These are input-generation draws only;
the draws the sampler itself makes (gain z, n_corr omega) are produced by each
side's own counter-based Philox implementation.
"""
from __future__ import annotations

import dataclasses
import math
import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np

from .healpix import ang2pix_ring, pix2ang_ring, nside2npix  # noqa: F401

N_PSI = 4096

# purposes for the input-generation streams
_P_MAP, _P_LEN, _P_GAIN, _P_NOISEPAR, _P_FLAGS, _P_WHITE, _P_CORR, _P_SCAN, _P_FLAGINFO = range(9)


def _gen(seed: int, purpose: int, sub: int = 0) -> np.random.Generator:
    return np.random.Generator(np.random.Philox(key=[seed & (2**64 - 1), (purpose << 32) | sub]))


@dataclasses.dataclass
class BandConfig:
    """Shape of one synthetic band (one TOD object)."""
    name: str
    nside: int
    ndet: int
    nscan: int
    fsamp: float
    len_lo: int                 # raw scan length range, uniform integer draw
    len_hi: int
    fknee_lo: float = 0.05
    fknee_hi: float = 0.05
    alpha_lo: float = -1.5
    alpha_hi: float = -1.5
    sigma0: float = 1e-3
    sigma0_jitter: float = 0.0  # sigma0 * U[1-j, 1+j] per detector
    flag_frac: float = 0.0      # fraction of each detscan flagged, in gaps
    gap_lo: int = 10
    gap_hi: int = 500
    gain_rms: float = 0.01
    spin_period_s: float = 60.0     # 1 rpm
    opening_deg: float = 85.0
    precess_period_s: float = 0.0   # 0 = spin axis fixed within a scan
    precess_deg: float = 0.0
    axis_step_deg: float | None = None  # spin-axis longitude step per scan
    seed: int = 20220110


# Workloads: the 70 GHz band is the benchmark's headline, the 30 GHz band
# its secondary section; the three sweep bands (30/44/70 GHz-like, 1500
# scans each, lengths the band's mean +-20 %) make the multi-band Gibbs
# sweep; the rest are parity-test cases.
CONFIGS = {
    "tiny": BandConfig(name="tiny: 1 det x 16 scans x 4096 @32.5Hz, Nside 16",
                       nside=16, ndet=1, nscan=16, fsamp=32.5, len_lo=4096, len_hi=4096,
                       fknee_lo=0.05, fknee_hi=0.05, alpha_lo=-1.5, alpha_hi=-1.5,
                       spin_period_s=7.0, opening_deg=60.0, precess_period_s=51.0,
                       precess_deg=40.0, axis_step_deg=112.5, seed=20220111),
    "lfi30": BandConfig(name="30GHz-like: 4 det x 1000 scans x U[90k,140k] @32.5Hz, Nside 512",
                        nside=512, ndet=4, nscan=1000, fsamp=32.5, len_lo=90000, len_hi=140000,
                        fknee_lo=0.02, fknee_hi=0.2, alpha_lo=-2.0, alpha_hi=-1.0,
                        sigma0_jitter=0.2, flag_frac=0.02, seed=20220112),
    "lfi70": BandConfig(name="70GHz-like: 12 det x 2000 scans x U[150k,300k] @78.8Hz, Nside 1024",
                        nside=1024, ndet=12, nscan=2000, fsamp=78.8, len_lo=150000, len_hi=300000,
                        fknee_lo=0.02, fknee_hi=0.2, alpha_lo=-2.0, alpha_hi=-1.0,
                        sigma0_jitter=0.2, flag_frac=0.02, seed=20220113),
    "sweep30": BandConfig(name="sweep 30GHz-like: 4 det x 1500 scans x U[94k,140k] @32.5Hz, Nside 512",
                          nside=512, ndet=4, nscan=1500, fsamp=32.5, len_lo=93600, len_hi=140400,
                          fknee_lo=0.02, fknee_hi=0.2, alpha_lo=-2.0, alpha_hi=-1.0,
                          sigma0_jitter=0.2, flag_frac=0.02, seed=20220115),
    "sweep44": BandConfig(name="sweep 44GHz-like: 6 det x 1500 scans x U[136k,204k] @46.5Hz, Nside 512",
                          nside=512, ndet=6, nscan=1500, fsamp=46.5, len_lo=136000, len_hi=204000,
                          fknee_lo=0.02, fknee_hi=0.2, alpha_lo=-2.0, alpha_hi=-1.0,
                          sigma0_jitter=0.2, flag_frac=0.02, seed=20220116),
    "sweep70": BandConfig(name="sweep 70GHz-like: 12 det x 1500 scans x U[224k,336k] @78.8Hz, Nside 1024",
                          nside=1024, ndet=12, nscan=1500, fsamp=78.8, len_lo=224000, len_hi=336000,
                          fknee_lo=0.02, fknee_hi=0.2, alpha_lo=-2.0, alpha_hi=-1.0,
                          sigma0_jitter=0.2, flag_frac=0.02, seed=20220117),
    "chi2": BandConfig(name="chi2: 4 det x 200 scans x 65536 @32.5Hz, Nside 256",
                       nside=256, ndet=4, nscan=200, fsamp=32.5, len_lo=65536, len_hi=65536,
                       fknee_lo=0.02, fknee_hi=0.2, alpha_lo=-2.0, alpha_hi=-1.0,
                       sigma0_jitter=0.2, flag_frac=0.0, seed=20220114),
}


SWEEP_BANDS = ("sweep30", "sweep44", "sweep70")


def scaled(cfg: BandConfig, nscan: int | None = None, len_lo: int | None = None,
           len_hi: int | None = None, **kw) -> BandConfig:
    """A copy of ``cfg`` with fewer/shorter scans (same distributions)."""
    d = dataclasses.asdict(cfg)
    if nscan is not None:
        d["nscan"] = nscan
    if len_lo is not None:
        d["len_lo"] = len_lo
    if len_hi is not None:
        d["len_hi"] = len_hi
    d.update(kw)
    return BandConfig(**d)


# ----------------------------------------------------------------------------
# sky map
# ----------------------------------------------------------------------------

def sky_map(cfg: BandConfig) -> np.ndarray:
    """TQU map in K, shape (3, npix): T ~ N(0,(100uK)^2), Q,U ~ N(0,(10uK)^2)."""
    npix = nside2npix(cfg.nside)
    g = _gen(cfg.seed, _P_MAP)
    m = g.standard_normal((3, npix))
    m[0] *= 100e-6
    m[1:] *= 10e-6
    return m


# ----------------------------------------------------------------------------
# per-scan / per-detector parameters
# ----------------------------------------------------------------------------

def raw_lengths(cfg: BandConfig) -> np.ndarray:
    """Raw (pre-ingest) number of samples of each scan, int64[nscan]."""
    g = _gen(cfg.seed, _P_LEN)
    return g.integers(cfg.len_lo, cfg.len_hi + 1, size=cfg.nscan).astype(np.int64)


def gains(cfg: BandConfig) -> np.ndarray:
    """True gains g ~ N(1, gain_rms^2), float64[nscan*ndet] (detscan order)."""
    g = _gen(cfg.seed, _P_GAIN)
    return 1.0 + cfg.gain_rms * g.standard_normal(cfg.nscan * cfg.ndet)


def noise_params(cfg: BandConfig) -> np.ndarray:
    """Per-detector (sigma0 [K], f_knee [Hz], alpha), float64[ndet, 3]."""
    g = _gen(cfg.seed, _P_NOISEPAR)
    out = np.empty((cfg.ndet, 3))
    out[:, 0] = cfg.sigma0 * g.uniform(1 - cfg.sigma0_jitter, 1 + cfg.sigma0_jitter, cfg.ndet)
    out[:, 1] = g.uniform(cfg.fknee_lo, cfg.fknee_hi, cfg.ndet)
    out[:, 2] = g.uniform(cfg.alpha_lo, cfg.alpha_hi, cfg.ndet)
    return out


# ----------------------------------------------------------------------------
# scan strategy: precessing great-ish circles
# ----------------------------------------------------------------------------

def _rot_axis(v, axis, ang):
    """Rodrigues rotation of vectors v (...,3) about unit axis (3,) by ang (...)."""
    c = np.cos(ang)[..., None]
    s = np.sin(ang)[..., None]
    k = np.broadcast_to(axis, v.shape)
    return v * c + np.cross(k, v) * s + k * (np.sum(k * v, axis=-1, keepdims=True)) * (1 - c)


def scan_pointing(cfg: BandConfig, scan: int, n: int, det: int):
    """Continuous pointing of detector ``det`` during ``scan``.

    Returns (theta, phi, psi) float64[n]; psi in [0, 2pi).
    The spin axis lies near the ecliptic, stepping in longitude from scan to
    scan (one step per pointing period); the boresight circles it at the
    opening angle, one revolution per spin period.  Each detector sits at a
    small focal-plane offset and carries a polarisation angle offset of
    45 deg x det; psi follows the local scan direction.
    """
    t = np.arange(n, dtype=np.float64) / cfg.fsamp
    step = cfg.axis_step_deg if cfg.axis_step_deg is not None else 360.0 / 365.25 / 24.0
    lam = math.radians(step * scan)
    g = _gen(cfg.seed, _P_SCAN, scan)
    phase0 = g.uniform(0, 2 * math.pi)
    psi_scan = g.uniform(0, 2 * math.pi)
    # spin axis (possibly precessing about the ecliptic direction lam)
    base = np.array([math.cos(lam), math.sin(lam), 0.0])
    if cfg.precess_period_s > 0:
        pang = 2 * math.pi * t / cfg.precess_period_s + phase0
        tilt = math.radians(cfg.precess_deg)
        # perpendicular frame to base
        e1 = np.array([0.0, 0.0, 1.0])
        e2 = np.cross(base, e1)
        axis = (math.cos(tilt) * base[None, :]
                + math.sin(tilt) * (np.cos(pang)[:, None] * e1[None, :] + np.sin(pang)[:, None] * e2[None, :]))
    else:
        axis = np.broadcast_to(base, (n, 3))
    # boresight: start from the point at opening angle from the axis, rotate about it
    open_ang = math.radians(cfg.opening_deg + 0.35 * det)
    ez = np.array([0.0, 0.0, 1.0])
    perp = np.cross(axis, ez)
    perp /= np.linalg.norm(perp, axis=-1, keepdims=True)
    w = np.cross(axis, perp)
    spin = 2 * math.pi * t / cfg.spin_period_s + phase0 + 0.02 * det
    sa, ca = math.sin(open_ang), math.cos(open_ang)
    vec = ca * axis + sa * (np.cos(spin)[:, None] * perp + np.sin(spin)[:, None] * w)
    # scan direction (derivative wrt spin angle)
    dvec = sa * (-np.sin(spin)[:, None] * perp + np.cos(spin)[:, None] * w)
    z = np.clip(vec[:, 2], -1.0, 1.0)
    theta = np.arccos(z)
    phi = np.mod(np.arctan2(vec[:, 1], vec[:, 0]), 2 * math.pi)
    # local north (towards +z) and east unit vectors
    st = np.sqrt(np.maximum(1.0 - z * z, 1e-30))
    east = np.stack([-np.sin(phi), np.cos(phi), np.zeros_like(phi)], axis=-1)
    north = np.stack([-z * np.cos(phi), -z * np.sin(phi), st], axis=-1)
    ang = np.arctan2(np.sum(dvec * east, -1), np.sum(dvec * north, -1))
    psi = np.mod(ang + math.radians(45.0 * det) + psi_scan, 2 * math.pi)
    return theta, phi, psi


def psi_bin(psi: np.ndarray) -> np.ndarray:
    """Quantise a continuous angle in [0, 2pi) to one of N_PSI bins (uint16)."""
    b = np.floor(psi * (N_PSI / (2 * math.pi))).astype(np.int64)
    return np.mod(b, N_PSI).astype(np.uint16)


# ----------------------------------------------------------------------------
# flags and noise
# ----------------------------------------------------------------------------

def flag_mask(cfg: BandConfig, q: int, n: int) -> np.ndarray:
    """Boolean mask (True = flagged) with gaps of U{gap_lo..gap_hi} samples
    placed uniformly without overlap until >= flag_frac of the samples."""
    flagged = np.zeros(n, dtype=bool)
    if cfg.flag_frac <= 0:
        return flagged
    g = _gen(cfg.seed, _P_FLAGS, q)
    target = cfg.flag_frac * n
    total = 0
    tries = 0
    while total < target and tries < 100000:
        tries += 1
        L = int(g.integers(cfg.gap_lo, cfg.gap_hi + 1))
        if L >= n:
            continue
        a = int(g.integers(0, n - L + 1))
        lo, hi = max(0, a - 1), min(n, a + L + 1)
        if flagged[lo:hi].any():
            continue
        flagged[a:a + L] = True
        total += L
    return flagged


def correlated_noise(cfg: BandConfig, q: int, n: int, sigma0: float, fknee: float, alpha: float) -> np.ndarray:
    """1/f noise realisation with power sigma0^2 (f/fknee)^alpha per DCT mode."""
    import scipy.fft as sfft
    g = _gen(cfg.seed, _P_CORR, q)
    k = np.arange(n, dtype=np.float64)
    f = k * cfg.fsamp / (2.0 * n)
    amp = np.zeros(n)
    amp[1:] = sigma0 * (f[1:] / fknee) ** (alpha / 2.0)
    return sfft.idct(amp * g.standard_normal(n), norm="ortho")


# ----------------------------------------------------------------------------
# a whole band
# ----------------------------------------------------------------------------

@dataclasses.dataclass
class Band:
    cfg: BandConfig
    npix: int
    map_tqu: np.ndarray          # float64 (3, npix), K
    scan_len: np.ndarray         # raw samples per scan, int64[nscan]
    gain: np.ndarray             # true gains, float64[ndetscan]
    psd: np.ndarray              # float64[ndet, 3] (sigma0, fknee, alpha)
    pix: list                    # per detscan int32[n_raw]
    psi: list                    # per detscan uint16[n_raw] (bins)
    flags: list                  # per detscan bool[n_raw] (True = flagged)
    tod: list                    # per detscan float32[n_raw] (V)

    @property
    def ndet(self):
        return self.cfg.ndet

    @property
    def nscan(self):
        return self.cfg.nscan

    @property
    def ndetscan(self):
        return self.cfg.ndet * self.cfg.nscan


def _make_detscan(cfg, m, gain, psd, scan, det, n, with_noise):
    q = scan * cfg.ndet + det
    theta, phi, psi = scan_pointing(cfg, scan, n, det)
    pix = ang2pix_ring(cfg.nside, theta, phi).astype(np.int32)
    pb = psi_bin(psi)
    sig = m[0, pix] + m[1, pix] * np.cos(2 * psi) + m[2, pix] * np.sin(2 * psi)
    d = gain[q] * sig
    if with_noise:
        s0, fk, al = psd[det]
        gw = _gen(cfg.seed, _P_WHITE, q)
        d = d + s0 * gw.standard_normal(n) + correlated_noise(cfg, q, n, s0, fk, al)
    fl = flag_mask(cfg, q, n)
    return q, pix, pb, fl, d.astype(np.float32)


def make_band(cfg: BandConfig, with_noise: bool = True, threads: int | None = None) -> Band:
    """Generate every input of one band, seeded by ``cfg.seed``."""
    npix = nside2npix(cfg.nside)
    m = sky_map(cfg)
    L = raw_lengths(cfg)
    gn = gains(cfg)
    psd = noise_params(cfg)
    nq = cfg.nscan * cfg.ndet
    pix, psi, fl, tod = [None] * nq, [None] * nq, [None] * nq, [None] * nq
    jobs = [(s, d) for s in range(cfg.nscan) for d in range(cfg.ndet)]
    threads = threads or min(32, os.cpu_count() or 1)

    def work(sd):
        s, d = sd
        return _make_detscan(cfg, m, gn, psd, s, d, int(L[s]), with_noise)

    if threads > 1 and nq > 1:
        with ThreadPoolExecutor(threads) as ex:
            for q, a, b, c, e in ex.map(work, jobs):
                pix[q], psi[q], fl[q], tod[q] = a, b, c, e
    else:
        for sd in jobs:
            q, a, b, c, e = work(sd)
            pix[q], psi[q], fl[q], tod[q] = a, b, c, e
    return Band(cfg=cfg, npix=npix, map_tqu=m, scan_len=L, gain=gn, psd=psd,
                pix=pix, psi=psi, flags=fl, tod=tod)


@dataclasses.dataclass
class BandArrays:
    """A band generated straight into concatenated arrays: detscan q owns
    samples [offsets[q], offsets[q+1]), the first kept[q] samples of its raw
    timeline (the caller chooses kept; the values are those of make_band)."""
    cfg: BandConfig
    npix: int
    map_tqu: np.ndarray          # float64 (3, npix)
    scan_len: np.ndarray         # raw samples per scan
    gain: np.ndarray             # float64[ndetscan]
    psd: np.ndarray              # float64[ndet, 3]
    offsets: np.ndarray          # int64[ndetscan + 1]
    pix: np.ndarray              # int32[N]
    psi: np.ndarray              # uint16[N]
    flags: np.ndarray            # bool[N] (True = flagged)
    tod: np.ndarray              # float32[N]


def make_band_arrays(cfg: BandConfig, kept_per_scan, with_noise: bool = True,
                     threads: int | None = None, scans=None) -> BandArrays:
    """Generate every input of one band (or of the listed scans only), each
    detscan at its raw length as make_band does and truncated to
    kept_per_scan[scan] samples, written into concatenated arrays: the
    whole band never exists as per-detscan lists, so bands of billions of
    samples fit in host memory."""
    npix = nside2npix(cfg.nside)
    m = sky_map(cfg)
    L = raw_lengths(cfg)
    gn = gains(cfg)
    psd = noise_params(cfg)
    scans = list(range(cfg.nscan)) if scans is None else list(scans)
    kept = np.asarray(kept_per_scan, dtype=np.int64)
    qs = [(sc, d) for sc in scans for d in range(cfg.ndet)]
    nlen = np.array([kept[sc] for sc, _ in qs], dtype=np.int64)
    off = np.zeros(len(qs) + 1, dtype=np.int64)
    off[1:] = np.cumsum(nlen)
    N = int(off[-1])
    pix = np.empty(N, np.int32)
    psi = np.empty(N, np.uint16)
    fl = np.empty(N, bool)
    tod = np.empty(N, np.float32)
    threads = threads or min(32, os.cpu_count() or 1)

    def work(i):
        sc, d = qs[i]
        _, a, b, c, e = _make_detscan(cfg, m, gn, psd, sc, d, int(L[sc]), with_noise)
        k = int(nlen[i])
        o = int(off[i])
        pix[o:o + k] = a[:k]
        psi[o:o + k] = b[:k]
        fl[o:o + k] = c[:k]
        tod[o:o + k] = e[:k]

    if threads > 1 and len(qs) > 1:
        with ThreadPoolExecutor(threads) as ex:
            list(ex.map(work, range(len(qs))))
    else:
        for i in range(len(qs)):
            work(i)
    return BandArrays(cfg=cfg, npix=npix, map_tqu=m, scan_len=L, gain=gn, psd=psd, offsets=off,
                      pix=pix, psi=psi, flags=fl, tod=tod)


# ----------------------------------------------------------------------------
# integer data streams: ADC counts and quality-flag words (paper Sect. 4.1
# stores the TOD and the flags as integers that are differenced and Huffman
# coded like the pointing)
# ----------------------------------------------------------------------------

# ADC quantum = sigma0 / 100 of the detector: differenced white noise then
# spans about 140 quanta rms, about 9.2 bits per sample after Huffman coding,
# the TOD compression the paper's table reports for the 30 GHz channel
# (361 MB of 8-byte samples to 52 MB).
ADC_STEPS_PER_SIGMA0 = 100.0
FLAG_EXCLUDE = 1 << 1       # set on the samples of the flagged gaps (flag_mask)
FLAG_INFO = 1 << 4          # informational bit on runs of samples; not a reason to exclude
FLAG_SELECT = 0xF           # the flag-word bits that exclude a sample


def adc_quantum(band: "Band") -> np.ndarray:
    """ADC quantum of every detscan, float64[ndetscan] (detector sigma0 / 100)."""
    nd = band.cfg.ndet
    return np.array([band.psd[q % nd, 0] / ADC_STEPS_PER_SIGMA0 for q in range(band.ndetscan)])


def adc_counts(tod: np.ndarray, quantum: float) -> np.ndarray:
    """Digitised timeline: the nearest integer count of tod / quantum, int32."""
    c = np.rint(np.asarray(tod, dtype=np.float64) / quantum)
    if np.any(np.abs(c) >= 2 ** 30):
        raise ValueError("ADC counts out of range")
    return c.astype(np.int32)


def flag_words(cfg: BandConfig, q: int, flagged: np.ndarray) -> np.ndarray:
    """Quality-flag words of one detscan, int32: FLAG_EXCLUDE on the flagged
    samples, FLAG_INFO on seeded runs (about 5 % of the samples) anywhere."""
    n = len(flagged)
    w = np.where(np.asarray(flagged, dtype=bool), FLAG_EXCLUDE, 0).astype(np.int32)
    g = _gen(cfg.seed, _P_FLAGINFO, q)
    for _ in range(max(1, n // 40000)):
        a = int(g.integers(0, max(1, n)))
        w[a:a + int(g.integers(100, 4000))] |= FLAG_INFO
    return w


def uniform_draws(seed: int, shape, purpose: int = 99) -> np.ndarray:
    """Plain seeded standard normals for tests that need arbitrary vectors."""
    return _gen(seed, purpose).standard_normal(shape)
