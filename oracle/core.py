"""FP64 CPU oracle for the Gibbs TOD step (Commander3, arXiv 2201.03509).

TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
CPU-baseline leg of bench.py may import this package.  It shares no code with
the GPU library; the two meet only in ``synth`` (seeded inputs) and in formats
that must be alike (stream layout, Philox counters), each written separately.

Plain definitions, FP64 throughout, no blocking or fusion.  Each function
cites the passage it follows.  Where the paper is silent (it defers the gain
and noise samplers to companion papers) the reading taken is stated in the
docstring.

Notation: a band has ndet detectors and nscan scans; a detscan q = scan*ndet
+ det holds n_q samples at [off[q], off[q+1]) of the concatenated arrays.
Map m = (T, Q, U) on HEALPix RING pixels.  M_t = 1 for unflagged samples.
"""
from __future__ import annotations

import math

import numpy as np
import scipy.fft as sfft

from . import _huff

N_PSI = 4096
HUFF_MAXLEN = 24
CKPT_BLOCK = 512

# Philox purposes (counter word 2)
PURPOSE_GAIN = 0
PURPOSE_NC_W1 = 1
PURPOSE_NC_W2 = 2
PURPOSE_PSD = 3
PURPOSE_GAIN_SMOOTH = 4

MODE_DRAW = 0
MODE_MEAN = 1


# ============================================================================
# A0. ingest: FFT length rule and compressed streams
# ============================================================================

def fft_length(n: int) -> int:
    """Largest even 2^a 3^b 5^c (a >= 1) not above n.

    Paper Sect. 4.2: each chunk is truncated at read-in to a length that is
    cheap to FFT (a local minimum of a measured cost table; powers of small
    primes are the cheap ones).  Reading: the cheap set is the even 5-smooth
    numbers; the chunk keeps its first n' samples.
    """
    if n < 2:
        return 0
    best = 0
    p2 = 2
    while p2 <= n:
        p3 = p2
        while p3 <= n:
            p5 = p3
            while p5 <= n:
                if p5 > best:
                    best = p5
                p5 *= 5
            p3 *= 3
        p2 *= 2
    return best


def deltas(x: np.ndarray) -> np.ndarray:
    """Sample differencing before compression, d(i) - d(i-1) with d(-1) = 0
    (paper Sect. 4.1)."""
    x = np.asarray(x, dtype=np.int64)
    out = np.empty_like(x)
    if len(x):
        out[0] = x[0]
        out[1:] = x[1:] - x[:-1]
    return out


def undelta(dl: np.ndarray) -> np.ndarray:
    """Inverse of the differencing: running sum from 0 (paper Sect. 4.1)."""
    return np.cumsum(np.asarray(dl, dtype=np.int64))


def build_code(delta_streams) -> tuple:
    """One Huffman code for a list of delta streams (one scan, one stream
    kind, all its detectors).  Returns (values ascending, lengths)."""
    allv = np.concatenate([np.asarray(s, dtype=np.int64) for s in delta_streams])
    vals, counts = np.unique(allv, return_counts=True)
    lengths = _huff.code_lengths(counts, HUFF_MAXLEN)
    return vals.astype(np.int32), lengths


def encode_band_streams(per_detscan_values, ndet: int, block: int = CKPT_BLOCK) -> dict:
    """Compress one stream kind (pixel or psi bin) of a whole band.

    per_detscan_values: list (detscan order) of integer arrays, already
    truncated to their FFT lengths.  Returns the stream layout:
      words    uint32[W]        MSB-first bit stream, each detscan starting on a word
      word_off int64[nq+1]      first word of each detscan
      nbits    int64[nq]        payload bits of each detscan
      blk_off  int64[nq+1]      first checkpoint block of each detscan
      ckpt_bit uint32[nblk]     bit offset of block start, relative to the detscan's first word
      ckpt_val int32[nblk]      value preceding the block's first sample (0 for block 0)
      sym_off  int64[nscan+1]   code table of each scan
      sym_vals int32[S]         symbols of each code, ascending value
      sym_len  uint8[S]         code length of each symbol
    """
    nq = len(per_detscan_values)
    nscan = nq // ndet
    dl = [deltas(v) for v in per_detscan_values]
    sym_vals, sym_len, sym_off = [], [], [0]
    codes = []
    for s in range(nscan):
        v, L = build_code(dl[s * ndet:(s + 1) * ndet])
        c = _huff.canonical_codes(L)
        sym_vals.append(v)
        sym_len.append(L)
        codes.append(c)
        sym_off.append(sym_off[-1] + len(v))
    chunks, word_off, nbits = [], [0], []
    blk_off, ckpt_bit, ckpt_val = [0], [], []
    for q in range(nq):
        s = q // ndet
        v, L, c = sym_vals[s], sym_len[s], codes[s]
        d = dl[q]
        n = len(d)
        total_bits = int(np.sum(L[np.searchsorted(v, d)].astype(np.int64))) if n else 0
        nw = (total_bits + 31) // 32
        w = np.zeros(max(nw, 1) if n else 0, dtype=np.uint32)
        pos = 0
        x = np.asarray(per_detscan_values[q], dtype=np.int64)
        nblk = (n + block - 1) // block
        for b in range(nblk):
            lo, hi = b * block, min(n, (b + 1) * block)
            ckpt_bit.append(pos)
            ckpt_val.append(int(x[lo - 1]) if lo > 0 else 0)
            pos = _huff.encode_into(w, pos, d[lo:hi], v, c, L)
        assert pos == total_bits
        chunks.append(w[:nw])
        word_off.append(word_off[-1] + nw)
        nbits.append(total_bits)
        blk_off.append(blk_off[-1] + nblk)
    return dict(
        words=np.concatenate(chunks) if chunks else np.zeros(0, np.uint32),
        word_off=np.array(word_off, dtype=np.int64),
        nbits=np.array(nbits, dtype=np.int64),
        blk_off=np.array(blk_off, dtype=np.int64),
        ckpt_bit=np.array(ckpt_bit, dtype=np.uint32),
        ckpt_val=np.array(ckpt_val, dtype=np.int32),
        sym_off=np.array(sym_off, dtype=np.int64),
        sym_vals=np.concatenate(sym_vals) if sym_vals else np.zeros(0, np.int32),
        sym_len=np.concatenate(sym_len) if sym_len else np.zeros(0, np.uint8),
    )


# ============================================================================
# A1. decode
# ============================================================================

def decode_detscan(st: dict, q: int, n: int, ndet: int) -> np.ndarray:
    """Huffman-decode detscan q's stream and undo the differencing
    (paper Sect. 4.1; Listing `tod`: pix/psi held as compressed bytes).
    Walks the whole stream from its first bit; the checkpoints are not used."""
    s = q // ndet
    a, b = st["sym_off"][s], st["sym_off"][s + 1]
    vals = np.ascontiguousarray(st["sym_vals"][a:b])
    L = np.ascontiguousarray(st["sym_len"][a:b])
    codes = _huff.canonical_codes(L)
    w0, w1 = st["word_off"][q], st["word_off"][q + 1]
    words = np.ascontiguousarray(st["words"][w0:w1])
    dl, end = _huff.decode(words, int(st["nbits"][q]), 0, n, vals, codes, L)
    if end != int(st["nbits"][q]):
        raise ValueError("stream length mismatch")
    return undelta(dl)


def decode_band(st: dict, offsets: np.ndarray, ndet: int) -> np.ndarray:
    nq = len(offsets) - 1
    out = np.empty(int(offsets[-1]), dtype=np.int64)
    for q in range(nq):
        out[offsets[q]:offsets[q + 1]] = decode_detscan(st, q, int(offsets[q + 1] - offsets[q]), ndet)
    return out


def decode_tod(st: dict, offsets: np.ndarray, ndet: int, scale: np.ndarray) -> np.ndarray:
    """The detector data from the compressed ADC counts (Sect. 4.1: the
    TOD is held as differenced, Huffman-coded integers; Listing `tod`:
    comm_detscan keeps tod as compressed bytes).  Reading (the paper does not
    print the conversion): the counts c_t are ADC integers and d_t = scale_q
    c_t, the product in FP64 rounded once to FP32, the precision the step
    reads d in."""
    c = decode_band(st, offsets, ndet).astype(np.float64)
    return (c * per_sample(np.asarray(scale, np.float64), offsets)).astype(np.float32)


def decode_flags(st: dict, offsets: np.ndarray, ndet: int, select: int) -> np.ndarray:
    """The flag mask from the compressed flag words (Sect. 4.1; Listing
    `tod`: flag kept as compressed bytes).  Reading: sample t is excluded
    (M_t = 0) when its word has any of the bits in ``select``."""
    w = decode_band(st, offsets, ndet)
    return (w & int(select)) != 0


# ============================================================================
# RNG: Philox4x64-10 (Salmon, Moraes, Dror, Shaw 2011) + Box-Muller
# ============================================================================

_PH_M0 = 0xD2E7470EE14C6C93
_PH_M1 = 0xCA5A826395121157
_PH_W0 = 0x9E3779B97F4A7C15
_PH_W1 = 0xBB67AE8584CAA73B
_MASK32 = np.uint64(0xFFFFFFFF)


def _mulhilo64(a: int, b: np.ndarray):
    """(hi, lo) 64-bit halves of the 128-bit product a*b, via 32-bit limbs."""
    b = b.astype(np.uint64)
    a_lo, a_hi = np.uint64(a & 0xFFFFFFFF), np.uint64(a >> 32)
    b_lo, b_hi = b & _MASK32, b >> np.uint64(32)
    ll = a_lo * b_lo
    lh = a_lo * b_hi
    hl = a_hi * b_lo
    hh = a_hi * b_hi
    mid = (ll >> np.uint64(32)) + (lh & _MASK32) + (hl & _MASK32)
    lo = (ll & _MASK32) | ((mid & _MASK32) << np.uint64(32))
    hi = hh + (lh >> np.uint64(32)) + (hl >> np.uint64(32)) + (mid >> np.uint64(32))
    return hi, lo


def philox4x64(ctr, key) -> np.ndarray:
    """Philox4x64-10 block function.  ctr: 4 arrays (or ints) of uint64,
    key: 2 ints.  Returns uint64 array (..., 4)."""
    c = [np.asarray(x, dtype=np.uint64) for x in ctr]
    c = list(np.broadcast_arrays(*c))
    k0, k1 = int(key[0]) & 0xFFFFFFFFFFFFFFFF, int(key[1]) & 0xFFFFFFFFFFFFFFFF
    with np.errstate(over="ignore"):
        for r in range(10):
            if r:
                k0 = (k0 + _PH_W0) & 0xFFFFFFFFFFFFFFFF
                k1 = (k1 + _PH_W1) & 0xFFFFFFFFFFFFFFFF
            hi0, lo0 = _mulhilo64(_PH_M0, c[0])
            hi1, lo1 = _mulhilo64(_PH_M1, c[2])
            c = [hi1 ^ c[1] ^ np.uint64(k0), lo1, hi0 ^ c[3] ^ np.uint64(k1), lo0]
    return np.stack(c, axis=-1)


def gain_normal(seed: int, band: int, q: int, it: int) -> float:
    """The standard normal of the gain draw of detscan q at Gibbs iteration
    it: counter (0, q, GAIN, it); 53-bit uniforms from words 0 and 1;
    Box-Muller cosine branch, FP64."""
    w = philox4x64([0, q, PURPOSE_GAIN, it], [seed, band])
    u1 = (float(w[0] >> np.uint64(11)) + 0.5) * 2.0 ** -53
    u2 = (float(w[1] >> np.uint64(11)) + 0.5) * 2.0 ** -53
    return math.sqrt(-2.0 * math.log(u1)) * math.cos(2.0 * math.pi * u2)


def stream_normals(seed: int, band: int, q: int, purpose: int, it: int, n: int) -> np.ndarray:
    """n standard normals of one (detscan, purpose, iteration) stream.

    Normal i comes from Philox block i//8 (counter (i//8, q, purpose, it)),
    whose four 64-bit words split into eight 32-bit halves, low half first;
    pair j = (i%8)//2 takes halves 2j, 2j+1 as uniforms u = (h>>9 + 1/2) 2^-23
    and gives sqrt(-2 ln u1) cos(2 pi u2) (even i) or ... sin(2 pi u2) (odd i).
    Evaluated here in FP64."""
    nb = (n + 7) // 8
    blk = np.arange(nb, dtype=np.uint64)
    w = philox4x64([blk, np.uint64(q), np.uint64(purpose), np.uint64(it)], [seed, band])
    halves = np.empty((nb, 8), dtype=np.uint64)
    halves[:, 0::2] = w & _MASK32
    halves[:, 1::2] = w >> np.uint64(32)
    u = ((halves >> np.uint64(9)).astype(np.float64) + 0.5) * 2.0 ** -23
    u1, u2 = u[:, 0::2], u[:, 1::2]
    r = np.sqrt(-2.0 * np.log(u1))
    z = np.empty((nb, 8))
    z[:, 0::2] = r * np.cos(2.0 * np.pi * u2)
    z[:, 1::2] = r * np.sin(2.0 * np.pi * u2)
    return z.reshape(-1)[:n]


def omega1(seed: int, band: int, q: int, it: int, n: int) -> np.ndarray:
    """White-noise normals of the correlated-noise right-hand side, one per
    sample.  Convention (the paper does not fix one): sample t takes normal
    number i(t) of stream (q, NC_W1, it), where i(t) is t's position in the
    even-then-reversed-odd order (x_0, x_2, ..., x_3, x_1): i = t/2 for even
    t, n-1-(t-1)/2 for odd t."""
    z = stream_normals(seed, band, q, PURPOSE_NC_W1, it, n)
    t = np.arange(n)
    i = np.where(t % 2 == 0, t // 2, n - 1 - (t - 1) // 2)
    return z[i]


def omega2(seed: int, band: int, q: int, it: int, n: int) -> np.ndarray:
    """Normals of the prior term, one per DCT mode kappa.  Convention: modes
    kappa and n-kappa (1 <= kappa < n/2) take normals 2 kappa and 2 kappa+1 of
    stream (q, NC_W2, it); mode 0 takes normal 0 and mode n/2 normal 1."""
    z = stream_normals(seed, band, q, PURPOSE_NC_W2, it, n)
    m = n // 2
    k = np.arange(n)
    nu = np.where(k < m, 2 * k, 2 * (n - k) + 1)
    nu[0] = 0
    nu[m] = 1
    return z[nu]


# ============================================================================
# A2. projection
# ============================================================================

def psi_trig_table() -> tuple:
    """cos 2psi, sin 2psi at the n_psi = 4096 bin centres psi_b = (b+1/2) 2pi/4096
    (paper Sect. 4.1: psi stored discretised), rounded to FP32 values: the
    tabulated angles are part of the discretised pointing."""
    b = np.arange(N_PSI, dtype=np.float64)
    psi = (b + 0.5) * (2.0 * np.pi / N_PSI)
    c = np.cos(2.0 * psi).astype(np.float32).astype(np.float64)
    s = np.sin(2.0 * psi).astype(np.float32).astype(np.float64)
    return c, s


def project(map_tqu: np.ndarray, pix: np.ndarray, psi: np.ndarray, gain_per_sample=None) -> np.ndarray:
    """s_t = g (T_p + Q_p cos 2psi_t + U_p sin 2psi_t) at p = pix_t
    (paper Eq. `todmodel`, the g P m term with the sky reduced to one TQU map;
    Sect. 4.1 discretised pointing).  FP64."""
    c, s = psi_trig_table()
    m = np.asarray(map_tqu, dtype=np.float64)
    pix = np.asarray(pix, dtype=np.int64)
    b = np.asarray(psi, dtype=np.int64)
    out = m[0, pix] + m[1, pix] * c[b] + m[2, pix] * s[b]
    if gain_per_sample is not None:
        out = out * gain_per_sample
    return out


def per_sample(values_per_detscan: np.ndarray, offsets: np.ndarray) -> np.ndarray:
    """Repeat one value per detscan over its samples."""
    return np.repeat(np.asarray(values_per_detscan), np.diff(offsets))


# ============================================================================
# A3. DCT-II (mirror-equivalent FFT)
# ============================================================================

def dct(x: np.ndarray) -> np.ndarray:
    """Orthonormal DCT-II, X_k = w_k sum_j x_j cos(pi k (j+1/2)/n),
    w_0 = sqrt(1/n), w_k = sqrt(2/n).  Paper Sect. 4.2: every FFT runs on the
    array doubled with its mirror image appended, which is periodic; the FFT
    of that half-sample-symmetric extension is, up to a phase, this DCT-II.
    Library routine (scipy) as the step; pinned in tests against the
    definition and against the mirrored FFT."""
    return sfft.dct(np.asarray(x, dtype=np.float64), type=2, norm="ortho")


def idct(X: np.ndarray) -> np.ndarray:
    """Inverse (= transpose) of ``dct``: orthonormal DCT-III."""
    return sfft.idct(np.asarray(X, dtype=np.float64), type=2, norm="ortho")


def dct_direct(x: np.ndarray) -> np.ndarray:
    """The DCT-II definition evaluated as an O(n^2) sum (tests only)."""
    x = np.asarray(x, dtype=np.float64)
    n = len(x)
    j = np.arange(n)
    k = j[:, None]
    C = np.cos(np.pi * k * (j[None, :] + 0.5) / n)
    w = np.full(n, math.sqrt(2.0 / n))
    w[0] = math.sqrt(1.0 / n)
    return w * (C @ x)


def dct_freqs(n: int, fsamp: float) -> np.ndarray:
    """Frequency of DCT mode k: f_k = k fsamp / (2n) (the mirrored array has
    period 2n)."""
    return np.arange(n, dtype=np.float64) * fsamp / (2.0 * n)


# ============================================================================
# A4. gain
# ============================================================================

def noise_psd(n: int, fsamp: float, sigma0: float, fknee: float, alpha: float) -> np.ndarray:
    """Total noise PSD per DCT mode, P_k = sigma0^2 (1 + (f_k/fknee)^alpha);
    P_0 set to +inf (the offset mode carries no weight).  Reading: the 1/f
    model of the correlated noise (paper Eq. `todmodel` n_corr + n_w), the
    exact form being deferred by the paper to its noise companion paper."""
    f = dct_freqs(n, fsamp)
    P = np.full(n, np.inf)
    P[1:] = sigma0 ** 2 * (1.0 + (f[1:] / fknee) ** alpha)
    return P


def corr_inv_psd(n: int, fsamp: float, sigma0: float, fknee: float, alpha: float) -> np.ndarray:
    """phi_k = 1 / (sigma0^2 (f_k/fknee)^alpha), the inverse correlated-noise
    PSD; phi_0 = 0 (no prior on the offset)."""
    f = dct_freqs(n, fsamp)
    phi = np.zeros(n)
    phi[1:] = 1.0 / (sigma0 ** 2 * (f[1:] / fknee) ** alpha)
    return phi


def gain_sums(s: np.ndarray, d: np.ndarray, mask: np.ndarray, P: np.ndarray) -> tuple:
    """a = sum_{k>=1} shat_k^2 / P_k,  b = sum_{k>=1} shat_k dhat_k / P_k with
    shat = C(M s), dhat = C(M d).  Reading of the gain conditional
    (paper Eq. `gibbsstart`: g drawn given d and xi_n but not n_corr, so the
    correlated noise is marginalised and N = N_w + N_corr)."""
    M = np.asarray(mask, dtype=np.float64)
    sh = dct(M * s)
    dh = dct(M * d)
    a = float(np.sum(sh[1:] ** 2 / P[1:]))
    b = float(np.sum(sh[1:] * dh[1:] / P[1:]))
    return a, b


def sample_gain(s, d, mask, P, z: float, mode: int = MODE_DRAW) -> tuple:
    """Gaussian conditional of one detscan's gain: mean b/a, rms 1/sqrt(a);
    g = mean + z rms (z = 0 in MODE_MEAN).  Returns (g, mean, rms)."""
    a, b = gain_sums(s, d, mask, P)
    mu = b / a
    sig = 1.0 / math.sqrt(a)
    return (mu + (z * sig if mode == MODE_DRAW else 0.0)), mu, sig


# ============================================================================
# A12. gains of all scans of a detector under a smooth prior
# ============================================================================

def gain_smooth_normals(seed: int, band: int, det: int, it: int, nscan: int) -> tuple:
    """The two standard normals of scan s in the smooth gain draw of detector
    det: Philox block (s, det, GAIN_SMOOTH, it); 53-bit uniforms from words
    0, 1 (w1_s) and 2, 3 (w2_s), Box-Muller cosine branch, FP64."""
    w1 = np.empty(nscan)
    w2 = np.empty(nscan)
    for sc in range(nscan):
        w = philox4x64([sc, det, PURPOSE_GAIN_SMOOTH, it], [seed, band])
        u = [(float(w[j] >> np.uint64(11)) + 0.5) * 2.0 ** -53 for j in range(4)]
        w1[sc] = math.sqrt(-2.0 * math.log(u[0])) * math.cos(2.0 * math.pi * u[1])
        w2[sc] = math.sqrt(-2.0 * math.log(u[2])) * math.cos(2.0 * math.pi * u[3])
    return w1, w2


def gain_prior_precision(nscan: int, sigma_g: float, alpha_g: float) -> np.ndarray:
    """Prior precision of a detector's scan gains in the orthonormal DCT-II
    basis of the scan index: lambda_0 = 0 (the mean gain is free),
    lambda_k = 1 / (sigma_g^2 k^alpha_g) for k >= 1 (reading: the paper
    defers the gain model to its calibration companion paper)."""
    lam = np.zeros(nscan)
    k = np.arange(1, nscan, dtype=np.float64)
    lam[1:] = 1.0 / (sigma_g ** 2 * k ** alpha_g)
    return lam


def sample_gain_smooth(mu, sigma, sigma_g: float, alpha_g: float, w1, w2, mode: int = MODE_DRAW) -> np.ndarray:
    """Joint draw of one detector's scan gains: each scan's gain conditional
    N(mu_s, sigma_s^2) (the per-detscan draw, n_corr marginalised) times the
    smooth prior of ``gain_prior_precision``.  Posterior precision
    A = diag(1/sigma^2) + C^T diag(lambda) C, with C the orthonormal DCT-II
    matrix; g = A^-1 (mu/sigma^2 + w1/sigma + C^T (sqrt(lambda) w2)), the
    noise terms dropped in MODE_MEAN.  Dense FP64 solve."""
    mu = np.asarray(mu, np.float64)
    sigma = np.asarray(sigma, np.float64)
    S = len(mu)
    C = sfft.dct(np.eye(S), type=2, norm="ortho", axis=0)     # column q = C e_q
    lam = gain_prior_precision(S, sigma_g, alpha_g)
    A = np.diag(1.0 / sigma ** 2) + C.T @ np.diag(lam) @ C
    rhs = mu / sigma ** 2
    if mode == MODE_DRAW:
        rhs = rhs + np.asarray(w1, np.float64) / sigma + C.T @ (np.sqrt(lam) * np.asarray(w2, np.float64))
    return np.linalg.solve(A, rhs)


# ============================================================================
# A5. correlated noise
# ============================================================================

def ncorr_rhs(r, mask, sigma0, phi, w1, w2) -> np.ndarray:
    """b = M r / sigma0^2 + M w1 / sigma0 + C^T(sqrt(phi) w2): the standard
    constrained-realisation right-hand side (reading; the paper defers the
    sampler to its noise companion paper: the n_corr conditional of Eq.
    `gibbsstart` and Sect. 5 on CG gap filling)."""
    M = np.asarray(mask, dtype=np.float64)
    return M * r / sigma0 ** 2 + M * w1 / sigma0 + idct(np.sqrt(phi) * w2)


def ncorr_apply_A(x, mask, sigma0, phi) -> np.ndarray:
    """A x with A = C^T diag(phi) C + M / sigma0^2."""
    M = np.asarray(mask, dtype=np.float64)
    return idct(phi * dct(x)) + M * x / sigma0 ** 2


def ncorr_solve_gapfree(b, sigma0, phi) -> np.ndarray:
    """Exact solution when no sample is flagged: A is diagonal in the DCT
    basis, x = C^T[(C b) / (phi + 1/sigma0^2)]."""
    return idct(dct(b) / (phi + 1.0 / sigma0 ** 2))


def ncorr_solve_pcg(b, mask, sigma0, phi, tol=1e-12, maxiter=5000) -> tuple:
    """Preconditioned conjugate gradients for A x = b (paper Sect. 5: the
    correlated-noise step gap-fills flagged samples with a CG solver).
    Preconditioner C^T diag(1/(phi + 1/sigma0^2)) C, the exact inverse of A
    with every sample unflagged.  Returns (x, iterations)."""
    pdiag = 1.0 / (phi + 1.0 / sigma0 ** 2)
    x = np.zeros_like(b)
    r = b.copy()
    z = idct(pdiag * dct(r))
    p = z.copy()
    rz = float(r @ z)
    nb = float(np.linalg.norm(b))
    if nb == 0:
        return x, 0
    for it in range(1, maxiter + 1):
        Ap = ncorr_apply_A(p, mask, sigma0, phi)
        alpha = rz / float(p @ Ap)
        x += alpha * p
        r -= alpha * Ap
        if np.linalg.norm(r) <= tol * nb:
            return x, it
        z = idct(pdiag * dct(r))
        rz_new = float(r @ z)
        p = z + (rz_new / rz) * p
        rz = rz_new
    return x, -1


def ncorr_solve_allflagged(b, phi) -> np.ndarray:
    """Every sample flagged: A = C^T diag(phi) C, singular in the offset mode
    (phi_0 = 0) which no data constrain.  Reading: the draw is the
    minimum-norm solution x = C^T[(C b) / phi] with mode 0 set to zero
    (the right-hand side has no offset component then: b = C^T(sqrt(phi) w2))."""
    X = dct(b)
    inv = np.zeros_like(phi)
    inv[1:] = 1.0 / phi[1:]
    return idct(X * inv)


def ncorr_dense_A(n, mask, sigma0, phi) -> np.ndarray:
    """The explicit n x n matrix A (brute force, small n only)."""
    C = np.stack([dct(e) for e in np.eye(n)], axis=1)     # column j = C e_j
    return C.T @ np.diag(phi) @ C + np.diag(np.asarray(mask, np.float64)) / sigma0 ** 2


def ncorr_solve_dense(b, mask, sigma0, phi) -> np.ndarray:
    """Dense Cholesky solve of the explicit A (brute force reference)."""
    A = ncorr_dense_A(len(b), mask, sigma0, phi)
    L = np.linalg.cholesky(A)
    y = np.linalg.solve(L, b)
    return np.linalg.solve(L.T, y)


def sample_ncorr(d, s, gain, mask, sigma0, fknee, alpha, fsamp, w1, w2, tol=1e-12) -> tuple:
    """One detscan's correlated-noise draw.  r = d - g s; solve A x = b.
    Gap-free detscans use the exact diagonal solve, others PCG.
    Returns (x, cg_iterations)."""
    n = len(d)
    phi = corr_inv_psd(n, fsamp, sigma0, fknee, alpha)
    r = np.asarray(d, np.float64) - gain * np.asarray(s, np.float64)
    b = ncorr_rhs(r, mask, sigma0, phi, w1, w2)
    if np.all(np.asarray(mask) != 0):
        return ncorr_solve_gapfree(b, sigma0, phi), 0
    if not np.any(np.asarray(mask) != 0):
        return ncorr_solve_allflagged(b, phi), 0
    return ncorr_solve_pcg(b, mask, sigma0, phi, tol=tol)


# ============================================================================
# A6. binning, A7. per-pixel solve
# ============================================================================

def bin_maps(npix, pix, psi, resid, weight) -> tuple:
    """Per-pixel normal equations (paper Sect. 5 table rows "TOD binning" and
    "Map solution (Ax=b for each pixel)"):
        A_p = sum_t w_t u_t u_t^T,   b_p = sum_t v_t u_t resid_t,
    u_t = (1, cos 2psi_t, sin 2psi_t).  ``weight`` is (w_t, v_t) per sample,
    w = M g^2 / sigma0^2 and v = M g / sigma0^2 (P includes the gain; the
    residual is calibrated by g and weighted by the white-noise variance).
    Sums in ascending t, FP64.  A is returned as its 6 unique entries
    (TT, TQ, TU, QQ, QU, UU); hits_p counts unflagged samples."""
    c, s = psi_trig_table()
    w, v = weight
    pix = np.asarray(pix, dtype=np.int64)
    b_ = np.asarray(psi, dtype=np.int64)
    ct, st = c[b_], s[b_]
    A = np.empty((npix, 6))
    for i, term in enumerate((w, w * ct, w * st, w * ct * ct, w * ct * st, w * st * st)):
        A[:, i] = np.bincount(pix, weights=term, minlength=npix)
    rv = v * np.asarray(resid, np.float64)
    b = np.empty((npix, 3))
    for i, term in enumerate((rv, rv * ct, rv * st)):
        b[:, i] = np.bincount(pix, weights=term, minlength=npix)
    return A, b


def bin_partials(npix, pix, psi, resid, weight) -> tuple:
    """The ten per-pixel sums of bin_maps (A 6, b 3, hits) as exact partial
    sums: each the correctly rounded sum of its terms (math.fsum) and the
    correctly rounded remainder, hi + lo, so that partial sums of separate
    sample sets add without a rounding of their own (the reduction of a
    band split over processes).  Returns (hi, lo), each float64[npix, 10]."""
    c, sn = psi_trig_table()
    pix = np.asarray(pix, np.int64)
    b = np.asarray(psi, np.int64)
    w, v = weight
    cc, ss = c[b], sn[b]
    terms = np.stack([w, w * cc, w * ss, w * cc * cc, w * cc * ss, w * ss * ss,
                      v * resid, v * cc * resid, v * ss * resid, (np.asarray(w) > 0).astype(np.float64)], axis=1)
    order = np.argsort(pix, kind="stable")
    ps = pix[order]
    edges = np.searchsorted(ps, np.arange(npix + 1))
    hi = np.zeros((npix, 10))
    lo = np.zeros((npix, 10))
    for p in range(npix):
        sel = order[edges[p]:edges[p + 1]]
        if len(sel) == 0:
            continue
        for k in range(10):
            col = terms[sel, k].tolist()
            h = math.fsum(col)
            hi[p, k] = h
            lo[p, k] = math.fsum(col + [-h])
    return hi, lo


def combine_partials(partials) -> tuple:
    """Partial sums (hi, lo) of several sample sets, in order, to the
    correctly rounded totals: A float64[npix, 6], b float64[npix, 3],
    hits int64[npix]."""
    his = [h for h, _ in partials]
    los = [l for _, l in partials]
    npix = his[0].shape[0]
    tot = np.zeros((npix, 10))
    for p in range(npix):
        for k in range(10):
            tot[p, k] = math.fsum([x[p, k] for x in his] + [x[p, k] for x in los])
    return tot[:, :6], tot[:, 6:9], np.rint(tot[:, 9]).astype(np.int64)


def solve_maps(A6: np.ndarray, b3: np.ndarray, hits: np.ndarray, rcond_min: float = 1e-6) -> tuple:
    """m_p = A_p^{-1} b_p by an explicit 3x3 Cholesky factorisation.
    Reading of validity (the paper is silent): a pixel is solved iff it has
    at least 3 hits and the Hadamard ratio det(A)/(A_TT A_QQ A_UU) is at
    least rcond_min; otherwise m_p = 0 and valid = 0.
    Returns (map (3, npix), rcond (Hadamard ratio), valid uint8)."""
    a00, a01, a02, a11, a12, a22 = (A6[:, i] for i in range(6))
    det = (a00 * (a11 * a22 - a12 * a12) - a01 * (a01 * a22 - a12 * a02)
           + a02 * (a01 * a12 - a11 * a02))
    diagprod = a00 * a11 * a22
    with np.errstate(divide="ignore", invalid="ignore"):
        had = np.where(diagprod > 0, det / diagprod, 0.0)
    valid = (np.asarray(hits) >= 3) & (had >= rcond_min) & (a00 > 0) & (a11 > 0) & (a22 > 0)
    npix = A6.shape[0]
    m = np.zeros((3, npix))
    v = np.nonzero(valid)[0]
    a00, a01, a02, a11, a12, a22 = a00[v], a01[v], a02[v], a11[v], a12[v], a22[v]
    l00 = np.sqrt(a00)
    l10 = a01 / l00
    l20 = a02 / l00
    l11 = np.sqrt(a11 - l10 * l10)
    l21 = (a12 - l20 * l10) / l11
    l22 = np.sqrt(a22 - l20 * l20 - l21 * l21)
    y0 = b3[v, 0] / l00
    y1 = (b3[v, 1] - l10 * y0) / l11
    y2 = (b3[v, 2] - l20 * y0 - l21 * y1) / l22
    x2 = y2 / l22
    x1 = (y1 - l21 * x2) / l11
    x0 = (y0 - l10 * x1 - l20 * x2) / l00
    m[0, v], m[1, v], m[2, v] = x0, x1, x2
    return m, had, valid.astype(np.uint8)


# ============================================================================
# the whole step, A1..A7
# ============================================================================

def ingest(band, ndet=None, data_streams: bool = False) -> dict:
    """A0 on a synthetic band: truncate every scan to its FFT length and
    compress its pixel and psi streams (with ``data_streams``, its ADC
    counts and flag words too).  Returns the arrays the step uses."""
    ndet = band.cfg.ndet
    nq = band.ndetscan
    nlen = np.array([fft_length(int(band.scan_len[q // ndet])) for q in range(nq)], dtype=np.int64)
    off = np.zeros(nq + 1, dtype=np.int64)
    off[1:] = np.cumsum(nlen)
    pix = [np.asarray(band.pix[q][:nlen[q]], np.int64) for q in range(nq)]
    psi = [np.asarray(band.psi[q][:nlen[q]], np.int64) for q in range(nq)]
    out = dict(
        offsets=off,
        pix_streams=encode_band_streams(pix, ndet),
        psi_streams=encode_band_streams(psi, ndet),
        tod=np.concatenate([band.tod[q][:nlen[q]] for q in range(nq)]).astype(np.float32),
        flags=np.concatenate([band.flags[q][:nlen[q]] for q in range(nq)]),
    )
    if data_streams:
        import synth
        scale = synth.adc_quantum(band)
        counts = [synth.adc_counts(band.tod[q][:nlen[q]], scale[q]) for q in range(nq)]
        words = [synth.flag_words(band.cfg, q, band.flags[q][:nlen[q]]) for q in range(nq)]
        out.update(tod_streams=encode_band_streams(counts, ndet), tod_scale=scale, tod_counts=counts,
                   flag_streams=encode_band_streams(words, ndet), flag_words=words,
                   flag_select=synth.FLAG_SELECT)
    return out


def gibbs_tod_step(ing: dict, band_cfg, npix: int, map_tqu: np.ndarray, psd: np.ndarray,
                   seed: int, band_id: int, it: int, mode: int = MODE_DRAW,
                   detscans=None, rcond_min: float = 1e-6, pcg_tol: float = 1e-12) -> dict:
    """One Gibbs TOD step (paper Listing `code:gibbs` step 1 and Sect. 2.4):
    decode -> project -> sample gain -> sample n_corr -> bin -> solve.
    ``detscans`` restricts the work to a subset (bounded CPU timing)."""
    ndet = band_cfg.ndet
    fs = band_cfg.fsamp
    off = ing["offsets"]
    nq = len(off) - 1
    qs = range(nq) if detscans is None else detscans
    gain = np.zeros(nq)
    mu = np.zeros(nq)
    sig = np.zeros(nq)
    iters = np.zeros(nq, dtype=np.int64)
    A = np.zeros((npix, 6))
    b = np.zeros((npix, 3))
    hits = np.zeros(npix, dtype=np.int64)
    ncorr = {}
    for q in qs:
        det = q % ndet
        a0, a1 = int(off[q]), int(off[q + 1])
        n = a1 - a0
        s0, fk, al = psd[det]
        pix = decode_detscan(ing["pix_streams"], q, n, ndet)
        psi = decode_detscan(ing["psi_streams"], q, n, ndet)
        s = project(map_tqu, pix, psi)
        d = ing["tod"][a0:a1].astype(np.float64)
        M = (~ing["flags"][a0:a1]).astype(np.float64)
        P = noise_psd(n, fs, s0, fk, al)
        z = gain_normal(seed, band_id, q, it)
        gain[q], mu[q], sig[q] = sample_gain(s, d, M, P, z, mode)
        if mode == MODE_DRAW:
            w1 = omega1(seed, band_id, q, it, n)
            w2 = omega2(seed, band_id, q, it, n)
        else:
            w1 = np.zeros(n)
            w2 = np.zeros(n)
        x, iters[q] = sample_ncorr(d, s, gain[q], M, s0, fk, al, fs, w1, w2, tol=pcg_tol)
        ncorr[q] = x
        w = M * gain[q] ** 2 / s0 ** 2
        v = M * gain[q] / s0 ** 2
        Aq, bq = bin_maps(npix, pix, psi, d - x, (w, v))
        A += Aq
        b += bq
        hits += np.bincount(pix, weights=M, minlength=npix).astype(np.int64)
    m, had, valid = solve_maps(A, b, hits, rcond_min)
    return dict(gain=gain, mu=mu, sigma=sig, cg_iters=iters, ncorr=ncorr,
                A=A, b=b, hits=hits, map=m, rcond=had, valid=valid)


# ============================================================================
# A8. TOD chi^2 of the correlated-noise-marginalised likelihood and its
# gradients (the adjoint of the projection is the binning)
# ============================================================================

def chi2_detscan(d, s, gain, mask, sigma0, fknee, alpha, fsamp) -> dict:
    """L = 1/2 sum_{k>=1} [ rhat_k^2 / P_k + ln P_k ],  rhat = C(M (d - g s)),
    the negative log-likelihood of one detscan under the noise model
    P_k = sigma0^2 (1 + (f_k/fknee)^alpha) with n_corr marginalised (the
    likelihood of the gain conditional of paper Eq. `gibbsstart`, as a
    function of the map, the gain and xi_n).  Returns L and the gradients
    dL/dg, dL/d(sigma0, fknee, alpha), and the per-sample vector
    v = M C^T (rhat / P) with dL/ds = -g v (so dL/dm = -g P^T v)."""
    n = len(d)
    M = np.asarray(mask, np.float64)
    f = dct_freqs(n, fsamp)
    r = M * (np.asarray(d, np.float64) - gain * np.asarray(s, np.float64))
    rh = dct(r)
    k = slice(1, n)
    x = (f[k] / fknee) ** alpha
    P = sigma0 ** 2 * (1.0 + x)
    L = 0.5 * float(np.sum(rh[k] ** 2 / P + np.log(P)))
    w = np.zeros(n)
    w[k] = rh[k] / P
    v = M * idct(w)
    dLdg = -float(np.dot(M * np.asarray(s, np.float64), v))
    c = 0.5 * (1.0 / P - rh[k] ** 2 / P ** 2)
    dP_ds = 2.0 * P / sigma0
    dP_dfk = -sigma0 ** 2 * alpha * x / fknee
    dP_da = sigma0 ** 2 * x * np.log(f[k] / fknee)
    return dict(L=L, dg=dLdg, dpsd=np.array([np.sum(c * dP_ds), np.sum(c * dP_dfk), np.sum(c * dP_da)]),
                v=v)


def chi2_band(map_tqu, pix, psi, d, gains, mask, psd, offsets, ndet, fsamp) -> dict:
    """Sum over detscans of chi2_detscan, with s = P m (unit gain) and the map
    gradient dL/dm = -P^T(g v) accumulated by binning (the adjoint of
    ``project``).  Returns L, dm (3, npix), dg (ndetscan), dpsd (ndet, 3)."""
    npix = map_tqu.shape[1]
    s = project(map_tqu, pix, psi)
    L = 0.0
    dg = np.zeros(len(offsets) - 1)
    dpsd = np.zeros((ndet, 3))
    gv = np.zeros(len(d))
    for q in range(len(offsets) - 1):
        a, b = int(offsets[q]), int(offsets[q + 1])
        det = q % ndet
        res = chi2_detscan(d[a:b], s[a:b], gains[q], mask[a:b], *psd[det], fsamp)
        L += res["L"]
        dg[q] = res["dg"]
        dpsd[det] += res["dpsd"]
        gv[a:b] = gains[q] * res["v"]
    c, sn = psi_trig_table()
    pix = np.asarray(pix, np.int64)
    b_ = np.asarray(psi, np.int64)
    dm = -np.stack([np.bincount(pix, weights=gv, minlength=npix),
                    np.bincount(pix, weights=gv * c[b_], minlength=npix),
                    np.bincount(pix, weights=gv * sn[b_], minlength=npix)])
    return dict(L=L, dm=dm, dg=dg, dpsd=dpsd)


# ============================================================================
# A10. noise PSD step: (f_knee, alpha) of each detector given n_corr
# ============================================================================
#
# Reading (the paper defers the noise sampler to its noise companion paper;
# Sect. 5 lists the noise PSD step among the TOD steps, and the Gibbs chain
# of Eq. `gibbsstart` conditions xi_n on n_corr): with sigma0 held fixed,
# each detector's (ln f_knee, alpha) is drawn from
#   p(ln f_knee, alpha | n_corr) ~ L(f_knee, alpha) 1{(ln f_knee, alpha) in BOX},
#   ln L = -1/2 sum_{q of the detector} sum_{k>=1} [ xhat_{q,k}^2 / Pc_{q,k}
#                                                      + ln Pc_{q,k} ],
#   Pc_{q,k} = sigma0^2 (f_{q,k} / f_knee)^alpha,  xhat_q = C n_corr_q,
# i.e. the Gaussian density of n_corr under its 1/f prior, the offset mode
# excluded as everywhere (reading 4).  Sampler: nsteps random-walk Metropolis
# steps on (ln f_knee, alpha) per call.

PSD_BOX = ((math.log(1e-4), math.log(10.0)), (-4.0, -0.25))


def psd_loglike(spectra, lengths, fsamp: float, sigma0: float, fknee: float, alpha: float) -> float:
    """ln L of one detector: spectra[j] = C n_corr of its j-th detscan (the
    orthonormal DCT-II, length lengths[j]), modes k >= 1; the definition
    above, term by term in FP64."""
    tot = 0.0
    for xh, n in zip(spectra, lengths):
        f = dct_freqs(int(n), fsamp)[1:]
        Pc = sigma0 ** 2 * (f / fknee) ** alpha
        x = np.asarray(xh, np.float64)[1:int(n)]
        tot += float(np.sum(x * x / Pc + np.log(Pc)))
    return -0.5 * tot


def psd_proposal(seed: int, band: int, det: int, step: int, it: int) -> tuple:
    """The random numbers of Metropolis step `step` of detector det at Gibbs
    iteration it: Philox block (step, det, PSD, it) with key (seed, band);
    words 0 and 1 give 53-bit uniforms u1, u2 and the normal pair
    (sqrt(-2 ln u1) cos 2 pi u2, sqrt(-2 ln u1) sin 2 pi u2); word 2 gives
    the 53-bit acceptance uniform."""
    w = philox4x64([step, det, PURPOSE_PSD, it], [seed, band])
    u1 = (float(w[0] >> np.uint64(11)) + 0.5) * 2.0 ** -53
    u2 = (float(w[1] >> np.uint64(11)) + 0.5) * 2.0 ** -53
    ua = (float(w[2] >> np.uint64(11)) + 0.5) * 2.0 ** -53
    r = math.sqrt(-2.0 * math.log(u1))
    return r * math.cos(2.0 * math.pi * u2), r * math.sin(2.0 * math.pi * u2), ua


def psd_in_box(lnfk: float, alpha: float) -> bool:
    return PSD_BOX[0][0] <= lnfk <= PSD_BOX[0][1] and PSD_BOX[1][0] <= alpha <= PSD_BOX[1][1]


def sample_noise_psd(spectra_by_det, lengths_by_det, fsamp: float, psd, seed: int, band: int, it: int,
                     nsteps: int, step_lnfk: float, step_alpha: float) -> tuple:
    """nsteps Metropolis steps on (ln f_knee, alpha) for every detector, from
    psd[det] = (sigma0, f_knee, alpha).  Step s proposes (ln f_knee + step_lnfk
    z1, alpha + step_alpha z2) with (z1, z2, u) = psd_proposal(..., s, it) and
    accepts iff the proposal is in PSD_BOX and ln u < ln L(proposal) -
    ln L(current).  Returns (psd_out (ndet, 3), accepted counts (ndet,))."""
    psd = np.array(psd, dtype=np.float64, copy=True)
    acc = np.zeros(len(psd), dtype=np.int64)
    for det in range(len(psd)):
        s0, fk, al = psd[det]
        lnfk = math.log(fk)
        cur = psd_loglike(spectra_by_det[det], lengths_by_det[det], fsamp, s0, fk, al)
        for step in range(nsteps):
            z1, z2, ua = psd_proposal(seed, band, det, step, it)
            lp, ap = lnfk + step_lnfk * z1, al + step_alpha * z2
            if not psd_in_box(lp, ap):
                continue
            new = psd_loglike(spectra_by_det[det], lengths_by_det[det], fsamp, s0, math.exp(lp), ap)
            if math.log(ua) < new - cur:
                lnfk, al, cur = lp, ap, new
                acc[det] += 1
        psd[det, 1], psd[det, 2] = math.exp(lnfk), al
    return psd, acc
