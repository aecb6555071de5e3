"""GB300 Gibbs TOD step (Commander3 / BeyondPlanck, arXiv 2201.03509).

Thin Python binding over the C ABI in ``include/todgibbs.h`` (library
``_build/libtodgibbs.so``, built by ``build()``): argument marshalling only.
Every step of the TOD path runs in the library's CUDA kernels; device arrays
are torch tensors, streams are torch streams.  There is no CPU fallback: if
the library is missing the calls raise.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from ._build import LIB as _LIB_PATH, build as _build_lib

__all__ = ["build", "lib", "fft_length", "huff_encode", "ingest", "ingest_data", "pack_flags", "Plan", "Rng",
           "TodError", "MODE_DRAW", "MODE_MEAN", "N_PSI", "CKPT_BLOCK", "PREC_NONE", "PREC_BLOCKS",
           "PREC_TWO_LEVEL"]

MODE_DRAW = 0
MODE_MEAN = 1
PREC_NONE, PREC_BLOCKS, PREC_TWO_LEVEL = 0, 1, 2      # n_corr CG preconditioner (set_preconditioner)
N_PSI = 4096
CKPT_BLOCK = 512

_P = ctypes.c_void_p
_i32, _i64, _u64, _f64 = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, ctypes.c_double


class TodError(RuntimeError):
    def __init__(self, code: int, what: str = ""):
        msg = lib().tod_status_string(code).decode() if _lib is not None else str(code)
        super().__init__("%s: %s (%d)" % (what, msg, code))
        self.code = code


class _HuffStreams(ctypes.Structure):
    _fields_ = [("words", _P), ("nwords", _i64), ("word_off", _P), ("nbits", _P), ("blk_off", _P),
                ("ckpt_bit", _P), ("ckpt_val", _P), ("nblk", _i64), ("sym_off", _P), ("sym_vals", _P),
                ("sym_len", _P), ("nsym", _i64)]


class _HuffBuffers(ctypes.Structure):
    _fields_ = [("words", ctypes.POINTER(ctypes.c_uint32)), ("nwords", _i64),
                ("word_off", ctypes.POINTER(_i64)), ("nbits", ctypes.POINTER(_i64)),
                ("blk_off", ctypes.POINTER(_i64)), ("ckpt_bit", ctypes.POINTER(ctypes.c_uint32)),
                ("ckpt_val", ctypes.POINTER(_i32)), ("nblk", _i64),
                ("sym_off", ctypes.POINTER(_i64)), ("sym_vals", ctypes.POINTER(_i32)),
                ("sym_len", ctypes.POINTER(ctypes.c_uint8)), ("nsym", _i64)]


class _BandDesc(ctypes.Structure):
    _fields_ = [("nside", _i32), ("ndet", _i32), ("nscan", _i32), ("n_psi", _i32), ("fsamp", _f64),
                ("offsets", _P), ("pix", _HuffStreams), ("psi", _HuffStreams),
                ("tile_pairs", _i32), ("device", _i32), ("max_radix", _i32)]


class _DataDesc(ctypes.Structure):
    _fields_ = [("tod", _HuffStreams), ("tod_scale", _P), ("flag", _HuffStreams), ("flag_select", ctypes.c_uint32)]


class Rng(ctypes.Structure):
    """Counter-based random streams: key (seed, band), counter carries the
    Gibbs iteration."""
    _fields_ = [("seed", _u64), ("band", _u64), ("gibbs_iter", _u64), ("gibbs_iter_dev", _P)]


_lib = None

SYMBOLS = ["tod_status_string", "tod_fft_length", "tod_huff_encode", "tod_huff_free",
           "tod_plan_create", "tod_plan_destroy", "tod_plan_info", "tod_plan_status",
           "tod_plan_set_schedule", "tod_plan_set_preconditioner", "tod_chi2", "tod_project_adjoint",
           "tod_project_f64", "tod_bin_partial",
           "tod_combine_partials", "tod_solve_range", "tod_decode", "tod_project", "tod_sample_gain", "tod_sample_ncorr", "tod_bin",
           "tod_solve_maps", "tod_ncorr_static_setup", "tod_sample_ncorr_static", "tod_ncorr_prepare",
           "tod_sample_ncorr_prepared", "tod_sample_noise_psd", "tod_plan_set_ncorr_spectrum",
           "tod_plan_attach_data", "tod_decode_data", "tod_sample_gain_smooth", "tod_kernel_name",
           "tod_plan_set_kernel_timing", "tod_plan_kernel_times", "tod_plan_binning_info"]


def build(force: bool = False) -> str:
    """Compile the CUDA library for sm_103a into the package's _build/."""
    global _lib
    _lib = None
    return _build_lib(force=force)


def lib():
    """The loaded C library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(_LIB_PATH):
            raise RuntimeError("libtodgibbs.so is not built: call paper_2201_03509_gb300.build()")
        L = ctypes.CDLL(_LIB_PATH)
        L.tod_status_string.argtypes = [_i32]
        L.tod_status_string.restype = ctypes.c_char_p
        L.tod_fft_length.argtypes = [_i64]
        L.tod_fft_length.restype = _i64
        L.tod_huff_encode.argtypes = [_i32, _i32, _P, _P, ctypes.POINTER(_HuffBuffers)]
        L.tod_huff_free.argtypes = [ctypes.POINTER(_HuffBuffers)]
        L.tod_huff_free.restype = None
        L.tod_plan_create.argtypes = [ctypes.POINTER(_P), ctypes.POINTER(_BandDesc)]
        L.tod_plan_destroy.argtypes = [_P]
        L.tod_plan_info.argtypes = [_P, _P, _P, _P, _P, _P]
        L.tod_plan_status.argtypes = [_P, _P]
        L.tod_plan_set_schedule.argtypes = [_P, _i32]
        L.tod_plan_set_preconditioner.argtypes = [_P, _i32]
        L.tod_kernel_name.argtypes = [_i32]
        L.tod_kernel_name.restype = ctypes.c_char_p
        L.tod_plan_set_kernel_timing.argtypes = [_P, _i32]
        L.tod_plan_kernel_times.argtypes = [_P, _P, _P]
        L.tod_plan_binning_info.argtypes = [_P, _P, _P]
        L.tod_decode.argtypes = [_P, _P, _P, _P]
        L.tod_project.argtypes = [_P, _P, _P, _P, _P, _P, _P]
        L.tod_sample_gain.argtypes = [_P, _P, _P, _P, _P, Rng, _i32, _P, _P, _P, _P]
        L.tod_sample_ncorr.argtypes = [_P, _P, _P, _P, _P, _P, Rng, _i32, _f64, _i32, _P, _P, _P]
        L.tod_bin.argtypes = [_P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P]
        L.tod_solve_maps.argtypes = [_P, _P, _P, _P, _f64, _P, _P, _P, _P, _P]
        L.tod_chi2.argtypes = [_P, _P, _P, _P, _P, _P, _i32, _P, _P, _P, _P, _P, _P]
        L.tod_project_adjoint.argtypes = [_P, _P, _P, _i32, _P, _P, _P]
        L.tod_project_f64.argtypes = [_P, _P, _P, _P, _P, _P, _P]
        L.tod_bin_partial.argtypes = [_P, _P, _P, _P, _P, _P, _P, _P, _P]
        L.tod_combine_partials.argtypes = [_P, _i32, _i64, _P, _P, _P, _P]
        L.tod_solve_range.argtypes = [_i64, _P, _P, _P, _f64, _P, _P, _P, _P, _P]
        L.tod_ncorr_static_setup.argtypes = [_P, _P]
        L.tod_sample_ncorr_static.argtypes = [_P, _P, _P, _P, _P, _P, Rng, _i32, _f64, _i32, _P, _P, _P]
        L.tod_ncorr_prepare.argtypes = [_P, _P, _P]
        L.tod_sample_ncorr_prepared.argtypes = [_P, _P, _P, _P, _P, _P, Rng, _i32, _f64, _i32, _P, _P, _P]
        L.tod_sample_noise_psd.argtypes = [_P, _P, _P, Rng, _i32, _f64, _f64, _P, _P, _P, _P]
        L.tod_plan_set_ncorr_spectrum.argtypes = [_P, _P]
        L.tod_plan_attach_data.argtypes = [_P, ctypes.POINTER(_DataDesc)]
        L.tod_decode_data.argtypes = [_P, _P, _P, _P]
        L.tod_sample_gain_smooth.argtypes = [_P, _P, _P, _P, Rng, _i32, _f64, _i32, _P, _P, _P]
        for name in SYMBOLS:
            if name not in ("tod_status_string", "tod_fft_length", "tod_huff_free", "tod_kernel_name"):
                getattr(L, name).restype = _i32
        _lib = L
    return _lib


def _check(code: int, what: str):
    if code != 0:
        raise TodError(code, what)


def fft_length(n: int) -> int:
    return int(lib().tod_fft_length(int(n)))


def _arr(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


def huff_encode(ndet: int, nscan: int, offsets: np.ndarray, values: np.ndarray) -> dict:
    """Compress one pointing stream kind (host).  Returns numpy arrays with
    the stream layout documented in todgibbs.h."""
    offsets = _arr(offsets, np.int64)
    values = _arr(values, np.int32)
    buf = _HuffBuffers()
    _check(lib().tod_huff_encode(ndet, nscan, offsets.ctypes.data, values.ctypes.data,
                                 ctypes.byref(buf)), "tod_huff_encode")
    nq = ndet * nscan

    def take(ptr, n, dt):
        return np.ctypeslib.as_array(ptr, shape=(n,)).astype(dt, copy=True) if n else np.zeros(0, dt)

    try:
        out = dict(words=take(buf.words, buf.nwords, np.uint32),
                   word_off=take(buf.word_off, nq + 1, np.int64),
                   nbits=take(buf.nbits, nq, np.int64),
                   blk_off=take(buf.blk_off, nq + 1, np.int64),
                   ckpt_bit=take(buf.ckpt_bit, buf.nblk, np.uint32),
                   ckpt_val=take(buf.ckpt_val, buf.nblk, np.int32),
                   sym_off=take(buf.sym_off, nscan + 1, np.int64),
                   sym_vals=take(buf.sym_vals, buf.nsym, np.int32),
                   sym_len=take(buf.sym_len, buf.nsym, np.uint8))
    finally:
        lib().tod_huff_free(ctypes.byref(buf))
    return out


def combine_partials(parts, A_out, b_out, hits_out, stream=None):
    """Rank-order double-double sum of parts [nparts, np, 20] into A [np, 6],
    b [np, 3], hits [np] (todgibbs.h: tod_combine_partials)."""
    _check(lib().tod_combine_partials(_ptr(parts), int(parts.shape[0]), int(parts.shape[1]), _ptr(A_out),
                                      _ptr(b_out), _ptr(hits_out), _stream(stream)), "tod_combine_partials")


def solve_range(A, b, hits, rcond_min, map_out, map_f32_out=None, rcond_out=None, valid_out=None, stream=None):
    """The per-pixel solve of a pixel range (todgibbs.h: tod_solve_range);
    map_out float64 [3, np]."""
    _check(lib().tod_solve_range(int(A.shape[0]), _ptr(A), _ptr(b), _ptr(hits), float(rcond_min), _ptr(map_out),
                                 _ptr(map_f32_out), _ptr(rcond_out), _ptr(valid_out), _stream(stream)),
           "tod_solve_range")


def pack_flags(flagged: np.ndarray) -> np.ndarray:
    """Bool per sample (True = flagged) -> uint32 words, bit t&31 of word t>>5."""
    f = np.asarray(flagged, dtype=bool)
    pad = (-len(f)) % 32
    if pad:
        f = np.concatenate([f, np.zeros(pad, bool)])
    return np.packbits(f, bitorder="little").view("<u4").copy()


def ingest(band, data_streams: bool = False) -> dict:
    """Ingest of a synthetic band (not on the per-step path): truncate each
    scan to its FFT length (paper Sect. 4.2) and compress its pixel and psi
    streams (Sect. 4.1).  With ``data_streams`` the band's ADC counts and
    flag words are compressed too (``tod_streams``, ``tod_scale``,
    ``flag_streams``, ``flag_select``; the step then decodes d and the flags
    on the device)."""
    ndet, nscan = band.cfg.ndet, band.cfg.nscan
    nq = ndet * nscan
    nlen = np.array([fft_length(int(band.scan_len[q // ndet])) for q in range(nq)], dtype=np.int64)
    off = np.zeros(nq + 1, dtype=np.int64)
    off[1:] = np.cumsum(nlen)
    pix = np.concatenate([band.pix[q][:nlen[q]] for q in range(nq)]).astype(np.int32)
    psi = np.concatenate([band.psi[q][:nlen[q]] for q in range(nq)]).astype(np.int32)
    flags = np.concatenate([band.flags[q][:nlen[q]] for q in range(nq)])
    out = dict(offsets=off,
               pix_streams=huff_encode(ndet, nscan, off, pix),
               psi_streams=huff_encode(ndet, nscan, off, psi),
               tod=np.concatenate([band.tod[q][:nlen[q]] for q in range(nq)]).astype(np.float32),
               flags=flags, flag_words=pack_flags(flags))
    if data_streams:
        out.update(ingest_data(band, off))
    return out


def kernel_names() -> list:
    """The kernel classes of tod_plan_kernel_times, in id order."""
    out = []
    while True:
        nm = lib().tod_kernel_name(len(out))
        if nm is None:
            return out
        out.append(nm.decode())


def kept_lengths(cfg) -> np.ndarray:
    """FFT length (tod_fft_length) of every scan of a synthetic band."""
    import synth
    return np.array([fft_length(int(n)) for n in synth.raw_lengths(cfg)], dtype=np.int64)


def ingest_arrays(arr) -> dict:
    """ingest() for a band generated straight into concatenated arrays
    (synth.make_band_arrays with kept_lengths): compress its pixel and psi
    streams; the arrays are used in place (psi is widened to int32 for the
    coder)."""
    cfg = arr.cfg
    off = arr.offsets
    ndet = cfg.ndet
    nscan = (len(off) - 1) // ndet        # the generated scans (all, or a scan range)
    psi32 = np.empty(len(arr.psi), np.int32)
    np.copyto(psi32, arr.psi, casting="unsafe")
    out = dict(offsets=off,
               pix_streams=huff_encode(ndet, nscan, off, arr.pix),
               psi_streams=huff_encode(ndet, nscan, off, psi32),
               tod=arr.tod, flags=arr.flags, flag_words=pack_flags(arr.flags))
    del psi32
    return out


def ingest_data(band, offsets: np.ndarray) -> dict:
    """The band's detector data as ADC counts and its flags as flag words
    (from the synthetic generator), each compressed like the pointing
    (Sect. 4.1), over the ingest's offsets."""
    import synth
    ndet, nscan = band.cfg.ndet, band.cfg.nscan
    nlen = np.diff(offsets)
    nq = len(nlen)
    scale = synth.adc_quantum(band)
    counts = np.concatenate([synth.adc_counts(band.tod[q][:nlen[q]], scale[q]) for q in range(nq)])
    words = np.concatenate([synth.flag_words(band.cfg, q, band.flags[q][:nlen[q]]) for q in range(nq)])
    return dict(tod_streams=huff_encode(ndet, nscan, offsets, counts), tod_scale=scale,
                flag_streams=huff_encode(ndet, nscan, offsets, words), flag_select=synth.FLAG_SELECT)


def _streams(d: dict, keep: list) -> _HuffStreams:
    arrs = {k: _arr(d[k], dt) for k, dt in (("words", np.uint32), ("word_off", np.int64),
                                             ("nbits", np.int64), ("blk_off", np.int64),
                                             ("ckpt_bit", np.uint32), ("ckpt_val", np.int32),
                                             ("sym_off", np.int64), ("sym_vals", np.int32),
                                             ("sym_len", np.uint8))}
    keep.append(arrs)
    return _HuffStreams(arrs["words"].ctypes.data, len(arrs["words"]), arrs["word_off"].ctypes.data,
                        arrs["nbits"].ctypes.data, arrs["blk_off"].ctypes.data,
                        arrs["ckpt_bit"].ctypes.data, arrs["ckpt_val"].ctypes.data,
                        len(arrs["ckpt_bit"]), arrs["sym_off"].ctypes.data,
                        arrs["sym_vals"].ctypes.data, arrs["sym_len"].ctypes.data,
                        len(arrs["sym_vals"]))


def _ptr(t):
    """Device pointer of a torch tensor (or None -> NULL)."""
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("device tensor expected")
    if not t.is_contiguous():
        raise ValueError("contiguous tensor expected")
    return t.data_ptr()


def _stream(stream):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream


class Plan:
    """The band's TOD object on the GPU (todgibbs.h: tod_plan)."""

    def __init__(self, nside: int, ndet: int, nscan: int, fsamp: float, offsets: np.ndarray,
                 pix_streams: dict, psi_streams: dict, tile_pairs: int = 0, device: int = 0,
                 max_radix: int = 0):
        keep = []
        off = _arr(offsets, np.int64)
        keep.append(off)
        desc = _BandDesc(nside, ndet, nscan, N_PSI, float(fsamp), off.ctypes.data,
                         _streams(pix_streams, keep), _streams(psi_streams, keep),
                         int(tile_pairs), int(device), int(max_radix))
        h = _P()
        _check(lib().tod_plan_create(ctypes.byref(h), ctypes.byref(desc)), "tod_plan_create")
        self._h = h
        self.ndet, self.nscan, self.nq = ndet, nscan, ndet * nscan
        self.offsets = off.copy()
        self.nside = nside
        self.npix = 12 * nside * nside
        self.N = int(off[-1])
        self.device = device

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            lib().tod_plan_destroy(self._h)
            self._h = _P()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def toeplitz_prep_launches(self) -> int:
        """Launches of tod_ncorr_prepare: the gap kernel (fill, the FFT
        passes of length 2H, chunk sums, prefix tables) and the Durbin
        recursion, H the power-of-two reference length (>= 1024) covering
        the longest detscan."""
        h = 1024
        while h < int(np.diff(self.offsets).max()):
            h *= 2
        lg = (2 * h).bit_length() - 1
        return 1 + (lg + 1) // 2 + 2 + 1

    def info(self) -> dict:
        ns, nq, npix, cs, nb = _i64(), _i32(), _i32(), _i32(), _i64()
        _check(lib().tod_plan_info(self._h, ctypes.byref(ns), ctypes.byref(nq), ctypes.byref(npix),
                                   ctypes.byref(cs), ctypes.byref(nb)), "tod_plan_info")
        nr, nt = _i64(), _i32()
        _check(lib().tod_plan_binning_info(self._h, ctypes.byref(nr), ctypes.byref(nt)), "tod_plan_binning_info")
        return dict(nsamples=ns.value, ndetscan=nq.value, npix=npix.value, tile_pairs=cs.value,
                    device_bytes=nb.value, nruns=nr.value, nbin_tiles=nt.value)

    SCHED_PERSISTENT = 0
    SCHED_PER_SCAN = 1

    def set_schedule(self, schedule: int):
        _check(lib().tod_plan_set_schedule(self._h, int(schedule)), "tod_plan_set_schedule")

    def set_preconditioner(self, levels: int):
        """PREC_NONE, PREC_BLOCKS or PREC_TWO_LEVEL (the default) for the
        n_corr CG."""
        _check(lib().tod_plan_set_preconditioner(self._h, int(levels)), "tod_plan_set_preconditioner")

    def set_kernel_timing(self, on: bool):
        """Bracket every kernel launch of this plan with CUDA events on its
        stream (on: records cleared) or stop (records kept)."""
        _check(lib().tod_plan_set_kernel_timing(self._h, 1 if on else 0), "tod_plan_set_kernel_timing")

    def kernel_times(self) -> dict:
        """{kernel name: (milliseconds, launches)} of the launches recorded
        while timing was on (synchronises on their events)."""
        names = kernel_names()
        ms = np.zeros(len(names), np.float64)
        n = np.zeros(len(names), np.int32)
        _check(lib().tod_plan_kernel_times(self._h, ms.ctypes.data, n.ctypes.data), "tod_plan_kernel_times")
        return {nm: (float(ms[i]), int(n[i])) for i, nm in enumerate(names) if n[i] > 0}

    def status(self, raise_on_error: bool = True) -> np.ndarray:
        st = np.zeros(self.nq, dtype=np.int32)
        code = lib().tod_plan_status(self._h, st.ctypes.data)
        if raise_on_error and code != 0:
            raise TodError(code, "device status")
        return st

    # --- A1..A7 -------------------------------------------------------------
    def decode(self, pix_out, psi_out, stream=None):
        _check(lib().tod_decode(self._h, _ptr(pix_out), _ptr(psi_out), _stream(stream)), "tod_decode")

    def attach_data(self, tod_streams: dict, tod_scale, flag_streams: dict, flag_select: int):
        """Compressed ADC counts (with each detscan's quantum) and flag
        words of the band, copied to the device once."""
        keep = []
        scale = _arr(tod_scale, np.float64)
        keep.append(scale)
        desc = _DataDesc(_streams(tod_streams, keep), scale.ctypes.data, _streams(flag_streams, keep),
                         int(flag_select) & 0xFFFFFFFF)
        _check(lib().tod_plan_attach_data(self._h, ctypes.byref(desc)), "tod_plan_attach_data")

    def sample_gain_smooth(self, mu, sigma, prior, rng: Rng, mode, gain_out, cg_iters_out=None,
                           cg_tol: float = 1e-6, cg_maxiter: int = 200, stream=None):
        """Joint draw of each detector's scan gains under the smooth prior
        (prior: device float64[ndet, 2] = sigma_g, alpha_g)."""
        _check(lib().tod_sample_gain_smooth(self._h, _ptr(mu), _ptr(sigma), _ptr(prior), rng, int(mode),
                                            float(cg_tol), int(cg_maxiter), _ptr(gain_out), _ptr(cg_iters_out),
                                            _stream(stream)), "tod_sample_gain_smooth")

    def decode_data(self, d_out, flags_out, stream=None):
        _check(lib().tod_decode_data(self._h, _ptr(d_out), _ptr(flags_out), _stream(stream)),
               "tod_decode_data")

    def project(self, map_tqu4, pix, psi, gain, s_out, stream=None):
        _check(lib().tod_project(self._h, _ptr(map_tqu4), _ptr(pix), _ptr(psi), _ptr(gain),
                                 _ptr(s_out), _stream(stream)), "tod_project")

    def sample_gain(self, d, s, flags, psd, rng: Rng, mode, gain_out, mu_out=None, sigma_out=None,
                    stream=None):
        _check(lib().tod_sample_gain(self._h, _ptr(d), _ptr(s), _ptr(flags), _ptr(psd), rng, mode,
                                     _ptr(gain_out), _ptr(mu_out), _ptr(sigma_out), _stream(stream)),
               "tod_sample_gain")

    def sample_ncorr(self, d, s, gain, flags, psd, rng: Rng, mode, ncorr_out, cg_iters_out=None,
                     cg_tol: float = 0.0, cg_maxiter: int = 0, stream=None):
        _check(lib().tod_sample_ncorr(self._h, _ptr(d), _ptr(s), _ptr(gain), _ptr(flags), _ptr(psd),
                                      rng, mode, float(cg_tol), int(cg_maxiter), _ptr(ncorr_out),
                                      _ptr(cg_iters_out), _stream(stream)), "tod_sample_ncorr")

    def ncorr_prepare(self, psd, stream=None):
        """First half of sample_ncorr: the per-detector gap preconditioner
        tables from psd (may run on another stream; see the header)."""
        _check(lib().tod_ncorr_prepare(self._h, _ptr(psd), _stream(stream)), "tod_ncorr_prepare")

    def sample_ncorr_prepared(self, d, s, gain, flags, psd, rng: Rng, mode, ncorr_out, cg_iters_out=None,
                              cg_tol: float = 0.0, cg_maxiter: int = 0, stream=None):
        """Second half of sample_ncorr, with the tables of the last ncorr_prepare."""
        _check(lib().tod_sample_ncorr_prepared(self._h, _ptr(d), _ptr(s), _ptr(gain), _ptr(flags), _ptr(psd),
                                               rng, mode, float(cg_tol), int(cg_maxiter), _ptr(ncorr_out),
                                               _ptr(cg_iters_out), _stream(stream)), "tod_sample_ncorr_prepared")

    def set_ncorr_spectrum(self, spec_out):
        """Every following n_corr draw also writes its orthonormal DCT-II
        coefficients into spec_out (float32[N], mode order per detscan);
        None stops it.  The plan keeps a reference to the tensor."""
        self._spec_ref = spec_out
        _check(lib().tod_plan_set_ncorr_spectrum(self._h, _ptr(spec_out)), "tod_plan_set_ncorr_spectrum")

    def sample_noise_psd(self, spec, psd_in, rng: Rng, nsteps: int, step_lnfknee: float, step_alpha: float,
                         psd_out, accepted_out=None, loglike_out=None, stream=None):
        """nsteps Metropolis steps on (ln f_knee, alpha) of every detector
        from the n_corr spectra (row A10; see the header for the target)."""
        _check(lib().tod_sample_noise_psd(self._h, _ptr(spec), _ptr(psd_in), rng, int(nsteps), float(step_lnfknee),
                                          float(step_alpha), _ptr(psd_out), _ptr(accepted_out), _ptr(loglike_out),
                                          _stream(stream)), "tod_sample_noise_psd")

    def ncorr_static_setup(self) -> int:
        """Look up the fixed scratch array of sample_ncorr_static on this
        plan's device; returns the most samples one wave of the draw takes."""
        n = _i64()
        _check(lib().tod_ncorr_static_setup(self._h, ctypes.byref(n)), "tod_ncorr_static_setup")
        return n.value

    def sample_ncorr_static(self, d, s, gain, flags, psd, rng: Rng, mode, ncorr_out, cg_iters_out=None,
                            cg_tol: float = 0.0, cg_maxiter: int = 0, stream=None):
        """sample_ncorr with its scratch in the library's fixed device array
        (allocates nothing; calls on one device must not overlap)."""
        _check(lib().tod_sample_ncorr_static(self._h, _ptr(d), _ptr(s), _ptr(gain), _ptr(flags), _ptr(psd),
                                             rng, mode, float(cg_tol), int(cg_maxiter), _ptr(ncorr_out),
                                             _ptr(cg_iters_out), _stream(stream)), "tod_sample_ncorr_static")

    def bin(self, psi, d, ncorr, gain, flags, psd, A_out, b_out, hits_out, stream=None):
        _check(lib().tod_bin(self._h, _ptr(psi), _ptr(d), _ptr(ncorr), _ptr(gain), _ptr(flags),
                             _ptr(psd), _ptr(A_out), _ptr(b_out), _ptr(hits_out), _stream(stream)),
               "tod_bin")

    PREC_F32 = 0
    PREC_F64 = 1

    def bin_partial(self, psi, d, ncorr, gain, flags, psd, part_out, stream=None):
        """tod_bin with the per-pixel sums left as double-double pairs,
        part_out float64 [npix, 20] (todgibbs.h: tod_bin_partial)."""
        _check(lib().tod_bin_partial(self._h, _ptr(psi), _ptr(d), _ptr(ncorr), _ptr(gain), _ptr(flags), _ptr(psd),
                                     _ptr(part_out), _stream(stream)), "tod_bin_partial")

    def chi2(self, d, s, gain, flags, psd, chi2_out, dgain_out, total_out, dpsd_out, v_out=None,
             precision: int = 0, stream=None):
        """Per-detscan chi^2 and gain gradient, band total and per-detector
        PSD gradient (todgibbs.h: tod_chi2); v_out float32 or float64 [N]."""
        _check(lib().tod_chi2(self._h, _ptr(d), _ptr(s), _ptr(gain), _ptr(flags), _ptr(psd), int(precision),
                              _ptr(chi2_out), _ptr(dgain_out), _ptr(total_out), _ptr(dpsd_out), _ptr(v_out),
                              _stream(stream)), "tod_chi2")

    def project_f64(self, map3, pix, psi, gain, s_out, stream=None):
        """FP64 projection: map3 float64 [3, npix] -> s_out float64 [N]."""
        _check(lib().tod_project_f64(self._h, _ptr(map3), _ptr(pix), _ptr(psi), _ptr(gain), _ptr(s_out),
                                     _stream(stream)), "tod_project_f64")

    def pointing(self):
        """The plan's decoded pointing (pix int32[N], psi int16[N] device
        tensors), decoded once and kept."""
        import torch
        if getattr(self, "_pointing", None) is None:
            dev = torch.device("cuda", self.device)
            pix = torch.empty(self.N, dtype=torch.int32, device=dev)
            psi = torch.empty(self.N, dtype=torch.int16, device=dev)
            self.decode(pix, psi)
            self._pointing = (pix, psi)
        return self._pointing

    def project_adjoint(self, psi, y, gain, out, precision: int = 0, stream=None):
        """out[npix, 3] = P^T (g y) (todgibbs.h: tod_project_adjoint)."""
        _check(lib().tod_project_adjoint(self._h, _ptr(psi), _ptr(y), int(precision), _ptr(gain), _ptr(out),
                                         _stream(stream)), "tod_project_adjoint")

    def solve_maps(self, A, b, hits, rcond_min, map_out, map_f32_out=None, rcond_out=None,
                   valid_out=None, stream=None):
        _check(lib().tod_solve_maps(self._h, _ptr(A), _ptr(b), _ptr(hits), float(rcond_min),
                                    _ptr(map_out), _ptr(map_f32_out), _ptr(rcond_out),
                                    _ptr(valid_out), _stream(stream)), "tod_solve_maps")
