"""Measured choice of the transform tile shape: the column pairs per tile of
the column passes (tile_pairs) and the largest Stockham radix, timed on a
slice of the band's own detscans (the first scans of the band, every
detector) through the same gain and n_corr calls the Gibbs step makes.  The
plan's own choice (tile_pairs = 0) is always a candidate, so the result is
never slower on the slice than the default."""
from __future__ import annotations

import numpy as np

from . import MODE_DRAW, Plan, Rng


def _slice_streams(st: dict, ndet: int, nscan_sub: int) -> dict:
    """The compressed streams of the first nscan_sub scans."""
    nq = ndet * nscan_sub
    w1, b1, s1 = int(st["word_off"][nq]), int(st["blk_off"][nq]), int(st["sym_off"][nscan_sub])
    return dict(words=st["words"][:w1], word_off=st["word_off"][:nq + 1], nbits=st["nbits"][:nq],
                blk_off=st["blk_off"][:nq + 1], ckpt_bit=st["ckpt_bit"][:b1], ckpt_val=st["ckpt_val"][:b1],
                sym_off=st["sym_off"][:nscan_sub + 1], sym_vals=st["sym_vals"][:s1],
                sym_len=st["sym_len"][:s1])


def autotune(nside: int, ndet: int, nscan: int, fsamp: float, offsets: np.ndarray, pix_streams: dict,
             psi_streams: dict, tod: np.ndarray, flag_words: np.ndarray, psd: np.ndarray, map32,
             candidates=None, nscan_sample: int = 48, reps: int = 3, device: int = 0):
    """Time (tile_pairs, max radix) candidates; returns (tile_pairs,
    max_radix, {(T, R): ms per gain + n_corr pass over the slice})."""
    import torch
    nsub = max(1, min(nscan, nscan_sample))
    nq = ndet * nsub
    off = np.ascontiguousarray(offsets[:nq + 1], dtype=np.int64)
    N = int(off[-1])
    pix_s, psi_s = _slice_streams(pix_streams, ndet, nsub), _slice_streams(psi_streams, ndet, nsub)
    dev = torch.device("cuda", device)
    d = torch.from_numpy(np.ascontiguousarray(tod[:N], np.float32)).to(dev)
    nw = (N + 31) // 32
    fl = torch.from_numpy(np.ascontiguousarray(flag_words[:nw], np.uint32).view(np.int32)).to(dev)
    ps = torch.from_numpy(np.ascontiguousarray(psd, np.float64)).to(dev)
    pix = torch.empty(N, dtype=torch.int32, device=dev)
    psi = torch.empty(N, dtype=torch.int16, device=dev)
    s = torch.empty(N, dtype=torch.float32, device=dev)
    x = torch.empty(N, dtype=torch.float32, device=dev)
    g = torch.zeros(nq, dtype=torch.float64, device=dev)
    its = torch.zeros(nq, dtype=torch.int32, device=dev)
    if candidates is None:
        candidates = [(t, r) for t in (0, 4, 8) for r in (8, 16)]
    timings = {}
    for (c, r) in candidates:
        try:
            plan = Plan(nside, ndet, nsub, fsamp, off, pix_s, psi_s, tile_pairs=c, device=device, max_radix=r)
        except Exception:
            continue                        # no split of these lengths for this radix
        try:
            plan.decode(pix, psi)
            plan.project(map32, pix, psi, None, s)

            def one(it):
                rng = Rng(1, 0, it)
                plan.sample_gain(d, s, fl, ps, rng, MODE_DRAW, g)
                plan.sample_ncorr(d, s, g, fl, ps, rng, MODE_DRAW, x, its)

            one(0)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for k in range(reps):
                one(1 + k)
            e1.record()
            torch.cuda.synchronize()
            plan.status()
            timings[(c, r)] = e0.elapsed_time(e1) / reps
        finally:
            plan.close()
    if not timings:
        raise RuntimeError("no transform tile shape fits this band")
    best = min(timings, key=timings.get)
    return best[0], best[1], timings
