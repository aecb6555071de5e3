"""A band split over several processes (paper Sect. 2.3-2.4: the TOD is
distributed in chunks, each process coadds its own into the maps, and the
maps are synchronised once per sweep).

Partition: contiguous scan ranges of nearly equal sample counts (a scan's
detectors stay together, as they share a Huffman code).  Exchange, once per
Gibbs step: every process bins its detscans into per-pixel double-double
partial sums (tod_bin_partial), sends each process the partials of its
pixel range (all-to-all), the receiver adds them in rank order and rounds
once (tod_combine_partials), solves its range (tod_solve_range), and the
ranges are gathered into the map every process projects in the next step.
The combined normal equations equal those of the whole band on one
process (tod_bin) bit for bit.  This module holds only that host logic: the
collectives go through torch.distributed (gloo on CPU tensors, NCCL on
device tensors) and every sum runs in the library's kernels."""
from __future__ import annotations

import numpy as np


def partition_scans(scan_samples, nranks: int) -> np.ndarray:
    """Boundaries b[0] = 0 <= ... <= b[nranks] = nscan: rank r takes scans
    [b[r], b[r+1]); each boundary is the scan edge nearest to r/nranks of
    the band's samples (never empty while there are at least as many scans
    as ranks)."""
    w = np.asarray(scan_samples, dtype=np.float64)
    nscan = len(w)
    if nranks < 1:
        raise ValueError("nranks >= 1")
    cum = np.concatenate([[0.0], np.cumsum(w)])
    b = [0]
    for r in range(1, nranks):
        target = cum[-1] * r / nranks
        i = int(np.searchsorted(cum, target))
        if i > 0 and abs(cum[i - 1] - target) <= abs(cum[min(i, nscan)] - target):
            i -= 1
        lo = b[-1] + (1 if nscan - b[-1] > nranks - r else 0)     # leave at least one scan per rank
        hi = nscan - (nranks - r)
        b.append(int(min(max(i, lo), max(lo, hi))))
    b.append(nscan)
    return np.array(b, dtype=np.int64)


def pixel_chunk(npix: int, nranks: int) -> int:
    """Pixels per rank range (the last range padded to this size)."""
    return -(-npix // nranks)


def exchange_partials(part, nranks: int, group=None):
    """part: this rank's [npix, 20] double-double partials.  Returns the
    [nranks, chunk, 20] partials of this rank's pixel range, row r from rank
    r (all-to-all; padding pixels are zero)."""
    import torch
    import torch.distributed as dist
    npix = part.shape[0]
    chunk = pixel_chunk(npix, nranks)
    send = torch.zeros((nranks * chunk, 20), dtype=part.dtype, device=part.device)
    send[:npix] = part
    recv = torch.empty_like(send)
    if nranks == 1:
        recv.copy_(send)
    else:
        dist.all_to_all_single(recv, send, group=group)
    return recv.view(nranks, chunk, 20)


def gather_range(chunk_tensor, npix: int, nranks: int, group=None):
    """All ranks' [..., chunk] (or [chunk, ...]) range results gathered and
    concatenated along the pixel axis (dim 0 for [chunk, k], dim -1 for
    [k, chunk]), trimmed to npix."""
    import torch
    import torch.distributed as dist
    parts = [torch.empty_like(chunk_tensor) for _ in range(nranks)]
    if nranks == 1:
        parts[0].copy_(chunk_tensor)
    else:
        dist.all_gather(parts, chunk_tensor.contiguous(), group=group)
    if chunk_tensor.dim() == 2 and chunk_tensor.shape[0] == 3 and chunk_tensor.shape[1] != 3:
        return torch.cat(parts, dim=1)[:, :npix].contiguous()
    return torch.cat(parts, dim=0)[:npix].contiguous()


class ShardedMaps:
    """The per-step map reduction of one rank: partials of its own
    detscans in, the solved map of the whole band out (every rank)."""

    def __init__(self, plan, nranks: int, rank: int, group=None):
        import torch
        self.plan, self.nranks, self.rank, self.group = plan, nranks, rank, group
        dev = torch.device("cuda", plan.device)
        npix = plan.npix
        self.chunk = pixel_chunk(npix, nranks)
        c = self.chunk
        f64 = torch.float64
        self.part = torch.empty((npix, 20), dtype=f64, device=dev)
        self.A = torch.empty((c, 6), dtype=f64, device=dev)
        self.b = torch.empty((c, 3), dtype=f64, device=dev)
        self.hits = torch.empty(c, dtype=torch.int32, device=dev)
        self.map_c = torch.empty((3, c), dtype=f64, device=dev)
        self.map32_c = torch.empty((c, 4), dtype=torch.float32, device=dev)
        self.valid_c = torch.empty(c, dtype=torch.uint8, device=dev)

    def reduce_and_solve(self, psi, d, ncorr, gain, flags, psd, rcond_min: float = 1e-6):
        """Bin this rank's detscans, reduce over ranks, solve this rank's
        pixel range, gather.  Returns (map [3, npix] float64, map32 [npix, 4]
        float32, valid [npix] uint8)."""
        from . import combine_partials, solve_range
        self.plan.bin_partial(psi, d, ncorr, gain, flags, psd, self.part)
        parts = exchange_partials(self.part, self.nranks, self.group)
        combine_partials(parts, self.A, self.b, self.hits)
        solve_range(self.A, self.b, self.hits, rcond_min, self.map_c, self.map32_c, None, self.valid_c)
        npix = self.plan.npix
        return (gather_range(self.map_c, npix, self.nranks, self.group),
                gather_range(self.map32_c, npix, self.nranks, self.group),
                gather_range(self.valid_c, npix, self.nranks, self.group))
