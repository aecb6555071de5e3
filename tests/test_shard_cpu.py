"""The band split over processes (paper Sect. 2.3-2.4), host logic on CPU:
the scan partition, and two gloo ranks that each bin their own scans with
the oracle (exact double-double partial sums), exchange pixel ranges through
paper_2201_03509_gb300.shard, add the partials in rank order, solve their
range and gather the map -- equal bit for bit to the unsharded normal
equations and map."""
import os
import socket

import numpy as np
import pytest

import oracle
import synth
from paper_2201_03509_gb300.shard import partition_scans, pixel_chunk


def test_partition_balances_samples():
    rng = np.random.default_rng(3)
    w = rng.integers(90_000, 140_000, size=1000)
    for n in (1, 2, 3, 8):
        b = partition_scans(w, n)
        assert b[0] == 0 and b[-1] == len(w) and np.all(np.diff(b) >= 1)
        loads = np.array([w[b[r]:b[r + 1]].sum() for r in range(n)])
        assert loads.max() - loads.min() <= 2 * w.max()
    # as many scans as ranks: one each
    assert list(partition_scans([5, 5, 5], 3)) == [0, 1, 2, 3]
    assert pixel_chunk(3072, 2) == 1536 and pixel_chunk(10, 3) == 4


def _inputs():
    cfg = synth.scaled(synth.CONFIGS["tiny"], nscan=6)
    band = synth.make_band(cfg)
    ing = oracle.ingest(band)
    off = ing["offsets"]
    nq = len(off) - 1
    pix = np.concatenate([band.pix[q][:off[q + 1] - off[q]] for q in range(nq)]).astype(np.int64)
    psi = np.concatenate([band.psi[q][:off[q + 1] - off[q]] for q in range(nq)]).astype(np.int64)
    mask = (~ing["flags"]).astype(np.float64)
    gs = oracle.per_sample(band.gain, off)
    s0 = oracle.per_sample(np.tile(band.psd[:, 0], cfg.nscan), off)
    w = mask * gs ** 2 / s0 ** 2
    v = mask * gs / s0 ** 2
    resid = ing["tod"].astype(np.float64)
    scan_samples = np.array([off[(s + 1) * cfg.ndet] - off[s * cfg.ndet] for s in range(cfg.nscan)])
    return cfg, band.npix, off, pix, psi, resid, (w, v), scan_samples


def _interleave(hi, lo):
    out = np.empty((hi.shape[0], 20))
    out[:, 0::2] = hi
    out[:, 1::2] = lo
    return out


def _rank(rank, ws, port, q):
    import torch
    import torch.distributed as dist
    from paper_2201_03509_gb300.shard import exchange_partials, gather_range
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        cfg, npix, off, pix, psi, resid, (w, v), scan_samples = _inputs()
        b = partition_scans(scan_samples, ws)
        t0, t1 = int(off[b[rank] * cfg.ndet]), int(off[b[rank + 1] * cfg.ndet])
        hi, lo = oracle.bin_partials(npix, pix[t0:t1], psi[t0:t1], resid[t0:t1], (w[t0:t1], v[t0:t1]))
        parts = exchange_partials(torch.from_numpy(_interleave(hi, lo)), ws)
        A, bb, hits = oracle.combine_partials([(parts[r, :, 0::2].numpy(), parts[r, :, 1::2].numpy())
                                                for r in range(ws)])
        m, _, valid = oracle.solve_maps(A, bb, hits, 1e-6)
        full_m = gather_range(torch.from_numpy(m), npix, ws)
        chunk = pixel_chunk(npix, ws)
        q.put((rank, A, bb, hits, full_m.numpy(), chunk))
    finally:
        dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_ranks_reduce_bit_for_bit():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    res = {}
    for _ in range(2):
        r, A, bb, hits, m, chunk = q.get(timeout=300)
        res[r] = (A, bb, hits, m, chunk)
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    cfg, npix, off, pix, psi, resid, wv, _ = _inputs()
    hi, lo = oracle.bin_partials(npix, pix, psi, resid, wv)
    A, bb, hits = oracle.combine_partials([(hi, lo)])
    m_ref, _, _ = oracle.solve_maps(A, bb, hits, 1e-6)
    chunk = res[0][4]
    for r in range(2):
        a, b_ = r * chunk, min(npix, (r + 1) * chunk)
        Ar, br, hr = res[r][0][:b_ - a], res[r][1][:b_ - a], res[r][2][:b_ - a]
        assert np.array_equal(Ar.view(np.uint64), A[a:b_].view(np.uint64))
        assert np.array_equal(br.view(np.uint64), bb[a:b_].view(np.uint64))
        assert np.array_equal(hr, hits[a:b_])
        assert np.array_equal(res[r][3].view(np.uint64), m_ref.view(np.uint64))
    # and the exact sums agree with the plain FP64 binning to rounding
    rA, rb = oracle.bin_maps(npix, pix, psi, resid, wv)
    assert np.allclose(A, rA, rtol=1e-12, atol=0) and np.allclose(bb, rb, rtol=1e-12, atol=1e-300)
