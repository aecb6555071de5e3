"""The band split into scan ranges on the GPU: each range's plan bins its
own detscans into double-double partials (tod_bin_partial), the partials
are added in rank order (tod_combine_partials) and solved per pixel range
(tod_solve_range); the normal equations and the map equal tod_bin and
tod_solve_maps of the whole band bit for bit."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


def test_two_scan_ranges_combine_bit_for_bit():
    torch = pytest.importorskip("torch")
    import paper_2201_03509_gb300 as tg
    from paper_2201_03509_gb300.shard import partition_scans, pixel_chunk
    cfg = synth.scaled(synth.CONFIGS["lfi30"], nscan=5, len_lo=9000, len_hi=30000, nside=64)
    band = synth.make_band(cfg)
    ing = tg.ingest(band)
    off = ing["offsets"]
    dev = torch.device("cuda:0")
    npix = band.npix
    rng = np.random.default_rng(2)
    N = int(off[-1])
    x = (1e-4 * rng.standard_normal(N)).astype(np.float32)
    gains = band.gain.copy()
    whole = tg.Plan(cfg.nside, cfg.ndet, cfg.nscan, cfg.fsamp, off, ing["pix_streams"], ing["psi_streams"])
    pix = torch.empty(N, dtype=torch.int32, device=dev)
    psi = torch.empty(N, dtype=torch.int16, device=dev)
    whole.decode(pix, psi)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    psd = t(band.psd)
    A = torch.empty((npix, 6), dtype=torch.float64, device=dev)
    b = torch.empty((npix, 3), dtype=torch.float64, device=dev)
    h = torch.empty(npix, dtype=torch.int32, device=dev)
    whole.bin(psi, t(ing["tod"]), t(x), t(gains), t(ing["flag_words"].view(np.int32)), psd, A, b, h)
    m = torch.empty((3, npix), dtype=torch.float64, device=dev)
    va = torch.empty(npix, dtype=torch.uint8, device=dev)
    whole.solve_maps(A, b, h, 1e-6, m, None, None, va)
    whole.status()
    # two scan ranges, each its own plan over its own samples
    scan_samples = np.array([off[(s + 1) * cfg.ndet] - off[s * cfg.ndet] for s in range(cfg.nscan)])
    bnd = partition_scans(scan_samples, 2)
    parts = torch.empty((2, npix, 20), dtype=torch.float64, device=dev)
    for r in range(2):
        s0, s1 = int(bnd[r]), int(bnd[r + 1])
        q0, q1 = s0 * cfg.ndet, s1 * cfg.ndet
        t0, t1 = int(off[q0]), int(off[q1])
        sub = synth.Band(cfg=synth.scaled(cfg, nscan=s1 - s0), npix=npix, map_tqu=band.map_tqu,
                         scan_len=band.scan_len[s0:s1], gain=band.gain[q0:q1], psd=band.psd,
                         pix=band.pix[q0:q1], psi=band.psi[q0:q1], flags=band.flags[q0:q1], tod=band.tod[q0:q1])
        sing = tg.ingest(sub)
        assert np.array_equal(sing["offsets"], off[q0:q1 + 1] - off[q0])
        plan = tg.Plan(cfg.nside, cfg.ndet, s1 - s0, cfg.fsamp, sing["offsets"], sing["pix_streams"],
                       sing["psi_streams"])
        spix = torch.empty(t1 - t0, dtype=torch.int32, device=dev)
        spsi = torch.empty(t1 - t0, dtype=torch.int16, device=dev)
        plan.decode(spix, spsi)
        plan.bin_partial(spsi, t(sing["tod"]), t(x[t0:t1]), t(gains[q0:q1]),
                         t(sing["flag_words"].view(np.int32)), psd, parts[r])
        plan.status()
        plan.close()
    A2 = torch.empty_like(A)
    b2 = torch.empty_like(b)
    h2 = torch.empty_like(h)
    tg.combine_partials(parts, A2, b2, h2)
    assert torch.equal(A2, A) and torch.equal(b2, b) and torch.equal(h2, h)
    # the solve by pixel ranges equals the whole-map solve
    c = pixel_chunk(npix, 2)
    m2 = torch.empty((3, npix), dtype=torch.float64, device=dev)
    for r in range(2):
        a, e = r * c, min(npix, (r + 1) * c)
        mr = torch.empty((3, e - a), dtype=torch.float64, device=dev)
        tg.solve_range(A2[a:e].contiguous(), b2[a:e].contiguous(), h2[a:e].contiguous(), 1e-6, mr)
        m2[:, a:e] = mr
    torch.cuda.synchronize()
    assert torch.equal(m2, m)
    whole.close()
