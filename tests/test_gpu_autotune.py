"""The launch-shape autotuner: it times every feasible candidate on a slice
of the band and returns the fastest, and the band then runs with it."""
import numpy as np
import pytest

import synth


@pytest.mark.gpu
def test_autotune_picks_a_measured_candidate():
    import torch
    import paper_2201_03509_gb300 as tg
    from paper_2201_03509_gb300.autotune import autotune
    cfg = synth.scaled(synth.CONFIGS["lfi30"], nscan=6, len_lo=20000, len_hi=40000)
    band = synth.make_band(cfg)
    ing = tg.ingest(band)
    m4 = np.zeros((band.npix, 4), np.float32)
    m4[:, :3] = band.map_tqu.T
    map_in = torch.from_numpy(m4).cuda()
    cands = [(0, 16), (4, 8), (8, 16), (3, 16)]
    c, r, t = autotune(cfg.nside, cfg.ndet, cfg.nscan, cfg.fsamp, ing["offsets"], ing["pix_streams"],
                       ing["psi_streams"], ing["tod"], ing["flag_words"], band.psd, map_in,
                       candidates=cands, nscan_sample=4, reps=2)
    assert (c, r) in t and set(t) <= set(cands) and len(t) >= 3
    assert t[(c, r)] == min(t.values())
    plan = tg.Plan(cfg.nside, cfg.ndet, cfg.nscan, cfg.fsamp, ing["offsets"], ing["pix_streams"],
                   ing["psi_streams"], tile_pairs=c, max_radix=r)
    assert plan.info()["tile_pairs"] == c
    plan.close()
