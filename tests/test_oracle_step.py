"""Pins of the oracle's whole Gibbs TOD step (paper Listing `code:gibbs`
step 1: decode, sample gain, sample n_corr, bin, solve)."""
import numpy as np

import oracle


def test_step_noiseless_mean_mode(tiny_band, tiny_ingest):
    """Noise-free d = g P m: the conditional-mean gain is the true gain, the
    correlated-noise mean vanishes and the solved map is m."""
    band = tiny_band
    ing = dict(tiny_ingest)
    off = ing["offsets"]
    pix = oracle.decode_band(ing["pix_streams"], off, 1)
    psi = oracle.decode_band(ing["psi_streams"], off, 1)
    d = oracle.project(band.map_tqu, pix, psi, oracle.per_sample(band.gain, off))
    ing["tod"] = d            # FP64 data: exactness is the point here
    res = oracle.gibbs_tod_step(ing, band.cfg, band.npix, band.map_tqu, band.psd, 1, 0, 0,
                                mode=oracle.MODE_MEAN)
    assert np.allclose(res["gain"], band.gain, rtol=1e-11)
    assert max(np.abs(x).max() for x in res["ncorr"].values()) < 1e-14
    ok = res["valid"] > 0
    assert np.abs(res["map"][:, ok] - band.map_tqu[:, ok]).max() < 1e-10 * np.abs(band.map_tqu).max()


def test_step_deterministic_and_counter_keyed(tiny_band, tiny_ingest):
    band = tiny_band
    r1 = oracle.gibbs_tod_step(tiny_ingest, band.cfg, band.npix, band.map_tqu, band.psd, 5, 0, 3,
                               detscans=[0, 1])
    r2 = oracle.gibbs_tod_step(tiny_ingest, band.cfg, band.npix, band.map_tqu, band.psd, 5, 0, 3,
                               detscans=[0, 1])
    r3 = oracle.gibbs_tod_step(tiny_ingest, band.cfg, band.npix, band.map_tqu, band.psd, 5, 0, 4,
                               detscans=[0, 1])
    assert np.array_equal(r1["gain"], r2["gain"]) and np.array_equal(r1["A"], r2["A"])
    assert not np.array_equal(r1["gain"][:2], r3["gain"][:2])
