"""The multi-band Gibbs sweep (three bands shaped like the 30, 44 and 70 GHz
ones, scaled down so that the oracle can run every detscan) against the
oracle's own chain: each band's iterations carry the map from one to the
next, and every iteration's gains and map equal the oracle's Gibbs step on
the oracle's map of the previous iteration (relative 1e-5 for the gains,
1e-4 of the map's largest value; validity flags exact).  With the noise-PSD
step in the sweep the bands carry their noise parameters too: reruns are
identical and the parameters stay in the sampler's box."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

SEED, NIT = 31, 3


def _band_cfgs():
    t = synth.CONFIGS["tiny"]
    return [synth.scaled(t, nscan=8, len_lo=4096, len_hi=4700, flag_frac=0.02, seed=20220121),
            synth.scaled(t, nscan=8, ndet=2, fsamp=46.5, len_lo=5000, len_hi=6000, flag_frac=0.02, seed=20220122),
            synth.scaled(t, nscan=6, ndet=3, fsamp=78.8, nside=32, len_lo=7000, len_hi=8400, flag_frac=0.02,
                         seed=20220123)]


@pytest.fixture(scope="module")
def bands():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2201_03509_gb300 as tg
    out = []
    for b, cfg in enumerate(_band_cfgs()):
        band = synth.make_band(cfg)
        ing = tg.ingest(band)
        plan = tg.Plan(cfg.nside, cfg.ndet, cfg.nscan, cfg.fsamp, ing["offsets"], ing["pix_streams"],
                       ing["psi_streams"])
        out.append(dict(cfg=cfg, band=band, ing=ing, plan=plan, oing=oracle.ingest(band), band_id=b))
    return out


def _sweep(bands, psd_steps=0):
    from paper_2201_03509_gb300.sweep import BandChain, MultiBandSweep
    chains = [BandChain(B["plan"], B["band"].psd, B["ing"]["flag_words"], B["ing"]["tod"], B["band"].map_tqu,
                        B["band_id"], cg_tol=1e-7, psd_steps=psd_steps) for B in bands]
    return chains, MultiBandSweep(chains)


def test_sweep_chain_matches_oracle_chain(bands):
    chains, sw = _sweep(bands)
    omap = [B["band"].map_tqu.copy() for B in bands]
    for k in range(NIT):
        sw.run(1, SEED, it0=k)
        for B, c in zip(bands, chains):
            B["plan"].status()
            ref = oracle.gibbs_tod_step(B["oing"], B["cfg"], B["band"].npix, omap[B["band_id"]], B["band"].psd,
                                        SEED, B["band_id"], k)
            g = c.step.gain.cpu().numpy()
            np.testing.assert_allclose(g, ref["gain"], rtol=1e-5, atol=0)
            valid = c.step.valid.cpu().numpy()
            assert np.array_equal(valid, ref["valid"]), (B["band_id"], k)
            m = c.step.map.cpu().numpy()
            ok = ref["valid"] > 0
            assert ok.sum() > 0.5 * ok.size, (B["band_id"], k)
            scale = np.abs(ref["map"][:, ok]).max()
            assert np.abs(m[:, ok] - ref["map"][:, ok]).max() <= 1e-4 * scale, (B["band_id"], k)
            omap[B["band_id"]] = ref["map"]


def test_sweep_with_noise_psd_step_is_deterministic(bands):
    runs = []
    for rep in range(2):
        chains, sw = _sweep(bands, psd_steps=3)
        res = sw.run(2, SEED)
        assert res["samples_per_iteration"] == sum(B["plan"].N for B in bands)
        for B in bands:
            B["plan"].status()
        runs.append([(c.step.psd.cpu().numpy(), c.step.map.cpu().numpy()) for c in chains])
    for (p0, m0), (p1, m1), B in zip(runs[0], runs[1], bands):
        assert np.array_equal(p0, p1) and np.array_equal(m0, m1)
        lnfk = np.log(p0[:, 1])
        assert np.all(lnfk >= -9.2103403719761836 - 1e-12) and np.all(lnfk <= 2.3025850929940457 + 1e-12)
        assert np.all((p0[:, 2] >= -4.0) & (p0[:, 2] <= -0.25))
        assert np.array_equal(p0[:, 0], B["band"].psd[:, 0])      # sigma0 is held fixed
