"""Row A10 on the GPU, through the C ABI: the spectra that the n_corr draw
writes (against the DCT of the oracle's own draw), and the noise-PSD
Metropolis step (against the oracle's chain on the same spectra: the same
proposals, decisions, final state and log-likelihood)."""
import math

import numpy as np
import pytest

import oracle
import synth

SEED, BAND, IT = 21, 1, 4


@pytest.fixture(scope="module")
def wl():
    from gpu_workload import Workload
    cfg = synth.scaled(synth.CONFIGS["lfi30"], nscan=3, len_lo=9000, len_hi=30000)
    assert cfg.flag_frac > 0
    return Workload(cfg, tile_pairs=0)


@pytest.mark.gpu
def test_ncorr_spectrum_matches_the_oracle_draw(wl):
    import torch
    import paper_2201_03509_gb300 as tg
    gains = synth.gains(wl.cfg)[:wl.nq].astype(np.float64)
    t_g = torch.from_numpy(gains).to(wl.dev)
    x = torch.zeros(wl.N, dtype=torch.float32, device=wl.dev)
    spec = torch.full((wl.N,), float("nan"), dtype=torch.float32, device=wl.dev)
    its = torch.zeros(wl.nq, dtype=torch.int32, device=wl.dev)
    wl.plan.set_ncorr_spectrum(spec)
    try:
        wl.plan.sample_ncorr(wl.t_d, wl.t_s, t_g, wl.t_flags, wl.t_psd, tg.Rng(SEED, BAND, IT), tg.MODE_DRAW, x,
                             its, cg_tol=1e-7)
        wl.plan.status()
    finally:
        wl.plan.set_ncorr_spectrum(None)
    spec = spec.cpu().numpy().astype(np.float64)
    its = its.cpu().numpy()
    assert np.all(np.isfinite(spec))                       # every mode written
    assert its.max() > 0                                   # flagged detscans went through the CG
    for q in range(wl.nq):
        sl = wl.sl(q)
        n = sl.stop - sl.start
        s0, fk, al = wl.band.psd[wl.det(q)]
        w1 = oracle.omega1(SEED, BAND, q, IT, n)
        w2 = oracle.omega2(SEED, BAND, q, IT, n)
        ref, _ = oracle.sample_ncorr(wl.d32[sl].astype(np.float64), wl.s32[sl].astype(np.float64), gains[q],
                                     wl.mask[sl], s0, fk, al, wl.cfg.fsamp, w1, w2)
        rh = oracle.dct(ref)
        err = np.linalg.norm(spec[sl] - rh) / np.linalg.norm(rh)
        assert err < 1e-5, (q, err)


def _spectra(wl, truth_by_det, seed):
    """Random spectra xhat_k ~ N(0, Pc_k) per detscan (FP32), built here."""
    rng = np.random.default_rng(seed)
    out = np.zeros(wl.N, dtype=np.float32)
    for q in range(wl.nq):
        sl = wl.sl(q)
        n = sl.stop - sl.start
        s0, fk, al = truth_by_det[wl.det(q)]
        k = np.arange(1, n, dtype=np.float64)
        pc = s0 ** 2 * (k * wl.cfg.fsamp / (2.0 * n) / fk) ** al
        xs = np.zeros(n)
        xs[1:] = np.sqrt(pc) * rng.standard_normal(n - 1)
        out[sl] = xs.astype(np.float32)
    return out


@pytest.mark.gpu
@pytest.mark.parametrize("nsteps", [0, 30])
def test_noise_psd_chain_matches_the_oracle(wl, nsteps):
    import torch
    import paper_2201_03509_gb300 as tg
    ndet = wl.cfg.ndet
    truth = np.array([[1.1e-3, 0.08, -1.5], [0.9e-3, 0.15, -1.1], [1.0e-3, 0.05, -2.0], [1.2e-3, 0.1, -1.3]])[:ndet]
    start = truth.copy()
    start[:, 1] *= 1.6                                      # start away from the truth
    start[:, 2] += 0.2
    sp = _spectra(wl, truth, 5)
    t_sp = torch.from_numpy(sp).to(wl.dev)
    psd_in = torch.from_numpy(start).to(wl.dev)
    psd_out = torch.zeros_like(psd_in)
    acc = torch.zeros(ndet, dtype=torch.int32, device=wl.dev)
    ll = torch.zeros(ndet, dtype=torch.float64, device=wl.dev)
    st_lnfk, st_al = 0.05, 0.01
    wl.plan.sample_noise_psd(t_sp, psd_in, tg.Rng(SEED, BAND, IT), nsteps, st_lnfk, st_al, psd_out, acc, ll)
    wl.plan.status()
    g_psd, g_acc, g_ll = psd_out.cpu().numpy(), acc.cpu().numpy(), ll.cpu().numpy()
    spectra = [[sp[wl.sl(q)].astype(np.float64) for q in range(wl.nq) if wl.det(q) == d] for d in range(ndet)]
    lengths = [[wl.sl(q).stop - wl.sl(q).start for q in range(wl.nq) if wl.det(q) == d] for d in range(ndet)]
    r_psd, r_acc = oracle.sample_noise_psd(spectra, lengths, wl.cfg.fsamp, start, SEED, BAND, IT, nsteps,
                                           st_lnfk, st_al)
    np.testing.assert_array_equal(g_acc, r_acc)
    np.testing.assert_allclose(g_psd, r_psd, rtol=1e-9)
    if nsteps:
        assert r_acc.sum() > 0
    for d in range(ndet):
        want = oracle.psd_loglike(spectra[d], lengths[d], wl.cfg.fsamp, *r_psd[d])
        assert g_ll[d] == pytest.approx(want, rel=1e-9, abs=1e-6 * math.sqrt(sum(lengths[d])))
