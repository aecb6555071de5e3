"""Parity at the full 70 GHz-like workload (12 detectors x 2000 scans of
U[150k, 300k] samples at 78.8 Hz, Nside 1024: 5.4e9 samples), in the launch
configuration the benchmark times: the band generated straight into
concatenated arrays, the plan's own tile shape, the persistent schedule,
one Gibbs step through GibbsTODStep at the benchmark's CG tolerance.

The oracle cannot redo the band in a test, so:
  * decode, projection, gain and n_corr are checked on sampled detscans
    (the longest, the shortest, the most flagged, the first, the last and a
    fixed one), each against the oracle run on that detscan alone;
  * hits are checked for every pixel against a bincount of the synthetic
    pointing;
  * binning (with gains and an n_corr timeline chosen by the test) and the
    3x3 solve are checked on sampled pixels against the oracle's normal
    equations, built from exactly the samples that hit those pixels.
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

SEED, BAND, IT = 5, 2, 3
CG_TOL = 1e-6          # the benchmark's setting


@pytest.fixture(scope="module")
def band70():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2201_03509_gb300 as tg
    from paper_2201_03509_gb300.step import GibbsTODStep
    cfg = synth.CONFIGS["lfi70"]
    arr = synth.make_band_arrays(cfg, tg.kept_lengths(cfg))
    ing = tg.ingest_arrays(arr)
    off = ing["offsets"]
    plan = tg.Plan(cfg.nside, cfg.ndet, cfg.nscan, cfg.fsamp, off, ing["pix_streams"], ing["psi_streams"])
    step = GibbsTODStep(plan, arr.psd, ing["flag_words"], cg_tol=CG_TOL)
    step.set_tod(arr.tod)
    m4 = np.zeros((arr.npix, 4), np.float32)
    m4[:, :3] = arr.map_tqu.T
    step.run(torch.from_numpy(m4).cuda(), tg.Rng(SEED, BAND, IT), tg.MODE_DRAW)
    torch.cuda.synchronize()
    plan.status()
    nq = len(off) - 1
    lens = np.diff(off)
    nflag = np.add.reduceat(arr.flags, off[:-1]).astype(np.float64)
    qs = sorted({int(np.argmax(lens)), int(np.argmin(lens)), int(np.argmax(nflag / lens)), 0, 12345 % nq, nq - 1})
    return dict(cfg=cfg, arr=arr, off=off, plan=plan, step=step, map32=m4[:, :3].T.astype(np.float64), qs=qs,
                torch=torch)


def _sl(F, q):
    return slice(int(F["off"][q]), int(F["off"][q + 1]))


def test_fullsize70_decode_project_gain_ncorr_sampled(band70):
    F = band70
    cfg, arr, step = F["cfg"], F["arr"], F["step"]
    g_gpu = step.gain.cpu().numpy()
    for q in F["qs"]:
        sl = _sl(F, q)
        n = sl.stop - sl.start
        pix = step.pix[sl].cpu().numpy()
        psi = step.psi[sl].cpu().numpy().view(np.uint16)
        assert np.array_equal(pix, arr.pix[sl]), q
        assert np.array_equal(psi, arr.psi[sl]), q
        det = q % cfg.ndet
        s0, fk, al = arr.psd[det]
        d = arr.tod[sl].astype(np.float64)
        mask = (~arr.flags[sl]).astype(np.float64)
        s = oracle.project(F["map32"], arr.pix[sl].astype(np.int64), arr.psi[sl].astype(np.int64))
        # the step's projection (unit gain, FP32 output)
        s_gpu = step.s[sl].cpu().numpy().astype(np.float64)
        assert np.abs(s_gpu - s).max() <= 1e-6 * np.abs(s).max(), q
        P = oracle.noise_psd(n, cfg.fsamp, s0, fk, al)
        rg, _, rsg = oracle.sample_gain(s, d, mask, P, oracle.gain_normal(SEED, BAND, q, IT), oracle.MODE_DRAW)
        assert g_gpu[q] == pytest.approx(rg, rel=1e-5, abs=1e-5 * rsg), q
        w1 = oracle.omega1(SEED, BAND, q, IT, n)
        w2 = oracle.omega2(SEED, BAND, q, IT, n)
        ref, _ = oracle.sample_ncorr(d, s, rg, mask, s0, fk, al, cfg.fsamp, w1, w2)
        x = step.ncorr[sl].cpu().numpy().astype(np.float64)
        err = np.linalg.norm(x - ref) / np.linalg.norm(ref)
        assert err < 1e-5, (q, err)


def test_fullsize70_hits_bin_and_solve_sampled(band70):
    F = band70
    torch, cfg, arr, step = F["torch"], F["cfg"], F["arr"], F["step"]
    off, npix = F["off"], arr.npix
    keep = ~arr.flags
    rh = np.bincount(arr.pix, weights=keep, minlength=npix).astype(np.int64)
    assert np.array_equal(step.hits.cpu().numpy(), rh)
    # binning with test-chosen gains and n_corr (written over the step's s),
    # on sampled pixels
    N = int(off[-1])
    gains = arr.gain.copy()
    x32 = (1e-4 * np.random.default_rng(3).standard_normal(N)).astype(np.float32)
    t_x = step.s
    t_x.copy_(torch.from_numpy(x32))
    dev = t_x.device
    A = torch.zeros((npix, 6), dtype=torch.float64, device=dev)
    b = torch.zeros((npix, 3), dtype=torch.float64, device=dev)
    hits = torch.zeros(npix, dtype=torch.int32, device=dev)
    F["plan"].bin(step.psi, step.d, t_x, torch.from_numpy(gains).to(dev), step.flags, step.psd, A, b, hits)
    F["plan"].status()
    assert np.array_equal(hits.cpu().numpy(), rh)
    hit_pix = np.nonzero(rh >= 3)[0]
    sp = np.sort(np.random.default_rng(4).choice(hit_pix, min(2000, hit_pix.size), replace=False))
    lut = np.zeros(npix, bool)
    lut[sp] = True
    sel = np.nonzero(lut[arr.pix])[0]
    qsel = np.searchsorted(off, sel, side="right") - 1
    gs = gains[qsel]
    s0 = arr.psd[qsel % cfg.ndet, 0]
    msel = keep[sel].astype(np.float64)
    resid = arr.tod[sel].astype(np.float64) - x32[sel].astype(np.float64)
    rA, rb = oracle.bin_maps(npix, arr.pix[sel].astype(np.int64), arr.psi[sel].astype(np.int64), resid,
                             (msel * gs ** 2 / s0 ** 2, msel * gs / s0 ** 2))
    gA, gb = A.cpu().numpy()[sp], b.cpu().numpy()[sp]
    for i in range(6):
        assert np.abs(gA[:, i] - rA[sp, i]).max() <= 1e-10 * np.abs(rA[sp, i]).max()
    for i in range(3):
        assert np.abs(gb[:, i] - rb[sp, i]).max() <= 1e-10 * np.abs(rb[sp, i]).max()
    # the solve at full size, on the oracle's normal equations of the sampled pixels
    rA_full = np.zeros((npix, 6))
    rb_full = np.zeros((npix, 3))
    rh_full = np.zeros(npix, np.int64)
    rA_full[sp], rb_full[sp], rh_full[sp] = rA[sp], rb[sp], rh[sp]
    m = torch.zeros((3, npix), dtype=torch.float64, device=dev)
    m32 = torch.zeros((npix, 4), dtype=torch.float32, device=dev)
    rc = torch.zeros(npix, dtype=torch.float64, device=dev)
    va = torch.zeros(npix, dtype=torch.uint8, device=dev)
    F["plan"].solve_maps(torch.from_numpy(rA_full).to(dev), torch.from_numpy(rb_full).to(dev),
                         torch.from_numpy(rh_full.astype(np.int32)).to(dev), 1e-6, m, m32, rc, va)
    rm, _, rvalid = oracle.solve_maps(rA_full[sp], rb_full[sp], rh_full[sp], 1e-6)
    gv = va.cpu().numpy()
    assert np.array_equal(gv[sp], rvalid)
    assert gv.sum() == rvalid.sum()          # nothing outside the sample is valid
    assert rvalid.sum() > 1000               # the full band solves most sampled pixels
    gm = m.cpu().numpy()[:, sp]
    ok = rvalid > 0
    for i in range(3):
        assert np.abs(gm[i, ok] - rm[i, ok]).max() <= 1e-10 * np.abs(rm[i, ok]).max()
