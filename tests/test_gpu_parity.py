"""GPU path vs the FP64 oracle, stage by stage, through the C ABI.

Tolerances (derived from the FP32 arithmetic): integer work bit-exact; FP32 timelines
1e-5 relative (l2 per detscan); FP64-accumulated maps 1e-10 relative."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

SEED, BAND, IT = 777, 3, 5


def _cfgs():
    """(band, column pairs per tile (0: the plan's choice), largest radix,
    per-scan schedule): several tiles per detscan and ragged last tiles."""
    tiny = synth.CONFIGS["tiny"]
    # a few LFI-30-like detscans, short enough for the oracle, with flags
    l30 = synth.scaled(synth.CONFIGS["lfi30"], nscan=3, len_lo=9000, len_hi=30000)
    return {"tiny_t1": (tiny, 1), "tiny_t4": (tiny, 4), "tiny_t3": (tiny, 3), "lfi30_small_t2": (l30, 2),
            "lfi30_small_t5": (l30, 5), "lfi30_small_t9": (l30, 9), "lfi30_small_auto": (l30, 0),
            "lfi30_small_t9_r8": (l30, 9, 8), "tiny_t2_r4": (tiny, 2, 4),
            "lfi30_small_perscan": (l30, 0, 0, True), "tiny_perscan_t3": (tiny, 3, 0, True)}


@pytest.fixture(scope="module", params=list(_cfgs().keys()))
def wl(request):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from gpu_workload import Workload
    cfg, tp, *rest = _cfgs()[request.param]
    rmax = rest[0] if rest else 0
    w = Workload(cfg, tile_pairs=tp, max_radix=rmax)
    if len(rest) > 1 and rest[1]:
        w.plan.set_schedule(w.plan.SCHED_PER_SCAN)
    return w


def test_plan_info(wl):
    info = wl.plan.info()
    assert info["nsamples"] == wl.N and info["ndetscan"] == wl.nq


def test_decode_bit_exact(wl):
    import torch
    pix = torch.empty(wl.N, dtype=torch.int32, device=wl.dev)
    psi = torch.empty(wl.N, dtype=torch.int16, device=wl.dev)
    wl.plan.decode(pix, psi)
    wl.plan.status()
    assert np.array_equal(pix.cpu().numpy().astype(np.int64), wl.pix_ref)
    assert np.array_equal(psi.cpu().numpy().view(np.uint16).astype(np.int64), wl.psi_ref)
    # and the oracle's own decoder agrees on the same streams
    q = wl.nq - 1
    n = int(wl.off[q + 1] - wl.off[q])
    assert np.array_equal(oracle.decode_detscan(wl.ing["pix_streams"], q, n, wl.cfg.ndet),
                          wl.pix_ref[wl.sl(q)])


def test_project(wl):
    import torch
    pix = torch.from_numpy(wl.pix_ref.astype(np.int32)).to(wl.dev)
    psi = torch.from_numpy(wl.psi_ref.astype(np.uint16).view(np.int16)).to(wl.dev)
    gain = torch.from_numpy(wl.band.gain.copy()).to(wl.dev)
    s = torch.empty(wl.N, dtype=torch.float32, device=wl.dev)
    wl.plan.project(wl.t_map, pix, psi, gain, s)
    wl.plan.status()
    ref = oracle.project(wl.band.map_tqu, wl.pix_ref, wl.psi_ref,
                         oracle.per_sample(wl.band.gain, wl.off))
    got = s.cpu().numpy().astype(np.float64)
    assert np.abs(got - ref).max() <= 1e-5 * np.abs(ref).max()


def _oracle_gain(wl, q, mode):
    det = wl.det(q)
    sl = wl.sl(q)
    n = sl.stop - sl.start
    s0, fk, al = wl.band.psd[det]
    P = oracle.noise_psd(n, wl.cfg.fsamp, s0, fk, al)
    z = oracle.gain_normal(SEED, BAND, q, IT)
    return oracle.sample_gain(wl.s32[sl].astype(np.float64), wl.d32[sl].astype(np.float64),
                              wl.mask[sl], P, z, mode)


@pytest.mark.parametrize("mode", [0, 1])
def test_sample_gain(wl, mode):
    import torch
    import paper_2201_03509_gb300 as tg
    g = torch.zeros(wl.nq, dtype=torch.float64, device=wl.dev)
    mu = torch.zeros_like(g)
    sg = torch.zeros_like(g)
    wl.plan.sample_gain(wl.t_d, wl.t_s, wl.t_flags, wl.t_psd, tg.Rng(SEED, BAND, IT), mode, g, mu, sg)
    wl.plan.status()
    g, mu, sg = g.cpu().numpy(), mu.cpu().numpy(), sg.cpu().numpy()
    for q in range(wl.nq):
        rg, rmu, rsg = _oracle_gain(wl, q, mode)
        assert mu[q] == pytest.approx(rmu, rel=1e-5, abs=1e-5 * rsg)
        assert sg[q] == pytest.approx(rsg, rel=1e-5)
        assert g[q] == pytest.approx(rg, rel=1e-5, abs=1e-5 * rsg)


@pytest.mark.parametrize("mode", [0, 1])
def test_sample_ncorr(wl, mode):
    import torch
    import paper_2201_03509_gb300 as tg
    gains = np.array([_oracle_gain(wl, q, 1)[1] for q in range(wl.nq)])
    t_g = torch.from_numpy(gains).to(wl.dev)
    x = torch.zeros(wl.N, dtype=torch.float32, device=wl.dev)
    its = torch.zeros(wl.nq, dtype=torch.int32, device=wl.dev)
    wl.plan.sample_ncorr(wl.t_d, wl.t_s, t_g, wl.t_flags, wl.t_psd, tg.Rng(SEED, BAND, IT), mode, x, its,
                         cg_tol=1e-7)
    wl.plan.status()
    x = x.cpu().numpy().astype(np.float64)
    its = its.cpu().numpy()
    for q in range(wl.nq):
        sl = wl.sl(q)
        n = sl.stop - sl.start
        s0, fk, al = wl.band.psd[wl.det(q)]
        if mode == 0:
            w1 = oracle.omega1(SEED, BAND, q, IT, n)
            w2 = oracle.omega2(SEED, BAND, q, IT, n)
        else:
            w1 = w2 = np.zeros(n)
        ref, rit = oracle.sample_ncorr(wl.d32[sl].astype(np.float64), wl.s32[sl].astype(np.float64),
                                       gains[q], wl.mask[sl], s0, fk, al, wl.cfg.fsamp, w1, w2)
        err = np.linalg.norm(x[sl] - ref) / np.linalg.norm(ref)
        assert err < 1e-5, (q, err, its[q], rit)
        assert (its[q] > 0) == (rit > 0)


def test_bin_and_solve(wl):
    import torch
    gains = wl.band.gain.copy()
    rng = np.random.default_rng(1)
    x32 = (1e-4 * rng.standard_normal(wl.N)).astype(np.float32)     # any FP32 n_corr
    t_x = torch.from_numpy(x32).to(wl.dev)
    psi = torch.from_numpy(wl.psi_ref.astype(np.uint16).view(np.int16)).to(wl.dev)
    t_g = torch.from_numpy(gains).to(wl.dev)
    npix = wl.band.npix
    A = torch.zeros((npix, 6), dtype=torch.float64, device=wl.dev)
    b = torch.zeros((npix, 3), dtype=torch.float64, device=wl.dev)
    hits = torch.zeros(npix, dtype=torch.int32, device=wl.dev)
    wl.plan.bin(psi, wl.t_d, t_x, t_g, wl.t_flags, wl.t_psd, A, b, hits)
    wl.plan.status()
    gs = oracle.per_sample(gains, wl.off)
    s0 = oracle.per_sample(np.tile(wl.band.psd[:, 0], wl.cfg.nscan), wl.off)
    w = wl.mask * gs ** 2 / s0 ** 2
    v = wl.mask * gs / s0 ** 2
    rA, rb = oracle.bin_maps(npix, wl.pix_ref, wl.psi_ref,
                             wl.d32.astype(np.float64) - x32.astype(np.float64), (w, v))
    rh = np.bincount(wl.pix_ref, weights=wl.mask, minlength=npix).astype(np.int64)
    gA, gb, gh = A.cpu().numpy(), b.cpu().numpy(), hits.cpu().numpy()
    assert np.array_equal(gh, rh)
    for i in range(6):
        assert np.abs(gA[:, i] - rA[:, i]).max() <= 1e-10 * np.abs(rA[:, i]).max()
    for i in range(3):
        assert np.abs(gb[:, i] - rb[:, i]).max() <= 1e-10 * np.abs(rb[:, i]).max()
    # solve on the oracle's normal equations
    m = torch.zeros((3, npix), dtype=torch.float64, device=wl.dev)
    m32 = torch.zeros((npix, 4), dtype=torch.float32, device=wl.dev)
    rc = torch.zeros(npix, dtype=torch.float64, device=wl.dev)
    va = torch.zeros(npix, dtype=torch.uint8, device=wl.dev)
    tA = torch.from_numpy(rA).to(wl.dev)
    tb = torch.from_numpy(rb).to(wl.dev)
    th = torch.from_numpy(rh.astype(np.int32)).to(wl.dev)
    wl.plan.solve_maps(tA, tb, th, 1e-6, m, m32, rc, va)
    rm, rhad, rvalid = oracle.solve_maps(rA, rb, rh, 1e-6)
    gm, gv = m.cpu().numpy(), va.cpu().numpy()
    assert np.array_equal(gv, rvalid)
    ok = rvalid > 0
    for i in range(3):
        assert np.abs(gm[i, ok] - rm[i, ok]).max() <= 1e-10 * np.abs(rm[i, ok]).max()
    assert np.allclose(rc.cpu().numpy(), rhad, rtol=1e-10, atol=1e-14)
