"""Row A12 on the GPU, through the C ABI: the joint gain draw of each
detector's scans under the smooth prior against the oracle's dense FP64
solve (mean and draw), its flat-prior limit, determinism, the largest scan
count, and misuse errors.

Tolerance: the transforms use an FP32 cosine table, so each DCT coefficient
carries an absolute error of about 1e-6 of the vector; the gain
fluctuations about the weighted mean are compared to 1e-5 relative (l2 per
detector), the weighted mean itself to ten times the bound that the CG
tolerance puts on it (tol |r| / sqrt(S) in units of the mean a)."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

SEED, BAND, IT = 13, 2, 6


@pytest.fixture(autouse=True)
def _needs_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")


def _plan(ndet, nscan):
    import paper_2201_03509_gb300 as tg
    cfg = synth.scaled(synth.CONFIGS["tiny"], nscan=nscan, len_lo=64, len_hi=64, ndet=ndet)
    band = synth.make_band(cfg, with_noise=False)
    ing = tg.ingest(band)
    return tg.Plan(cfg.nside, cfg.ndet, cfg.nscan, cfg.fsamp, ing["offsets"], ing["pix_streams"],
                   ing["psi_streams"])


def _inputs(ndet, nscan, seed=0):
    rng = np.random.default_rng(seed)
    drift = 0.01 * np.cumsum(rng.standard_normal((nscan, ndet)), axis=0) / np.sqrt(nscan)
    mu = 1.0 + drift + 1e-3 * rng.standard_normal((nscan, ndet))
    sigma = rng.uniform(0.8e-3, 1.5e-3, (nscan, ndet))
    return mu.reshape(-1), sigma.reshape(-1)             # detscan order q = scan * ndet + det


def _run(plan, mu, sigma, prior, mode, it=IT, tol=1e-7):
    import torch
    import paper_2201_03509_gb300 as tg
    dev = torch.device("cuda:0")
    t_mu = torch.from_numpy(mu).to(dev)
    t_sig = torch.from_numpy(sigma).to(dev)
    t_pr = torch.from_numpy(np.ascontiguousarray(prior, np.float64)).to(dev)
    g = torch.full_like(t_mu, float("nan"))
    its = torch.zeros(plan.ndet, dtype=torch.int32, device=dev)
    plan.sample_gain_smooth(t_mu, t_sig, t_pr, tg.Rng(SEED, BAND, it), mode, g, its, cg_tol=tol, cg_maxiter=500)
    plan.status()
    return g.cpu().numpy(), its.cpu().numpy()


def _oracle(mu, sigma, prior, ndet, mode, it=IT):
    S = len(mu) // ndet
    out = np.empty_like(mu)
    for d in range(ndet):
        w1, w2 = oracle.gain_smooth_normals(SEED, BAND, d, it, S)
        out[d::ndet] = oracle.sample_gain_smooth(mu[d::ndet], sigma[d::ndet], prior[d][0], prior[d][1], w1, w2,
                                                 mode)
    return out


def _check(g, ref, mu, sigma, ndet, prior, mode, it=IT, tol=1e-7):
    for d in range(ndet):
        a = 1.0 / sigma[d::ndet] ** 2
        S = len(a)
        gref = np.sum(a * mu[d::ndet]) / np.sum(a)
        fl = ref[d::ndet] - gref
        err = np.linalg.norm(g[d::ndet] - ref[d::ndet]) / np.linalg.norm(fl)
        assert err < 1e-5, (d, err)
        # the weighted mean of the gains is fixed by the right-hand side (the
        # prior does not see a constant): the sum of the final residual, at
        # most tol |r| sqrt(S), over sum a.  |r| of the system scaled by the
        # mean a, bounded by the triangle inequality (C is orthonormal).
        abar = a.mean()
        rn = np.linalg.norm(a * (mu[d::ndet] - gref))
        if mode == 0:
            w1, w2 = oracle.gain_smooth_normals(SEED, BAND, d, it, S)
            lam = oracle.gain_prior_precision(S, prior[d][0], prior[d][1])
            rn += np.linalg.norm(np.sqrt(a) * w1) + np.linalg.norm(np.sqrt(lam) * w2)
        bound = 10 * tol * (rn / abar) / np.sqrt(S)
        assert np.sum(a * g[d::ndet]) / np.sum(a) == pytest.approx(np.sum(a * ref[d::ndet]) / np.sum(a),
                                                                   abs=bound + 1e-12)


@pytest.mark.parametrize("ndet,nscan", [(4, 3), (1, 16), (2, 1000)])
@pytest.mark.parametrize("mode", [0, 1])
def test_matches_the_oracle(ndet, nscan, mode):
    plan = _plan(ndet, nscan)
    mu, sigma = _inputs(ndet, nscan, nscan)
    prior = [(1e-3 * (1 + 0.5 * d), -2.0 + 0.5 * d) for d in range(ndet)]
    g, its = _run(plan, mu, sigma, prior, mode)
    ref = _oracle(mu, sigma, prior, ndet, mode)
    _check(g, ref, mu, sigma, ndet, prior, mode)
    assert np.all(its >= 1) and np.all(its < 100)
    g2, _ = _run(plan, mu, sigma, prior, mode)
    assert np.array_equal(g, g2)                             # deterministic
    plan.close()


def test_flat_prior_limit_and_largest_scan_count():
    import paper_2201_03509_gb300 as tg
    S = 4096                                                 # TOD_GAIN_SMOOTH_MAX_SCANS
    plan = _plan(1, S)
    mu, sigma = _inputs(1, S, 5)
    g, _ = _run(plan, mu, sigma, [(1e9, -2.0)], 0)
    w1, _ = oracle.gain_smooth_normals(SEED, BAND, 0, IT, S)
    flat = mu + sigma * w1                                   # independent per-scan draws
    _check(g, flat, mu, sigma, 1, [(1e9, -2.0)], 0)
    # FP32 fluctuations of about 0.03 after CG to 1e-7: a few 1e-9 per scan
    np.testing.assert_allclose(g, flat, rtol=0, atol=3e-8)
    prior = [(2e-3, -1.5)]
    g, its = _run(plan, mu, sigma, prior, 0)
    _check(g, _oracle(mu, sigma, prior, 1, 0), mu, sigma, 1, prior, 0)
    plan.close()


def test_misuse():
    import torch
    import paper_2201_03509_gb300 as tg
    plan = _plan(2, 8)
    mu, sigma = _inputs(2, 8, 1)
    sigma[3] = 0.0
    with pytest.raises(tg.TodError):                         # marked on the device, raised by status
        _run(plan, mu, sigma, [(1e-3, -2.0)] * 2, 0)
    # a bad prior (sigma_g of zero, below the FP32 range, or NaN; alpha_g
    # infinite): every detscan of that detector is marked, the other detector runs
    mu, sigma = _inputs(2, 8, 1)
    dev = torch.device("cuda:0")
    t_mu, t_sig = torch.from_numpy(mu).to(dev), torch.from_numpy(sigma).to(dev)
    for bad in ((0.0, -2.0), (1e-30, -2.0), (float("nan"), -2.0), (1e-3, float("inf"))):
        t_pr = torch.tensor([bad, (1e-3, -2.0)], dtype=torch.float64, device=dev)
        g = torch.full_like(t_mu, float("nan"))
        plan.sample_gain_smooth(t_mu, t_sig, t_pr, tg.Rng(SEED, BAND, IT), 0, g)
        st = plan.status(raise_on_error=False)
        g = g.cpu().numpy()
        assert np.all(st[0::2] == -1) and np.all(st[1::2] == 0), bad
        assert np.all(g[0::2] == 0.0) and np.all(np.isfinite(g[1::2])), bad
    t = torch.zeros(16, dtype=torch.float64, device=dev)
    with pytest.raises(tg.TodError):                         # bad mode
        plan.sample_gain_smooth(t, t, t, tg.Rng(1, 0, 0), 7, t)
    plan.close()
    big = _plan(1, 4097)
    t = torch.ones(4097, dtype=torch.float64, device=dev)
    with pytest.raises(tg.TodError):                         # more scans than the kernel holds
        big.sample_gain_smooth(t, t, torch.ones(2, dtype=torch.float64, device=dev), tg.Rng(1, 0, 0), 0, t)
    big.close()


def test_step_with_the_smooth_prior():
    """A step with the prior: its gains are the joint draw from its own
    per-detscan conditionals, and the rest of the step uses them."""
    import torch
    import paper_2201_03509_gb300 as tg
    from paper_2201_03509_gb300.step import GibbsTODStep
    from gpu_workload import Workload
    wl = Workload(synth.CONFIGS["tiny"], tile_pairs=2)
    prior = np.array([[2e-3, -2.0]])
    st = GibbsTODStep(wl.plan, wl.band.psd, wl.ing["flag_words"], gain_prior=prior)
    st.set_tod(wl.d32)
    plain = GibbsTODStep(wl.plan, wl.band.psd, wl.ing["flag_words"])
    plain.set_tod(wl.d32)
    rng = tg.Rng(SEED, BAND, IT)
    st.run(wl.t_map, rng)
    torch.cuda.synchronize()
    wl.plan.status()
    g = torch.empty_like(st.gain)
    wl.plan.sample_gain_smooth(st.mu, st.sigma, st.gain_prior, rng, 0, g)
    wl.plan.status()
    assert torch.equal(g, st.gain)
    assert st.gain_iters.min().item() >= 1
    # the same step fed those gains through the plain path gives the same map
    plain.run(wl.t_map, rng)
    torch.cuda.synchronize()
    assert torch.equal(plain.mu, st.mu) and not torch.equal(plain.gain, st.gain)
    ncorr = torch.empty_like(st.ncorr)
    wl.plan.ncorr_prepare(st.psd)
    wl.plan.sample_ncorr_prepared(st.d, st.s, st.gain, st.flags, st.psd, rng, 0, ncorr, None, st.cg_tol,
                                  st.cg_maxiter)
    torch.cuda.synchronize()
    wl.plan.status()
    assert torch.equal(ncorr, st.ncorr)
    assert st.launches_per_step == plain.launches_per_step + 1
