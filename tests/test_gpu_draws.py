"""Distribution of the GPU draws and CUDA-graph replay.

* gain: over many Gibbs iterations, (g - mu) / sigma is N(0, 1)
  (Kolmogorov-Smirnov);
* n_corr on gap-free detscans: the draw minus the conditional mean, taken to
  the DCT basis and scaled by sqrt(phi_k + 1/sigma0^2), is N(0, 1) in every
  mode (the conditional covariance is C^T diag(1/(phi + 1/sigma0^2)) C);
* a step captured as a CUDA graph and replayed at Gibbs iteration k gives
  bit for bit what the eager step gives at k (with the pointing lookahead:
  two graphs swapping the pointing buffers, replayed in turn);
* steps whose detector data is prefetched into a second buffer on a copy
  stream give bit for bit the steps of plain copies;
* the n_corr draw split in preparation (on a side stream) and prepared draw
  gives bit for bit the one-call draw;
* steps that decode the next step's pointing ahead give bit for bit the
  steps that decode their own.
"""
import numpy as np
import pytest

import oracle
import synth


@pytest.fixture(scope="module")
def tiny():
    from gpu_workload import Workload
    cfg = synth.CONFIGS["tiny"]
    assert cfg.flag_frac == 0.0
    return Workload(cfg, tile_pairs=0)


@pytest.mark.gpu
def test_gain_draws_are_standard_normal(tiny):
    import torch
    from scipy import stats
    import paper_2201_03509_gb300 as tg
    wl = tiny
    g = torch.zeros(wl.nq, dtype=torch.float64, device=wl.dev)
    mu = torch.zeros_like(g)
    sg = torch.zeros_like(g)
    zs = []
    for it in range(300):
        wl.plan.sample_gain(wl.t_d, wl.t_s, wl.t_flags, wl.t_psd, tg.Rng(7, 1, it), tg.MODE_DRAW, g, mu, sg)
        zs.append(((g - mu) / sg).cpu().numpy())
    wl.plan.status()
    z = np.concatenate(zs)
    assert z.size == 300 * wl.nq
    assert stats.kstest(z, "norm").pvalue > 1e-3
    assert abs(z.mean()) < 4.0 / np.sqrt(z.size)


@pytest.mark.gpu
def test_ncorr_draws_have_the_conditional_covariance(tiny):
    import torch
    from scipy import fft, stats
    import paper_2201_03509_gb300 as tg
    wl = tiny
    gains = torch.from_numpy(wl.band.gain.copy()).to(wl.dev)
    xm = torch.zeros(wl.N, dtype=torch.float32, device=wl.dev)
    x = torch.zeros_like(xm)
    wl.plan.sample_ncorr(wl.t_d, wl.t_s, gains, wl.t_flags, wl.t_psd, tg.Rng(9, 2, 0), tg.MODE_MEAN, xm)
    mean = xm.cpu().numpy().astype(np.float64)
    ws = []
    for it in range(4):
        wl.plan.sample_ncorr(wl.t_d, wl.t_s, gains, wl.t_flags, wl.t_psd, tg.Rng(9, 2, it), tg.MODE_DRAW, x)
        dx = x.cpu().numpy().astype(np.float64) - mean
        for q in range(wl.nq):
            sl = wl.sl(q)
            n = sl.stop - sl.start
            s0, fk, al = wl.band.psd[wl.det(q)]
            phi = oracle.corr_inv_psd(n, wl.cfg.fsamp, s0, fk, al)
            ws.append(fft.dct(dx[sl], type=2, norm="ortho") * np.sqrt(phi + 1.0 / s0 ** 2))
    wl.plan.status()
    w = np.concatenate(ws)
    assert stats.kstest(w, "norm").pvalue > 1e-3
    assert abs(w.std() - 1.0) < 0.02


@pytest.mark.gpu
def test_graph_replay_matches_eager_step(tiny):
    import torch
    import paper_2201_03509_gb300 as tg
    from paper_2201_03509_gb300.step import GibbsTODStep
    wl = tiny
    step = GibbsTODStep(wl.plan, wl.band.psd, wl.ing["flag_words"])
    step.set_tod(wl.d32)
    step.run(wl.t_map, tg.Rng(3, 0, 5), tg.MODE_DRAW)
    torch.cuda.synchronize()
    ref = [t.clone() for t in (step.gain, step.ncorr, step.A, step.b, step.map)]
    step.capture(wl.t_map, 3, 0, tg.MODE_DRAW)
    step.replay(5)
    torch.cuda.synchronize()
    got = (step.gain, step.ncorr, step.A, step.b, step.map)
    for a, b in zip(ref, got):
        assert torch.equal(a, b)
    step.replay(6)
    torch.cuda.synchronize()
    assert not torch.equal(ref[0], step.gain)      # a fresh iteration draws fresh numbers
    wl.plan.status()


@pytest.mark.gpu
def test_graph_replays_with_lookahead_match_eager_steps(tiny):
    """With the pointing lookahead the step is captured as two graphs that
    swap the pointing buffers; replays alternate between them and give bit
    for bit the eager steps (which also decode ahead)."""
    import torch
    import paper_2201_03509_gb300 as tg
    from paper_2201_03509_gb300.step import GibbsTODStep
    wl = tiny
    eager = GibbsTODStep(wl.plan, wl.band.psd, wl.ing["flag_words"])
    eager.set_tod(wl.d32)
    assert eager.lookahead
    ref = []
    for it in (5, 6, 7, 8):
        eager.run(wl.t_map, tg.Rng(3, 0, it), tg.MODE_DRAW)
        torch.cuda.synchronize()
        ref.append([t.clone() for t in (eager.gain, eager.ncorr, eager.A, eager.map)])
    step = GibbsTODStep(wl.plan, wl.band.psd, wl.ing["flag_words"])
    step.set_tod(wl.d32)
    step.capture(wl.t_map, 3, 0, tg.MODE_DRAW)
    assert len(step.graphs) == 2
    for k, it in enumerate((5, 6, 7, 8)):
        step.replay(it)
        torch.cuda.synchronize()
        for a, b in zip(ref[k], (step.gain, step.ncorr, step.A, step.map)):
            assert torch.equal(a, b), it
    wl.plan.status()


@pytest.mark.gpu
def test_prefetched_tod_matches_set_tod(tiny):
    """Double-buffered detector data (copy of step k+1 on a second stream while
    step k runs) gives bit for bit the steps of plain set_tod copies."""
    import torch
    import paper_2201_03509_gb300 as tg
    from paper_2201_03509_gb300.step import GibbsTODStep
    wl = tiny
    ds = [wl.d32, (wl.d32 * np.float32(1.25)).astype(np.float32), (wl.d32 - np.float32(0.5)).astype(np.float32)]
    ref_step = GibbsTODStep(wl.plan, wl.band.psd, wl.ing["flag_words"])
    refs = []
    for k, d in enumerate(ds):
        ref_step.set_tod(d)
        ref_step.run(wl.t_map, tg.Rng(4, 0, k), tg.MODE_DRAW)
        torch.cuda.synchronize()
        refs.append([t.clone() for t in (ref_step.gain, ref_step.ncorr, ref_step.map)])
    step = GibbsTODStep(wl.plan, wl.band.psd, wl.ing["flag_words"])
    hosts = [torch.from_numpy(d).pin_memory() for d in ds]
    step.prefetch_tod(hosts[0])
    for k in range(len(ds)):
        step.run(wl.t_map, tg.Rng(4, 0, k), tg.MODE_DRAW)
        if k + 1 < len(ds):
            step.prefetch_tod(hosts[k + 1])
        torch.cuda.synchronize()
        for a, b in zip(refs[k], (step.gain, step.ncorr, step.map)):
            assert torch.equal(a, b), k
    wl.plan.status()


@pytest.mark.gpu
def test_prepared_ncorr_matches_sample_ncorr():
    """tod_ncorr_prepare on a side stream + tod_sample_ncorr_prepared gives
    bit for bit what tod_sample_ncorr gives (flagged detscans, so the gap
    preconditioner is used)."""
    import torch
    import paper_2201_03509_gb300 as tg
    from gpu_workload import Workload
    cfg = synth.scaled(synth.CONFIGS["lfi30"], nscan=2, len_lo=9000, len_hi=30000)
    assert cfg.flag_frac > 0
    wl = Workload(cfg, tile_pairs=0)
    gains = torch.from_numpy(synth.gains(cfg)[:wl.nq].astype(np.float64)).to(wl.dev)
    outs = []
    for prepared in (False, True):
        x = torch.full((wl.N,), float("nan"), dtype=torch.float32, device=wl.dev)
        its = torch.zeros(wl.nq, dtype=torch.int32, device=wl.dev)
        if prepared:
            side = torch.cuda.Stream(device=wl.dev)
            side.wait_stream(torch.cuda.current_stream())
            wl.plan.ncorr_prepare(wl.t_psd, side)
            ev = torch.cuda.Event()
            ev.record(side)
            torch.cuda.current_stream().wait_event(ev)
            wl.plan.sample_ncorr_prepared(wl.t_d, wl.t_s, gains, wl.t_flags, wl.t_psd, tg.Rng(5, 1, 2),
                                          tg.MODE_DRAW, x, its, cg_tol=1e-7)
        else:
            wl.plan.sample_ncorr(wl.t_d, wl.t_s, gains, wl.t_flags, wl.t_psd, tg.Rng(5, 1, 2), tg.MODE_DRAW, x,
                                 its, cg_tol=1e-7)
        torch.cuda.synchronize()
        wl.plan.status()
        outs.append((x.cpu().numpy(), its.cpu().numpy()))
    assert outs[0][1].max() > 0                  # the CG (and its preconditioner) ran
    assert np.array_equal(outs[0][0], outs[1][0])
    assert np.array_equal(outs[0][1], outs[1][1])


@pytest.mark.gpu
def test_pointing_lookahead_matches_in_step_decode(tiny):
    """Steps that decode the next step's pointing under their n_corr draw
    (GibbsTODStep.lookahead) give bit for bit the steps that decode in step."""
    import torch
    import paper_2201_03509_gb300 as tg
    from paper_2201_03509_gb300.step import GibbsTODStep
    wl = tiny
    outs = []
    for lookahead in (False, True):
        step = GibbsTODStep(wl.plan, wl.band.psd, wl.ing["flag_words"])
        step.lookahead = lookahead
        step.set_tod(wl.d32)
        got = []
        for k in range(3):
            step.run(wl.t_map, tg.Rng(6, 0, k), tg.MODE_DRAW)
            torch.cuda.synchronize()
            got.append([t.clone() for t in (step.pix, step.psi, step.gain, step.ncorr, step.map)])
        outs.append(got)
    for k in range(3):
        for a, b in zip(outs[0][k], outs[1][k]):
            assert torch.equal(a, b), k
    wl.plan.status()
