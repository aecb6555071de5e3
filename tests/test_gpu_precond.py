"""The n_corr CG under its three preconditioners (none, the gap blocks'
Toeplitz inverses, those plus the coarse correction) on a 70 GHz-like slice
(12 detscans of U[150k, 300k] samples, 2 % flagged in gaps of 10-500):
every level draws the oracle's n_corr (relative l2 1e-5 on sampled
detscans, CG tolerance 1e-7), and the iteration counts fall level by level.
Also: a step launches exactly the kernels it declares (launches_per_step,
counted by the library's kernel timing)."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

SEED, BAND, IT = 17, 2, 4


@pytest.fixture(scope="module")
def wl():
    pytest.importorskip("torch")
    from gpu_workload import Workload
    return Workload(synth.scaled(synth.CONFIGS["lfi70"], nscan=1))


def _draw(wl, levels, mode):
    import torch
    import paper_2201_03509_gb300 as tg
    gains = torch.from_numpy(np.asarray(wl.band.gain[:wl.nq], np.float64)).to(wl.dev)
    x = torch.zeros(wl.N, dtype=torch.float32, device=wl.dev)
    its = torch.zeros(wl.nq, dtype=torch.int32, device=wl.dev)
    wl.plan.set_preconditioner(levels)
    try:
        wl.plan.sample_ncorr(wl.t_d, wl.t_s, gains, wl.t_flags, wl.t_psd, tg.Rng(SEED, BAND, IT), mode, x, its,
                             cg_tol=1e-7)
        wl.plan.status()
    finally:
        wl.plan.set_preconditioner(tg.PREC_TWO_LEVEL)
    return x.cpu().numpy().astype(np.float64), its.cpu().numpy()


@pytest.mark.parametrize("mode", [0, 1])
def test_every_preconditioner_draws_the_oracle_ncorr(wl, mode):
    import paper_2201_03509_gb300 as tg
    runs = {lv: _draw(wl, lv, mode) for lv in (tg.PREC_NONE, tg.PREC_BLOCKS, tg.PREC_TWO_LEVEL)}
    flagged = [q for q in range(wl.nq) if wl.flags[wl.sl(q)].any()]
    assert len(flagged) == wl.nq
    lens = np.diff(wl.off)
    qs = sorted({0, int(np.argmax(lens)), int(np.argmin(lens)), wl.nq - 1})
    for q in qs:
        sl = wl.sl(q)
        n = sl.stop - sl.start
        s0, fk, al = wl.band.psd[wl.det(q)]
        if mode == 0:
            w1 = oracle.omega1(SEED, BAND, q, IT, n)
            w2 = oracle.omega2(SEED, BAND, q, IT, n)
        else:
            w1 = w2 = np.zeros(n)
        ref, _ = oracle.sample_ncorr(wl.d32[sl].astype(np.float64), wl.s32[sl].astype(np.float64),
                                     float(wl.band.gain[q]), wl.mask[sl], s0, fk, al, wl.cfg.fsamp, w1, w2)
        for lv, (x, its) in runs.items():
            err = np.linalg.norm(x[sl] - ref) / np.linalg.norm(ref)
            assert err < 1e-5, (lv, q, err, its[q])
    it_none, it_blk, it_two = (runs[lv][1] for lv in (tg.PREC_NONE, tg.PREC_BLOCKS, tg.PREC_TWO_LEVEL))
    assert np.all(it_two >= 1)
    assert it_two.mean() < it_blk.mean() < it_none.mean(), (it_none, it_blk, it_two)
    assert it_two.max() <= it_blk.max()


def test_unknown_preconditioner_level_is_refused(wl):
    import paper_2201_03509_gb300 as tg
    for bad in (-1, 3):
        with pytest.raises(tg.TodError):
            wl.plan.set_preconditioner(bad)


def test_step_launches_what_it_declares(wl):
    import torch
    import paper_2201_03509_gb300 as tg
    from paper_2201_03509_gb300.step import GibbsTODStep
    step = GibbsTODStep(wl.plan, wl.band.psd, wl.ing["flag_words"])
    step.lookahead = False
    step.set_tod(wl.d32)
    step.run(wl.t_map, tg.Rng(SEED, BAND, 0), tg.MODE_DRAW)
    torch.cuda.synchronize()
    wl.plan.set_kernel_timing(True)
    step.run(wl.t_map, tg.Rng(SEED, BAND, 1), tg.MODE_DRAW)
    torch.cuda.synchronize()
    wl.plan.set_kernel_timing(False)
    wl.plan.status()
    counts = {nm: n for nm, (_, n) in wl.plan.kernel_times().items()}
    assert sum(counts.values()) == step.launches_per_step, counts
    assert counts["k_nc_coarse"] == 1
    assert counts["k_toep_kernel"] == wl.plan.toeplitz_prep_launches - 1
