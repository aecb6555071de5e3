"""tod_sample_ncorr_static draws the correlated noise without allocating:
its working memory is a fixed array compiled into the library, for callers
that cannot allocate device memory once they run (their free memory held by
another allocator's pool, or a no-allocation policy after start-up).  It is
checked here against tod_sample_ncorr on the same inputs, on two draws in a
row and a conditional-mean call, on a band that fits one wave of the array
and on one that takes several.  The file name puts it last in collection,
so it runs after every other GPU test as well as alone."""
import numpy as np
import pytest

import synth

SEED, BAND = 11, 3


def _workload(cfg):
    from gpu_workload import Workload
    return Workload(cfg)


@pytest.fixture(scope="module")
def small():
    return _workload(synth.scaled(synth.CONFIGS["lfi30"], nscan=3, len_lo=9000, len_hi=30000))


@pytest.fixture(scope="module")
def waves():
    # 70-GHz-shaped scans: 12 detectors x 4 scans of up to 300k samples,
    # more than one wave of the fixed array
    return _workload(synth.scaled(synth.CONFIGS["lfi70"], nscan=4))


@pytest.mark.gpu
def test_draw_before_setup_is_refused_and_takes_no_memory(small):
    """Before tod_ncorr_static_setup has run on the device, the draw returns
    an argument error and enqueues nothing (the lookup that backs the array
    is set-up's job)."""
    import torch
    import paper_2201_03509_gb300 as tg
    wl = small
    gains = torch.from_numpy(synth.gains(wl.cfg)[:wl.nq].astype(np.float64)).to(wl.dev)
    x = torch.full((wl.N,), 7.0, dtype=torch.float32, device=wl.dev)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info(wl.dev)[0]
    with pytest.raises(tg.TodError) as ei:
        wl.plan.sample_ncorr_static(wl.t_d, wl.t_s, gains, wl.t_flags, wl.t_psd, tg.Rng(SEED, BAND, 1),
                                    tg.MODE_DRAW, x)
    assert ei.value.code == -1
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info(wl.dev)[0] >= free0
    assert bool((x == 7.0).all())


def _compare(wl, nwaves_min):
    import torch
    import paper_2201_03509_gb300 as tg
    gains = torch.from_numpy(synth.gains(wl.cfg)[:wl.nq].astype(np.float64)).to(wl.dev)
    wave = wl.plan.ncorr_static_setup()
    assert wave >= 1_000_000
    assert -(-wl.N // wave) >= nwaves_min
    bufs = [(torch.empty(wl.N, dtype=torch.float32, device=wl.dev),
             torch.empty(wl.nq, dtype=torch.int32, device=wl.dev)) for _ in range(2)]
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info(wl.dev)[0]
    for it, mode in ((1, tg.MODE_DRAW), (2, tg.MODE_DRAW), (3, tg.MODE_MEAN)):
        outs = []
        for static in (False, True):
            x, its = bufs[int(static)]
            x.fill_(float("nan"))
            its.zero_()
            f = wl.plan.sample_ncorr_static if static else wl.plan.sample_ncorr
            f(wl.t_d, wl.t_s, gains, wl.t_flags, wl.t_psd, tg.Rng(SEED, BAND, it), mode, x, its,
              cg_tol=1e-7)
            wl.plan.status()
            outs.append((x.cpu().numpy().astype(np.float64), its.cpu().numpy()))
        (xa, ia), (xb, ib) = outs
        assert np.all(np.isfinite(xb))
        # each detscan's arithmetic does not depend on the launch it runs in:
        # within the n_corr parity tolerance (relative l2 1e-5), in fact equal
        for q in range(wl.nq):
            sl = wl.sl(q)
            err = np.linalg.norm(xb[sl] - xa[sl]) / np.linalg.norm(xa[sl])
            assert err <= 1e-5, (it, q, err)
        np.testing.assert_array_equal(ia, ib)
    torch.cuda.synchronize()
    # no device memory was taken by the static-scratch draws
    assert torch.cuda.mem_get_info(wl.dev)[0] >= free0


@pytest.mark.gpu
def test_static_scratch_matches_plan_scratch(small):
    _compare(small, 1)


@pytest.mark.gpu
def test_static_scratch_in_several_waves(waves):
    _compare(waves, 2)
