"""tod_sample_ncorr_static (fixed device scratch, allocates nothing) against
tod_sample_ncorr on the same inputs, on two calls in a row.  The file name
puts it last in collection, so it runs after every other GPU test as well as
alone."""
import numpy as np
import pytest

import synth

SEED, BAND = 11, 3


@pytest.fixture(scope="module")
def wl():
    from gpu_workload import Workload
    cfg = synth.scaled(synth.CONFIGS["lfi30"], nscan=3, len_lo=9000, len_hi=30000)
    return Workload(cfg, cluster_size=8)


@pytest.mark.gpu
def test_static_scratch_matches_plan_scratch(wl):
    import torch
    import paper_2201_03509_gb300 as tg
    gains = torch.from_numpy(synth.gains(wl.cfg)[:wl.nq].astype(np.float64)).to(wl.dev)
    nfit = wl.plan.ncorr_static_setup()
    assert nfit >= 1
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
        # same arithmetic per detscan whichever cluster runs it: within the
        # n_corr parity tolerance (relative l2 1e-5 per detscan), in fact equal
        for q in range(wl.nq):
            sl = wl.sl(q)
            err = np.linalg.norm(xb[sl] - xa[sl]) / np.linalg.norm(xa[sl])
            assert err <= 1e-5, (it, q, err)
        np.testing.assert_array_equal(ia, ib)
    torch.cuda.synchronize()
    # no device memory was taken by the static-scratch calls
    assert torch.cuda.mem_get_info(wl.dev)[0] >= free0
