"""Edge cases of the correlated-noise draw and the status paths, through the
C ABI against the FP64 oracle: gaps longer than the preconditioner's block
(split into several Toeplitz blocks), gaps touching the first and the last
sample, a detscan with every sample flagged, a single flagged sample, more
gaps than the preconditioner takes (plain CG), more gaps than the coarse
correction takes (block inverses alone) and exactly as many, detscans of a
few dozen samples; and the per-detscan status words for an iteration cap of one and
for non-finite data."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

SEED, BAND, IT = 5, 1, 2


def _with_mask(wl, flagged):
    """Replace the workload's flags by `flagged` (bool per sample)."""
    import torch
    import paper_2201_03509_gb300 as tg
    wl.flags = flagged
    wl.mask = (~flagged).astype(np.float64)
    wl.t_flags = torch.from_numpy(tg.pack_flags(flagged).view(np.int32)).to(wl.dev)
    return wl


def _edge_mask(wl):
    f = np.zeros(wl.N, dtype=bool)
    def seg(q, a, b):
        o = int(wl.off[q])
        f[o + a:o + b] = True
    n = lambda q: int(wl.off[q + 1] - wl.off[q])
    seg(0, 0, 700)                            # touches sample 0, longer than one block
    seg(1, n(1) - 300, n(1))                  # touches the last sample
    seg(2, 0, n(2))                           # every sample flagged
    seg(3, 0, 1)                              # one flagged sample
    for k in range(300):                      # 300 one-sample gaps: more gaps than the preconditioner holds
        seg(4, 100 + 3 * k, 101 + 3 * k)
    seg(5, 1000, 2500)                        # three preconditioner blocks
    seg(5, 2600, 2610)
    seg(6, 4095, 4096) if n(6) >= 4096 else seg(6, n(6) - 1, n(6))
    seg(7, 2, 3)
    seg(7, 5, 6)
    for k in range(100):                      # 100 gaps: block inverses without the coarse correction
        seg(8, 40 + 30 * k, 43 + 30 * k)
    for k in range(64):                       # 64 gaps: the most blocks with the coarse correction
        seg(9, 40 + 40 * k, 40 + 40 * k + 2 + k % 7)
    return f


@pytest.fixture(scope="module", params=["persistent", "per_scan"])
def edge(request):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from gpu_workload import Workload
    wl = Workload(synth.CONFIGS["tiny"])
    if request.param == "per_scan":
        wl.plan.set_schedule(wl.plan.SCHED_PER_SCAN)
    return _with_mask(wl, _edge_mask(wl))


@pytest.fixture(scope="module")
def short():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from gpu_workload import Workload
    cfg = synth.scaled(synth.CONFIGS["tiny"], nscan=6, len_lo=40, len_hi=130)
    wl = Workload(cfg)
    f = np.zeros(wl.N, dtype=bool)
    for q in range(wl.nq):
        o, n = int(wl.off[q]), int(wl.off[q + 1] - wl.off[q])
        if q % 2:
            f[o + n // 3:o + n // 3 + 5] = True
    return _with_mask(wl, f)


def _ncorr_vs_oracle(wl, mode, cg_tol=1e-7):
    import torch
    import paper_2201_03509_gb300 as tg
    gains = np.asarray(wl.band.gain[:wl.nq], np.float64)
    x = torch.zeros(wl.N, dtype=torch.float32, device=wl.dev)
    its = torch.zeros(wl.nq, dtype=torch.int32, device=wl.dev)
    wl.plan.sample_ncorr(wl.t_d, wl.t_s, torch.from_numpy(gains).to(wl.dev), wl.t_flags, wl.t_psd,
                         tg.Rng(SEED, BAND, IT), mode, x, its, cg_tol=cg_tol)
    st = wl.plan.status(raise_on_error=False)
    x = x.cpu().numpy().astype(np.float64)
    its = its.cpu().numpy()
    for q in range(wl.nq):
        sl = wl.sl(q)
        n = sl.stop - sl.start
        s0, fk, al = wl.band.psd[wl.det(q)]
        w1 = oracle.omega1(SEED, BAND, q, IT, n) if mode == 0 else np.zeros(n)
        w2 = oracle.omega2(SEED, BAND, q, IT, n) if mode == 0 else np.zeros(n)
        ref, rit = oracle.sample_ncorr(wl.d32[sl].astype(np.float64), wl.s32[sl].astype(np.float64), gains[q],
                                       wl.mask[sl], s0, fk, al, wl.cfg.fsamp, w1, w2)
        if not np.any(ref):          # no data and no noise terms: the draw is zero
            assert not np.any(x[sl]), q
        else:
            err = np.linalg.norm(x[sl] - ref) / np.linalg.norm(ref)
            assert err < 1e-5, (q, err, its[q], rit)
        assert st[q] == 0, (q, st[q])
    return its


@pytest.mark.parametrize("mode", [0, 1])
def test_ncorr_edge_gaps(edge, mode):
    its = _ncorr_vs_oracle(edge, mode)
    assert its[2] == 0                   # every sample flagged: solved exactly in the DCT basis
    assert its[0] > 0 and its[4] > 0 and its[5] > 0


@pytest.mark.parametrize("mode", [0, 1])
def test_ncorr_short_detscans(short, mode):
    _ncorr_vs_oracle(short, mode)


def test_gain_edge_masks(edge):
    """Gain draws on the same masks; the fully flagged detscan has no usable
    sample and is reported (TOD_ERR_ARG, gain 0), the others match."""
    import torch
    import paper_2201_03509_gb300 as tg
    wl = edge
    g = torch.zeros(wl.nq, dtype=torch.float64, device=wl.dev)
    mu = torch.zeros_like(g)
    sg = torch.zeros_like(g)
    wl.plan.sample_gain(wl.t_d, wl.t_s, wl.t_flags, wl.t_psd, tg.Rng(SEED, BAND, IT), tg.MODE_DRAW, g, mu, sg)
    st = wl.plan.status(raise_on_error=False)
    g = g.cpu().numpy()
    for q in range(wl.nq):
        if q == 2:
            assert st[q] == -1 and g[q] == 0.0
            continue
        sl = wl.sl(q)
        n = sl.stop - sl.start
        s0, fk, al = wl.band.psd[wl.det(q)]
        P = oracle.noise_psd(n, wl.cfg.fsamp, s0, fk, al)
        rg, rmu, rsg = oracle.sample_gain(wl.s32[sl].astype(np.float64), wl.d32[sl].astype(np.float64),
                                          wl.mask[sl], P, oracle.gain_normal(SEED, BAND, q, IT))
        assert st[q] == 0
        assert g[q] == pytest.approx(rg, rel=1e-5, abs=1e-5 * rsg)


def test_iteration_cap_reports_not_converged():
    """cg_maxiter = 1 on a flagged band: every detscan whose CG needs more
    iterations is marked TOD_ERR_NOT_CONVERGED (and reports one iteration)."""
    import torch
    import paper_2201_03509_gb300 as tg
    from gpu_workload import Workload
    wl = Workload(synth.scaled(synth.CONFIGS["lfi30"], nscan=2, len_lo=9000, len_hi=20000))
    gains = torch.from_numpy(np.asarray(wl.band.gain[:wl.nq], np.float64)).to(wl.dev)
    x = torch.zeros(wl.N, dtype=torch.float32, device=wl.dev)
    its = torch.zeros(wl.nq, dtype=torch.int32, device=wl.dev)
    wl.plan.sample_ncorr(wl.t_d, wl.t_s, gains, wl.t_flags, wl.t_psd, tg.Rng(SEED, BAND, IT), tg.MODE_DRAW, x,
                         its, cg_tol=1e-9, cg_maxiter=1)
    st = wl.plan.status(raise_on_error=False)
    its = its.cpu().numpy()
    flagged = [q for q in range(wl.nq) if wl.flags[wl.sl(q)].any()]
    assert flagged
    for q in flagged:
        assert its[q] == 1 and st[q] == -3, (q, its[q], st[q])
    # the status words are cleared by reading them
    assert not wl.plan.status(raise_on_error=False).any()


def test_non_finite_data_reported_by_gain():
    """A NaN in one detscan's data: its gain draw is reported as TOD_ERR_ARG
    (non-finite sums) with gain 0; the other detscans are unaffected."""
    import torch
    import paper_2201_03509_gb300 as tg
    from gpu_workload import Workload
    wl = Workload(synth.CONFIGS["tiny"])
    d = wl.t_d.clone()
    q_bad = 5
    d[int(wl.off[q_bad]) + 17] = float("nan")
    g = torch.zeros(wl.nq, dtype=torch.float64, device=wl.dev)
    wl.plan.sample_gain(d, wl.t_s, wl.t_flags, wl.t_psd, tg.Rng(SEED, BAND, IT), tg.MODE_MEAN, g)
    st = wl.plan.status(raise_on_error=False)
    g = g.cpu().numpy()
    assert st[q_bad] == -1 and g[q_bad] == 0.0
    assert np.all(st[np.arange(wl.nq) != q_bad] == 0)
    assert np.all(np.isfinite(g))
