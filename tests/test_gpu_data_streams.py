"""Compressed TOD and flag streams on the GPU, through the C ABI (Sect. 4.1;
Listing `tod`): the decoded FP32 data and flag bitmask against the oracle's
decode (bit-exact), misuse errors, and whole steps that decode their own
data against the same steps fed the oracle's decoded data (bit-exact)."""
import dataclasses

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

SEED, BAND = 31, 2


def _pack(mask):
    f = np.asarray(mask, bool)
    f = np.concatenate([f, np.zeros((-len(f)) % 32, bool)])
    return np.packbits(f, bitorder="little").view("<u4")


@pytest.fixture(scope="module", params=["lfi30_small", "tiny"])
def dw(request):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2201_03509_gb300 as tg
    if request.param == "tiny":                           # word-aligned detscans, flags on
        cfg = dataclasses.replace(synth.CONFIGS["tiny"], flag_frac=0.05)
    else:                                                 # ragged detscans share flag words
        cfg = synth.scaled(synth.CONFIGS["lfi30"], nscan=3, len_lo=9000, len_hi=30000)
    band = synth.make_band(cfg)
    ing = tg.ingest(band, data_streams=True)
    off = ing["offsets"]
    plan = tg.Plan(cfg.nside, cfg.ndet, cfg.nscan, cfg.fsamp, off, ing["pix_streams"], ing["psi_streams"])
    plan.attach_data(ing["tod_streams"], ing["tod_scale"], ing["flag_streams"], ing["flag_select"])
    ref = oracle.ingest(band, data_streams=True)
    d_ref = oracle.decode_tod(ref["tod_streams"], off, cfg.ndet, ref["tod_scale"])
    m_ref = oracle.decode_flags(ref["flag_streams"], off, cfg.ndet, ref["flag_select"])
    return dict(cfg=cfg, band=band, ing=ing, plan=plan, off=off, N=int(off[-1]), d_ref=d_ref, m_ref=m_ref,
                ragged=request.param != "tiny")


def test_decode_data_bit_exact(dw):
    import torch
    N, dev = dw["N"], torch.device("cuda:0")
    assert np.any(dw["off"] % 32 != 0) == dw["ragged"]
    d = torch.full((N,), float("nan"), dtype=torch.float32, device=dev)
    fl = torch.full(((N + 31) // 32,), -1, dtype=torch.int32, device=dev)   # fully rewritten
    dw["plan"].decode_data(d, fl)
    dw["plan"].status()
    assert np.array_equal(d.cpu().numpy().view(np.uint32), dw["d_ref"].view(np.uint32))
    want = _pack(dw["m_ref"])
    assert dw["m_ref"].any()
    assert np.array_equal(fl.cpu().numpy().view(np.uint32), want)
    # one output alone
    d2 = torch.zeros_like(d)
    dw["plan"].decode_data(d2, None)
    fl2 = torch.zeros_like(fl)
    dw["plan"].decode_data(None, fl2)
    dw["plan"].status()
    assert torch.equal(d2, d) and torch.equal(fl2, fl)


def test_decode_data_misuse(dw):
    import torch
    import paper_2201_03509_gb300 as tg
    ing = dw["ing"]
    with pytest.raises(tg.TodError):                      # attached once per plan
        dw["plan"].attach_data(ing["tod_streams"], ing["tod_scale"], ing["flag_streams"], ing["flag_select"])
    with pytest.raises(tg.TodError):
        dw["plan"].decode_data(None, None)
    cfg = dw["cfg"]
    bare = tg.Plan(cfg.nside, cfg.ndet, cfg.nscan, cfg.fsamp, dw["off"], ing["pix_streams"], ing["psi_streams"])
    d = torch.zeros(dw["N"], dtype=torch.float32, device="cuda:0")
    with pytest.raises(tg.TodError):                      # nothing attached
        bare.decode_data(d, None)
    bad = ing["tod_scale"].copy()
    bad[0] = 0.0
    with pytest.raises(tg.TodError):
        bare.attach_data(ing["tod_streams"], bad, ing["flag_streams"], ing["flag_select"])
    bare.close()


@pytest.mark.parametrize("lookahead", [False, True])
def test_step_with_data_streams_equals_step_fed_decoded_data(dw, lookahead):
    import torch
    import paper_2201_03509_gb300 as tg
    from paper_2201_03509_gb300.step import GibbsTODStep
    band, plan = dw["band"], dw["plan"]
    m4 = np.zeros((band.npix, 4), np.float32)
    m4[:, :3] = band.map_tqu.T
    t_map = torch.from_numpy(m4).to("cuda:0")
    a = GibbsTODStep(plan, band.psd, None, data_streams=True)
    b = GibbsTODStep(plan, band.psd, _pack(dw["m_ref"]))
    b.set_tod(dw["d_ref"])
    a.lookahead = b.lookahead = lookahead
    for it in range(3):
        for st in (a, b):
            st.run(t_map, tg.Rng(SEED, BAND, it))
            torch.cuda.synchronize()
        plan.status()
        for name in ("gain", "ncorr", "map", "hits", "cg_iters"):
            assert torch.equal(getattr(a, name), getattr(b, name)), (it, name)
        assert torch.equal(a.d, b.d) and torch.equal(a.flags, b.flags)
    assert a.launches_per_step == b.launches_per_step + 2


def test_graph_replay_with_data_streams_and_gain_prior(dw):
    """A captured step that decodes its own data and draws the gains under
    the smooth prior replays bit for bit like the eager step."""
    import torch
    import paper_2201_03509_gb300 as tg
    from paper_2201_03509_gb300.step import GibbsTODStep
    band, plan = dw["band"], dw["plan"]
    m4 = np.zeros((band.npix, 4), np.float32)
    m4[:, :3] = band.map_tqu.T
    t_map = torch.from_numpy(m4).to("cuda:0")
    prior = np.array([[2e-3, -2.0]] * dw["cfg"].ndet)
    step = GibbsTODStep(plan, band.psd, None, data_streams=True, gain_prior=prior)
    step.lookahead = False
    step.run(t_map, tg.Rng(3, 0, 5), tg.MODE_DRAW)
    torch.cuda.synchronize()
    plan.status()
    ref = [t.clone() for t in (step.gain, step.ncorr, step.map, step.d, step.flags)]
    step.capture(t_map, 3, 0, tg.MODE_DRAW)
    step.replay(5)
    torch.cuda.synchronize()
    plan.status()
    for a, b in zip(ref, (step.gain, step.ncorr, step.map, step.d, step.flags)):
        assert torch.equal(a, b)
    assert step.gain_iters.min().item() >= 1


def test_decode_wide_values_and_long_codes(dw):
    """ADC counts whose differences include values too wide for the packed
    table entry (|delta| >= 2^26) and many rare symbols (codes longer than
    the 13-bit table) decode bit for bit."""
    import torch
    import paper_2201_03509_gb300 as tg
    cfg, off, ing = dw["cfg"], dw["off"], dw["ing"]
    rng = np.random.default_rng(11)
    N = int(off[-1])
    counts = np.empty(N, np.int64)
    for q in range(len(off) - 1):
        n = int(off[q + 1] - off[q])
        dl = rng.integers(-3, 4, n)
        rare = rng.random(n) < 0.05
        dl[rare] = rng.integers(-5000, 5000, rare.sum())             # many distinct, long codes
        wide = np.flatnonzero(rng.random(n) < 0.002)
        # jumps of 2^26 .. 2^27 with alternating signs: the walk stays bounded
        dl[wide] = np.where(np.arange(len(wide)) % 2 == 0, 1, -1) * rng.integers(1 << 26, 1 << 27, len(wide))
        c = np.cumsum(dl)
        c -= (c.max() + c.min()) // 2                              # centred: |c| well inside int32
        assert np.abs(c).max() < 2 ** 30
        counts[off[q]:off[q + 1]] = c
    st = tg.huff_encode(cfg.ndet, cfg.nscan, off, counts.astype(np.int32))
    if dw["ragged"]:                                               # 4 detscans per code: rare symbols get long codes
        assert st["sym_len"].max() > 13
    scale = np.full(len(off) - 1, 2.0 ** -10)
    plan = tg.Plan(cfg.nside, cfg.ndet, cfg.nscan, cfg.fsamp, off, ing["pix_streams"], ing["psi_streams"])
    plan.attach_data(st, scale, ing["flag_streams"], ing["flag_select"])
    d = torch.empty(N, dtype=torch.float32, device="cuda:0")
    plan.decode_data(d, None)
    plan.status()
    want = oracle.decode_tod(st, off, cfg.ndet, scale)
    assert np.array_equal(d.cpu().numpy().view(np.uint32), want.view(np.uint32))
    assert np.array_equal(oracle.decode_band(st, off, cfg.ndet), counts)
    plan.close()
