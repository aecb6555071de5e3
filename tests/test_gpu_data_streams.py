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
