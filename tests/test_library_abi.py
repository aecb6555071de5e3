"""CPU checks of the C ABI library: it loads, exports every entry point the
header declares, and its host-side ingest matches the oracle bit for bit."""
import os
import re

import numpy as np
import pytest

import oracle
import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def tgmod():
    import paper_2201_03509_gb300 as tg
    tg.build()
    return tg


def test_exports_every_declared_symbol(tgmod):
    hdr = open(os.path.join(ROOT, "include", "todgibbs.h")).read()
    hdr = re.sub(r"/\*.*?\*/", "", hdr, flags=re.S)
    names = set(re.findall(r"\b(tod_[a-z0-9_]+)\s*\(", hdr))
    assert len(names) >= 14
    L = tgmod.lib()
    for n in sorted(names):
        assert hasattr(L, n), n


def test_fft_length_matches_oracle(tgmod):
    for n in (0, 1, 2, 3, 4095, 4096, 90001, 115321, 140000, 299999):
        assert tgmod.fft_length(n) == oracle.fft_length(n)


def test_encoder_matches_oracle_bit_exact(tgmod):
    for cfg in (synth.CONFIGS["tiny"], synth.scaled(synth.CONFIGS["lfi30"], nscan=2, len_lo=5000,
                                                      len_hi=20000)):
        band = synth.make_band(cfg, with_noise=False)
        a = tgmod.ingest(band)
        b = oracle.ingest(band)
        assert np.array_equal(a["offsets"], b["offsets"])
        for kind in ("pix_streams", "psi_streams"):
            for k, v in b[kind].items():
                assert np.array_equal(np.asarray(v), np.asarray(a[kind][k])), (kind, k)


def test_encoder_adversarial_matches_oracle(tgmod):
    rng = np.random.default_rng(4)
    off = np.array([0, 1000, 2000, 2004], np.int64)   # ndet=1 nscan=3
    vals = np.concatenate([rng.integers(0, 1 << 20, 1000), np.full(1000, 5),
                           np.array([0, 2 ** 30, -2 ** 30, 7])]).astype(np.int32)
    a = tgmod.huff_encode(1, 3, off, vals)
    b = oracle.encode_band_streams([vals[0:1000], vals[1000:2000], vals[2000:2004]], 1)
    for k, v in b.items():
        assert np.array_equal(np.asarray(v), np.asarray(a[k])), k


def test_data_stream_encoder_matches_oracle(tgmod):
    cfg = synth.scaled(synth.CONFIGS["lfi30"], nscan=2, len_lo=5000, len_hi=20000)
    band = synth.make_band(cfg)
    a = tgmod.ingest(band, data_streams=True)
    b = oracle.ingest(band, data_streams=True)
    assert np.array_equal(a["tod_scale"], b["tod_scale"]) and a["flag_select"] == b["flag_select"]
    for kind in ("tod_streams", "flag_streams"):
        for k, v in b[kind].items():
            assert np.array_equal(np.asarray(v), np.asarray(a[kind][k])), (kind, k)


def test_encoder_rejects_a_difference_outside_int32(tgmod):
    vals = np.array([2 ** 31 - 1, -2 ** 31, 0, 1], np.int32)
    with pytest.raises(tgmod.TodError):
        tgmod.huff_encode(1, 1, np.array([0, 4]), vals)


def test_encoder_rejects_bad_offsets(tgmod):
    with pytest.raises(tgmod.TodError):
        tgmod.huff_encode(1, 2, np.array([0, 10, 5]), np.zeros(10, np.int32))


def test_pack_flags_layout(tgmod):
    f = np.zeros(70, bool)
    f[[0, 31, 32, 69]] = True
    w = tgmod.pack_flags(f)
    assert len(w) == 3 and w[0] == (1 | (1 << 31)) and w[1] == 1 and w[2] == (1 << 5)
