"""Pins of the oracle's decode of the compressed TOD and flag streams
(paper Sect. 4.1: ADC integers and flag words differenced and Huffman coded;
Listing `tod`: tod and flag kept as compressed bytes): exact round trips of
the integers, the quantisation bound of the FP32 data, an exact case, the
flag selection against the generator's own mask, and the compression the
paper's table reports for the 30 GHz TOD."""
import numpy as np
import pytest

import oracle
import synth


@pytest.fixture(scope="module")
def band_ing():
    cfg = synth.scaled(synth.CONFIGS["lfi30"], nscan=2, len_lo=20000, len_hi=40000)
    band = synth.make_band(cfg)
    return band, oracle.ingest(band, data_streams=True)


def test_counts_round_trip(band_ing):
    band, ing = band_ing
    off = ing["offsets"]
    c = oracle.decode_band(ing["tod_streams"], off, band.cfg.ndet)
    assert np.array_equal(c, np.concatenate(ing["tod_counts"]).astype(np.int64))
    assert c.min() < 0 < c.max()                       # signed counts with wide differences
    w = oracle.decode_band(ing["flag_streams"], off, band.cfg.ndet)
    assert np.array_equal(w, np.concatenate(ing["flag_words"]).astype(np.int64))


def test_tod_within_half_a_quantum(band_ing):
    band, ing = band_ing
    off = ing["offsets"]
    d = oracle.decode_tod(ing["tod_streams"], off, band.cfg.ndet, ing["tod_scale"]).astype(np.float64)
    ref = ing["tod"].astype(np.float64)
    sc = np.repeat(ing["tod_scale"], np.diff(off))
    # rounding to the nearest count, then one FP32 rounding of the product
    bound = 0.5 * sc * (1 + 1e-12) + np.abs(ref) * 2.0 ** -23
    assert np.all(np.abs(d - ref) <= bound)
    assert np.std(d - ref) > 0.2 * sc.mean()          # the quantisation is really there


def test_tod_exact_for_a_power_of_two_quantum():
    rng = np.random.default_rng(3)
    counts = [np.cumsum(rng.integers(-300, 301, size=n)).astype(np.int64) for n in (1000, 1000, 700, 700)]
    off = np.concatenate([[0], np.cumsum([len(c) for c in counts])]).astype(np.int64)
    st = oracle.encode_band_streams(counts, 2)
    scale = np.array([2.0 ** -7, 2.0 ** -7, 2.0 ** -3, 2.0 ** -3])
    d = oracle.decode_tod(st, off, 2, scale)
    want = np.concatenate([c / 128.0 for c in counts[:2]] + [c / 8.0 for c in counts[2:]])
    assert d.dtype == np.float32
    assert np.array_equal(d.astype(np.float64), want)     # every value exact in FP32


def test_flag_selection_matches_the_generator(band_ing):
    band, ing = band_ing
    off = ing["offsets"]
    m = oracle.decode_flags(ing["flag_streams"], off, band.cfg.ndet, ing["flag_select"])
    assert np.array_equal(m, ing["flags"])
    w = np.concatenate(ing["flag_words"])
    assert np.any(((w & synth.FLAG_INFO) != 0) & ~ing["flags"])   # informational bits are not selected
    assert not np.any(oracle.decode_flags(ing["flag_streams"], off, band.cfg.ndet, synth.FLAG_INFO << 1))


def test_tod_compression_matches_the_paper_table(band_ing):
    """Sect. 4.1, table of Huffman compression: the 30 GHz TOD takes 361 MB
    raw and 52 MB compressed; raw TOD, pixel, psi and flag volumes stand
    8:4:2:1 (361:181:90:45), i.e. 8-byte samples, so 52/361 x 64 = 9.2 bits
    per compressed sample.  The generator's ADC quantum is chosen for that."""
    band, ing = band_ing
    bits = ing["tod_streams"]["nbits"].sum() / ing["offsets"][-1]
    assert 52 / 361 * 64 == pytest.approx(9.22, abs=0.01)
    assert 8.6 < bits < 9.8, bits
    fbits = ing["flag_streams"]["nbits"].sum() / ing["offsets"][-1]
    assert 1.0 <= fbits < 1.2, fbits          # one bit per sample is a symbol code's floor


def test_round_trip_wide_differences_and_long_codes():
    """Counts whose differences reach +-2^27 and a heavy tail of rare
    symbols (codes longer than 13 bits) round-trip exactly."""
    rng = np.random.default_rng(12)
    vals = []
    for n in (20000, 20000, 15001, 15001):
        dl = rng.integers(-3, 4, n)
        rare = rng.random(n) < 0.05
        dl[rare] = rng.integers(-5000, 5000, rare.sum())
        wide = np.flatnonzero(rng.random(n) < 0.003)
        dl[wide] = np.where(np.arange(len(wide)) % 2 == 0, 1, -1) * rng.integers(1 << 26, 1 << 27, len(wide))
        vals.append(np.cumsum(dl))
    st = oracle.encode_band_streams(vals, 2)
    assert st["sym_len"].max() > 13
    assert np.abs(st["sym_vals"]).max() >= 2 ** 26
    off = np.concatenate([[0], np.cumsum([len(v) for v in vals])]).astype(np.int64)
    assert np.array_equal(oracle.decode_band(st, off, 2), np.concatenate(vals))
