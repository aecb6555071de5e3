"""Pins of the oracle's compression (paper Sect. 4.1): round trips, the
prefix-code invariants, and the paper's worked example of code lengths."""
import os

import numpy as np
import pytest

import oracle
from oracle import _huff

GOLD = os.path.join(os.path.dirname(__file__), "golden", "huffman_pid27646_shape.txt")


def _roundtrip(values_per_detscan, ndet):
    st = oracle.encode_band_streams(values_per_detscan, ndet)
    for q, v in enumerate(values_per_detscan):
        out = oracle.decode_detscan(st, q, len(v), ndet)
        assert np.array_equal(out, np.asarray(v, np.int64))
    return st


def test_roundtrip_random_walk():
    rng = np.random.default_rng(0)
    vals = [np.cumsum(rng.integers(-3, 4, size=n)) + 1000 for n in (1, 2, 511, 512, 513, 3000)]
    _roundtrip(vals, 1)


def test_roundtrip_iid_psi_and_single_symbol():
    rng = np.random.default_rng(1)
    iid = [rng.integers(0, 4096, size=2000) for _ in range(2)]
    _roundtrip(iid, 2)
    const = [np.full(700, 7), np.full(700, 7)]            # deltas {7, 0}
    _roundtrip(const, 2)
    zeros = [np.zeros(1000, np.int64)]                    # one distinct delta
    st = _roundtrip(zeros, 1)
    assert list(st["sym_len"]) == [1]


def test_roundtrip_tiny_band(tiny_band, tiny_ingest):
    off = tiny_ingest["offsets"]
    pix = oracle.decode_band(tiny_ingest["pix_streams"], off, 1)
    psi = oracle.decode_band(tiny_ingest["psi_streams"], off, 1)
    for q in range(tiny_band.ndetscan):
        n = off[q + 1] - off[q]
        assert np.array_equal(pix[off[q]:off[q + 1]], tiny_band.pix[q][:n])
        assert np.array_equal(psi[off[q]:off[q + 1]], tiny_band.psi[q][:n])


def test_kraft_equality_and_prefix_free():
    rng = np.random.default_rng(2)
    for k in (2, 3, 10, 300):
        counts = rng.integers(1, 10000, size=k)
        L = _huff.code_lengths(counts, 24)
        assert sum(2.0 ** -int(l) for l in L) == 1.0          # full binary tree
        codes = _huff.canonical_codes(L)
        words = ["{:0{}b}".format(int(c), int(l)) for c, l in zip(codes, L)]
        for i, a in enumerate(words):
            for j, b in enumerate(words):
                if i != j:
                    assert not b.startswith(a)


def test_lengths_are_optimal_small():
    """Huffman lengths minimise sum count*len over all prefix codes: compare
    the total with an exhaustive search over Kraft-feasible length vectors."""
    import itertools
    rng = np.random.default_rng(3)
    for _ in range(20):
        counts = rng.integers(1, 50, size=5)
        L = _huff.code_lengths(counts, 24)
        best = min(
            sum(c * l for c, l in zip(counts, ls))
            for ls in itertools.product(range(1, 6), repeat=5)
            if sum(2.0 ** -l for l in ls) <= 1.0)
        assert int(np.dot(counts, L.astype(np.int64))) == best


def test_length_limit():
    fib = [1, 1]
    while len(fib) < 40:
        fib.append(fib[-1] + fib[-2])
    L = _huff.code_lengths(np.array(fib), 24)
    assert L.max() <= 24
    assert sum(2.0 ** -int(l) for l in L) <= 1.0


def test_paper_example_code_lengths():
    """Paper Sect. 4.1 / Fig. `huffman`: with 0 at 42 % of the differenced
    stream, 0 gets a 1-bit code, +1 and -1 4-bit codes, -2 a 5-bit code, and
    the longest codes (symbols seen once) are 20 bits."""
    data = np.loadtxt(GOLD, dtype=np.int64)
    vals, counts = data[:, 0], data[:, 1]
    assert len(vals) == 670 and counts.sum() == 861276
    L = dict(zip(vals.tolist(), _huff.code_lengths(counts, 24).tolist()))
    assert L[0] == 1 and L[1] == 4 and L[-1] == 4 and L[-2] == 5
    assert max(L.values()) == 20
    # the 1-bit code is '0', as in the paper
    c = _huff.canonical_codes(np.array([L[v] for v in vals], np.uint8))
    assert int(c[list(vals).index(0)]) == 0


def test_checkpoints_restart_decoding(tiny_band, tiny_ingest):
    """Decoding from any checkpoint (bit offset + preceding value) gives the
    same samples as decoding from the start."""
    st = tiny_ingest["psi_streams"]
    off = tiny_ingest["offsets"]
    B = oracle.CKPT_BLOCK
    for q in (0, 7, 15):
        n = int(off[q + 1] - off[q])
        full = oracle.decode_detscan(st, q, n, 1)
        a = st["sym_off"][0]
        vals = st["sym_vals"][st["sym_off"][q]:st["sym_off"][q + 1]]
        L = st["sym_len"][st["sym_off"][q]:st["sym_off"][q + 1]]
        codes = _huff.canonical_codes(L)
        words = st["words"][st["word_off"][q]:st["word_off"][q + 1]]
        for blk in range(st["blk_off"][q], st["blk_off"][q + 1]):
            j = blk - st["blk_off"][q]
            m = min(B, n - j * B)
            dl, _ = _huff.decode(words, int(st["nbits"][q]), int(st["ckpt_bit"][blk]), m,
                                 np.ascontiguousarray(vals), codes, np.ascontiguousarray(L))
            x = st["ckpt_val"][blk] + np.cumsum(dl.astype(np.int64))
            assert np.array_equal(x, full[j * B:j * B + m])


def test_corrupt_stream_detected():
    st = oracle.encode_band_streams([np.arange(100)], 1)
    st["nbits"][0] -= 5
    with pytest.raises(ValueError):
        oracle.decode_detscan(st, 0, 100, 1)
