"""ctypes loader for the oracle's plain-C Huffman coder (``huffman.c``).

TEST INFRASTRUCTURE ONLY: imported by tests/, __graft_entry__.smoke() and the
CPU-baseline leg of bench.py, never by the GPU library.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "huffman.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_OUT_DIR, "liboracle_huffman.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile huffman.c with gcc into oracle/_build/ (idempotent)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".%d.tmp" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-std=c99", "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        P = ctypes.c_void_p
        L.oracle_huff_lengths.argtypes = [P, ctypes.c_int32, ctypes.c_int32, P]
        L.oracle_huff_lengths.restype = ctypes.c_int
        L.oracle_huff_canonical.argtypes = [P, ctypes.c_int32, P]
        L.oracle_huff_canonical.restype = ctypes.c_int
        L.oracle_huff_encode.argtypes = [P, ctypes.c_int64, P, P, P, ctypes.c_int32, P,
                                         ctypes.c_int64, P]
        L.oracle_huff_encode.restype = ctypes.c_int
        L.oracle_huff_decode.argtypes = [P, ctypes.c_int64, ctypes.c_int64, P, P, P,
                                         ctypes.c_int32, P, ctypes.c_int64]
        L.oracle_huff_decode.restype = ctypes.c_int64
        _lib = L
    return _lib


def _p(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data)


def code_lengths(counts: np.ndarray, maxlen: int) -> np.ndarray:
    counts = np.ascontiguousarray(counts, dtype=np.int64)
    out = np.zeros(len(counts), dtype=np.uint8)
    if lib().oracle_huff_lengths(_p(counts), len(counts), maxlen, _p(out)) != 0:
        raise ValueError("bad Huffman input")
    return out


def canonical_codes(lengths: np.ndarray) -> np.ndarray:
    lengths = np.ascontiguousarray(lengths, dtype=np.uint8)
    out = np.zeros(len(lengths), dtype=np.uint32)
    lib().oracle_huff_canonical(_p(lengths), len(lengths), _p(out))
    return out


def encode_into(words: np.ndarray, bitpos: int, syms: np.ndarray, vals, codes, lengths) -> int:
    syms = np.ascontiguousarray(syms, dtype=np.int32)
    bp = np.array([bitpos], dtype=np.int64)
    rc = lib().oracle_huff_encode(_p(syms), len(syms), _p(vals), _p(codes), _p(lengths), len(vals),
                                  _p(words), len(words), _p(bp))
    if rc != 0:
        raise ValueError("Huffman encode failed")
    return int(bp[0])


def decode(words: np.ndarray, nbits: int, bitpos: int, n: int, vals, codes, lengths):
    out = np.zeros(n, dtype=np.int32)
    words = np.ascontiguousarray(words, dtype=np.uint32)
    end = lib().oracle_huff_decode(_p(words), nbits, bitpos, _p(vals), _p(codes), _p(lengths),
                                   len(vals), _p(out), n)
    if end < 0:
        raise ValueError("corrupt Huffman stream")
    return out, int(end)
