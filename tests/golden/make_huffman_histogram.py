"""Writes huffman_pid27646_shape.txt: a symbol histogram shaped like the
differenced 30 GHz pointing stream the paper describes for PID 27646
(Fig. `huffman` caption and Sect. 4.1): 670 distinct symbols, 861,276
entries, symbol 0 holding 42 % of them.  The paper does not print the
histogram itself, so this one is a construction with that shape: 0 gets 42 %,
|delta| >= 1 follows a two-sided geometric law (ratio 0.71, negative side
weighted 0.5), and singletons far out in the tail bring the symbol count to
670.  The expected code lengths checked against it are the paper's own:
0 -> 1 bit, +1 and -1 -> 4 bits, -2 -> 5 bits, longest code 20 bits.

Calls nothing under oracle/ or the library; run it to regenerate the file.
"""
import os

import numpy as np

N, K, R, A = 861276, 670, 0.71, 0.5


def histogram():
    n0 = int(round(0.42 * N))
    ks = np.arange(1, 400)
    w = np.concatenate([R ** (ks - 1), A * R ** (ks - 1)])
    vals = np.concatenate([ks, -ks])
    w = w / w.sum() * (N - n0)
    c = np.floor(w).astype(np.int64)
    keep = c >= 1
    vals, c = vals[keep], c[keep]
    need = K - 1 - len(vals)
    vals = np.concatenate([vals, np.arange(1000, 1000 + need)])
    c = np.concatenate([c, np.ones(need, np.int64)])
    c[0] += N - n0 - c.sum()
    allv = np.concatenate([[0], vals])
    allc = np.concatenate([[n0], c])
    o = np.argsort(allv)
    return allv[o], allc[o]


if __name__ == "__main__":
    v, c = histogram()
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "huffman_pid27646_shape.txt")
    with open(path, "w") as f:
        f.write("# Symbol histogram shaped like the paper's PID 27646 30 GHz example\n")
        f.write("# (arXiv 2201.03509, Fig. `huffman` caption; Sect. 4.1 text):\n")
        f.write("# 670 symbols, 861276 entries, p(0) = 0.42.  Written by make_huffman_histogram.py.\n")
        f.write("# expected (paper): len(0)=1 len(1)=4 len(-1)=4 len(-2)=5 maxlen=20\n")
        f.write("# columns: symbol count\n")
        for a, b in zip(v, c):
            f.write("%d %d\n" % (a, b))
