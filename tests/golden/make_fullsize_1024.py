"""Write the sampled oracle solution of the 1024^3 random-source workload.

Workload: 1024^3 cells on the unit cube (spacing 1/1024 per axis), faces Neumann-x,
Dirichlet-y, Neumann-z ("NNDDNN"), source f = workloads.uniform_source(shape, seed=2):
i.i.d. U[-1,1] drawn by numpy's default_rng, mean removed.  The CPU oracle (naive
O(N^2) line transforms and textbook Thomas per mode, FP64) solves it once; this script
then stores u at a seeded set of cells -- every edge cell, four whole z-columns, two whole
x-lines and two whole y-lines, 4000 cells of every face and random interior cells, 100000
cells in all -- together with ||u||_2, sum(u) and max|u| of the whole grid.

Only the oracle computes anything stored here.  It takes about 2.5 hours on 8 host cores
and 32 GB of RAM:

    python tests/golden/make_fullsize_1024.py [--keep-full /path/u.npy]
"""
from __future__ import annotations

import argparse
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

N = 1024
BC = "NNDDNN"
SEED = 2
SAMPLE_SEED = 7
COUNT = 100000
OUT = os.path.join(HERE, "fullsize_1024_nnddnn.txt")


def sample_cells(n: int = N, count: int = COUNT, seed: int = SAMPLE_SEED) -> np.ndarray:
    """Flat indices (k*n*n + j*n + i) of the stored cells, sorted and unique."""
    rng = np.random.default_rng(seed)
    ar = np.arange(n)
    last = n - 1
    sel = []

    def flat(k, j, i):
        return (np.asarray(k, np.int64) * n + np.asarray(j, np.int64)) * n + np.asarray(i, np.int64)

    # the twelve edges of the cube (corners included)
    for a in (0, last):
        for b in (0, last):
            sel.append(flat(ar, a, b))      # along z
            sel.append(flat(a, ar, b))      # along y
            sel.append(flat(a, b, ar))      # along x
    # whole z-columns (one mode's tridiagonal line in physical space), x-lines and y-lines
    for (j, i) in ((1, 1), (511, 700), (1022, 3), (300, 1021)):
        sel.append(flat(ar, j, i))
    for (k, j) in ((1, 512), (777, 1022)):
        sel.append(flat(k, j, ar))
    for (k, i) in ((513, 1), (2, 333)):
        sel.append(flat(k, ar, i))
    # random cells of each face
    per_face = 4000
    for axis in range(3):
        for side in (0, last):
            c = rng.integers(0, n, size=(per_face, 3))
            c[:, axis] = side
            sel.append(flat(c[:, 0], c[:, 1], c[:, 2]))
    idx = np.unique(np.concatenate(sel))
    # random cells anywhere until `count` distinct cells are chosen
    while idx.size < count:
        extra = rng.integers(0, n ** 3, size=count - idx.size, dtype=np.int64)
        idx = np.unique(np.concatenate([idx, extra]))
    return idx


def main():
    import oracle
    from paper_1909_05423_gb300 import workloads

    ap = argparse.ArgumentParser()
    ap.add_argument("--keep-full", default=None, help="also save the whole oracle solution here (.npy)")
    ap.add_argument("--from-full", default=None, help="sample a previously saved solution instead of solving")
    args = ap.parse_args()
    shape = (N, N, N)
    if args.from_full:
        u = np.load(args.from_full, mmap_mode="r")
        threads, secs = oracle.num_threads(), float("nan")
    else:
        f = workloads.uniform_source(shape, seed=SEED)
        oracle.build()
        t0 = time.time()
        u = oracle.solve(f, BC, (1.0 / N, 1.0 / N, 1.0 / N))
        secs = time.time() - t0
        threads = oracle.num_threads()
        del f
        if args.keep_full:
            np.save(args.keep_full, u)
    idx = sample_cells()
    flat = np.asarray(u).reshape(-1)
    vals = np.asarray(flat[idx], dtype=np.float64)
    norm = float(np.sqrt(np.sum(np.square(flat, dtype=np.float64))))
    total = float(np.sum(flat, dtype=np.float64))
    umax = float(np.max(np.abs(flat)))
    with open(OUT, "w") as fh:
        fh.write("# Oracle solution of the 1024^3 random-source workload at sampled cells.\n")
        fh.write("# Written by tests/golden/make_fullsize_1024.py (calls only oracle/): bc %s, spacing 1/%d,\n" % (BC, N))
        fh.write("# f = workloads.uniform_source((%d,%d,%d), seed=%d) (numpy default_rng U[-1,1], mean removed).\n"
                 % (N, N, N, SEED))
        fh.write("# Cells: sample_cells(n=%d, count=%d, seed=%d); oracle ran %.0f s on %d threads.\n"
                 % (N, COUNT, SAMPLE_SEED, secs, threads))
        fh.write("# Columns: flat index k*n*n + j*n + i, u.\n")
        fh.write("norm2 %.17e\n" % norm)
        fh.write("sum %.17e\n" % total)
        fh.write("maxabs %.17e\n" % umax)
        for p, v in zip(idx.tolist(), vals.tolist()):
            fh.write("%d %.17e\n" % (p, v))
    print("wrote", OUT, idx.size, "cells; norm2", norm, "seconds", secs)


if __name__ == "__main__":
    main()
