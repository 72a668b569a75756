"""Write the stored FP64 oracle values that the large-size parity tests and the
benchmark compare against.

Every value written here comes from ``oracle/`` (dense FP64 rows of the P1
operator G of Section 2, applied to seeded inputs from ``workloads/``); nothing
is read from the CUDA library.  The files hold, for 1000 rows drawn with
``workloads.sample_rows(N, 1000, seed=0)`` and the input
``X = workloads.rand_vectors((F, N), seed=0)`` (uniform on [0, 1]):

  rows  int32 [1000]        sampled vertex ids (caller order)
  Y     float64 [F, 1000]   (G_{g(nu)} X_nu)_i at those rows

Usage:  python tests/golden/make_golden.py [cube32_F16] [cube64_F64s]
(about 5 minutes and 35 minutes on 8 cores).
"""
from __future__ import annotations

import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402
from oracle import oracle as O  # noqa: E402

ROWS = 1000
CHUNK = 25


def problems():
    return {"cube32_F16": W.multifreq_32, "cube64_F64s": W.shared_kappa_64}


def sampled_apply(p, rows, X):
    """(G_{g(nu)} X_nu) at `rows`, dense FP64 rows computed a chunk at a time."""
    _, gidx = O.groups_of(p.freqs)
    out = np.zeros((p.freqs.F, rows.shape[0]))
    for r0 in range(0, rows.shape[0], CHUNK):
        r = rows[r0:r0 + CHUNK]
        R = O.G_rows(p, r)   # [r, G, N]
        for f in range(p.freqs.F):
            out[f, r0:r0 + len(r)] = R[:, gidx[f], :] @ X[f]
    return out


def path(name: str) -> str:
    return os.path.join(HERE, f"{name}_apply_rows{ROWS}.npz")


def make(name: str) -> str:
    p = problems()[name]()
    rows = W.sample_rows(p.N, ROWS, seed=0)
    X = W.rand_vectors((p.freqs.F, p.N), seed=0)
    t0 = time.time()
    Y = sampled_apply(p, rows, X)
    np.savez_compressed(path(name), rows=rows, Y=Y)
    print(f"{name}: {ROWS} rows in {time.time() - t0:.0f} s -> {path(name)}")
    return path(name)


if __name__ == "__main__":
    for nm in sys.argv[1:] or list(problems()):
        make(nm)
