#!/usr/bin/env python3
"""Writes tests/golden/cr48_levels.txt: the lowest levels of the pf-shell
4-proton 4-neutron M = 0 space (48Cr, dim 1,963,461) with the seeded random
interaction, from the FP64 oracle alone.

The oracle builds the explicit M-scheme H from bit operations (about 1.2e9
stored elements, ~19 GB, ~38 GB while it is built) and runs its Lanczos with
full reorthogonalization (Sec. "Standard Lanczos algorithm") from the seeded
pivot; each kept level's residual |H psi - E psi| is taken with the explicit
matrix.  Nothing here touches the CUDA library.

    python tests/golden/make_cr48_levels.py [--niter 300] [--nkeep 10]
"""
import argparse
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle as O  # noqa: E402
from paper_1801_08432_gb300 import inputs as I  # noqa: E402


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--niter", type=int, default=300)
    ap.add_argument("--nkeep", type=int, default=10)
    ap.add_argument("--out", default=os.path.join(os.path.dirname(os.path.abspath(__file__)), "cr48_levels.txt"))
    a = ap.parse_args()
    orbits, spe, tb = I.space("pf")
    o = O.Oracle(orbits, 4, 4, 0, 0).set_interaction(spe, tb)
    t0 = time.time()
    nnz = o.build_matrix()
    t_build = time.time() - t0
    p = I.random_block(o.dim, 1, seed=I.PIVOT_SEED)[:, 0]
    t0 = time.time()
    ev, X = o.lanczos(p, a.niter, nkeep=a.nkeep, return_vectors=True)
    t_lanczos = time.time() - t0
    res = [float(np.linalg.norm(o.spmv(X[:, m]) - ev[m] * X[:, m]) / np.linalg.norm(X[:, m]))
           for m in range(a.nkeep)]
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    with open(a.out, "w") as f:
        f.write("# Lowest levels of pf 4p4n M = 0 (48Cr, dim %d), seeded random TBMEs (seed %d), from the FP64\n"
                % (o.dim, I.TBME_SEED))
        f.write("# oracle's explicit H (%d stored elements) and its Lanczos with full reorthogonalization\n" % nnz)
        f.write("# (Sec. \"Standard Lanczos algorithm\"), %d iterations from the seeded pivot (seed %d).\n"
                % (a.niter, I.PIVOT_SEED))
        f.write("# Written by tests/golden/make_cr48_levels.py (oracle only): H built in %.0f s, Lanczos %.0f s,\n"
                % (t_build, t_lanczos))
        f.write("# %d host threads.\n" % cores)
        f.write("# level  E (MeV)  residual |H psi - E psi| (MeV)\n")
        for m in range(a.nkeep):
            f.write("%d %.10f %.3e\n" % (m, ev[m], res[m]))
    print(open(a.out).read())


if __name__ == "__main__":
    main()
