"""Write ``oracle_cg_256cube.json``: how many iterations the oracle's
unpreconditioned FP64 CG needs on the 256^3 stretched variable-coefficient
workload (tanh stretching 1.5, k = exp(g) with the field of seed 3000,
correlation 8 cells, three mirror symmetries, the first uniform[-1, 1]
right-hand side of config 3) to reach a relative residual of 1e-8.

It calls only ``oracle/`` and the seeded inputs of ``synth``; the CPU legs of
``bench.py`` time a bounded sample of the same iteration and take the
iteration count from here.  The run takes tens of minutes on a few cores:

    python tests/golden/make_oracle_cg_256cube.py
"""

from __future__ import annotations

import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import fv, grid, native  # noqa: E402
from synth import gaussian_logk, rhs_uniform  # noqa: E402


def main():
    N, s, tol = (256, 256, 256), 3, 1e-8
    g = gaussian_logk(N, s, seed=3000, corr=8.0)
    A = fv.assemble(grid.widths(N, 1.5), np.exp(g))
    b = rhs_uniform(A.shape[0], 1, config=3)[0]
    t0 = time.time()
    x, info = native.cg(A, b, maxit=200000, tol=tol)
    out = dict(workload="3d7pt_vark_tanh_256cube_s3", n=int(A.shape[0]), nnz=int(A.nnz), tol=tol,
               iters=info["iters"], true_relres=info["relres"], threads=info["threads"],
               seconds=round(time.time() - t0, 1), cpu=native.cpu_model(),
               method="oracle/cg_omp.c: unpreconditioned FP64 CG from x = 0, recurrence residual <= tol ||b||")
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle_cg_256cube.json"), "w") as f:
        json.dump(out, f, indent=1)
    print(out)


if __name__ == "__main__":
    main()
