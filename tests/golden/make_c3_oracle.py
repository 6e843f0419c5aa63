"""Write tests/golden/c3_oracle_solution.txt: the FP64 oracle's solve of the
full-size N=128 Schur system (8,388,608 unknowns, lognormal viscosity
sigma = 1, Schur pressure correction with SA-AMG inner solves, GMRES(30) to
a relative residual of 1e-8).

It calls only the oracle and the seeded input generator.  The solution
itself (67 MB) is too large to keep, so the file stores what a GPU test
needs to measure its own solution against it:
  iterations   -- the oracle's GMRES iteration count;
  true_rel_res -- ||b - K x|| / ||b|| of the oracle's x;
  x_norm       -- ||x||_2;
  sample_idx / sample_x -- x at 2048 distinct indices drawn with
                  numpy.random.Generator(PCG64(3003)), from which
                  ||x_gpu - x|| / ||x|| is estimated as
                  sqrt(n/m sum_sample (x_gpu - x)^2) / ||x||.

Run from the repository root (about 5 minutes on one core):
    python tests/golden/make_c3_oracle.py
"""
from __future__ import annotations

import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import stokes_inputs as si  # noqa: E402
from oracle import bsr, krylov, schur  # noqa: E402

SAMPLES = 2048
SAMPLE_SEED = 3003
OUT = os.path.join(ROOT, "tests", "golden", "c3_oracle_solution.txt")


def main():
    s = si.make_system("c3")
    K = bsr.from_arrays(s.indptr, s.indices, s.data, 4)
    Ks = K.scipy().tocsr()
    t0 = time.perf_counter()
    pc = schur.build(K, 3)
    t1 = time.perf_counter()
    x, info = krylov.gmres(lambda v: Ks @ v, pc.apply, s.b, m=30, tol=1e-8)
    t2 = time.perf_counter()
    res = float(np.linalg.norm(s.b - Ks @ x) / np.linalg.norm(s.b))
    idx = np.sort(np.random.Generator(np.random.PCG64(SAMPLE_SEED)).choice(
        s.n, size=SAMPLES, replace=False))
    with open(OUT, "w") as fh:
        fh.write("# FP64 oracle solve of the N=128 Schur system (GMRES(30), tol 1e-8),\n")
        fh.write("# written by tests/golden/make_c3_oracle.py (oracle setup %.0f s, solve %.0f s\n"
                 % (t1 - t0, t2 - t1))
        fh.write("# on the machine that ran it; timings are not used by any test)\n")
        fh.write("n: %d\n" % s.n)
        fh.write("iterations: %d\n" % info.iters)
        fh.write("true_rel_res: %.17g\n" % res)
        fh.write("x_norm: %.17g\n" % float(np.linalg.norm(x)))
        fh.write("sample_idx: %s\n" % " ".join(str(int(i)) for i in idx))
        fh.write("sample_x: %s\n" % " ".join("%.17g" % v for v in x[idx]))
    print("iterations %d, true rel. residual %.3e, ||x|| %.6g -> %s"
          % (info.iters, res, np.linalg.norm(x), OUT))


if __name__ == "__main__":
    main()
