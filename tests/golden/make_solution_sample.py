"""Write the oracle's solution of the 256^3 headline problem at seeded sample points.

Problem: the sixth-order scheme (Eq. scheme6) on the staggered 256^3 grid of the unit cube (Sec. 5.2
grid), the 20-bump medium media.bumps(256, 3, 4) (~10 points per wavelength), its modified right-hand
side from the sampled f, solved by the oracle's right-preconditioned GMRES(30) with EigT (Sec. 4.1) to
rel-res 1e-12.  The solve took 1306 s (about 22 minutes) on eight host cores and 12 GB of memory, so the test suite
reads its result from the text file this script writes instead of running it:

    python tests/golden/make_solution_sample.py            # writes bumps256_order6_solution_sample.txt

Output: a header with the oracle's iteration count, its FP64 rel-res, the 2-norm of the whole solution and
the sample seed, then one line per sample point `flat_index re im` (4096 points drawn without replacement
by numpy.random.default_rng(256), sorted).  Only oracle/ and the seeded input generator are used.
"""
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

N, SEED_MEDIUM, SEED_ANGLE, SAMPLES, SAMPLE_SEED = 256, 3, 4, 4096, 256
OUT = os.path.join(HERE, "bumps256_order6_solution_sample.txt")


def main(n=N, out=OUT):
    from oracle.eigt import EigT
    from oracle.gmres import gmres
    from oracle.grid import Grid
    from oracle.operators import Operator
    from oracle.rhs import rhs6_sampled
    from paper_2602_07711_gb300 import media

    k2, f, k0 = media.bumps(n, SEED_MEDIUM, SEED_ANGLE)
    g = Grid(n, n, n, staggered=True)
    A = Operator(g, k2, k0, 6)
    F = rhs6_sampled(f, k2, A.dk2, True, g.h)
    t = time.time()
    hist = []
    x, info = gmres(A, EigT(g, k0).apply_Minv, F, m=30, rtol=1e-12, max_it=400, history=hist)
    dt = time.time() - t
    relres = float(np.linalg.norm(np.asarray(A(x)).ravel() - F.ravel()) / np.linalg.norm(F))
    idx = np.sort(np.random.default_rng(SAMPLE_SEED).choice(n ** 3, SAMPLES, replace=False))
    xs = x.ravel()[idx]
    with open(out, "w") as fh:
        fh.write("# oracle solution of media.bumps(%d, 3, 4), sixth order, staggered grid, GMRES(30)+EigT to "
                 "rel-res 1e-12 (tests/golden/make_solution_sample.py)\n" % n)
        fh.write("# iterations %d relres %.6e norm2 %.17e sample_seed %d solve_seconds %.0f\n"
                 % (info["iterations"], relres, np.linalg.norm(x), SAMPLE_SEED, dt))
        for i, v in zip(idx, xs):
            fh.write("%d %.17e %.17e\n" % (i, v.real, v.imag))
    print("wrote", out, info["iterations"], relres, dt)


def read(path=OUT):
    """(header dict, flat indices, complex values) of a sample file."""
    with open(path) as fh:
        lines = fh.read().splitlines()
    head = lines[1].lstrip("# ").split()
    meta = {head[i]: float(head[i + 1]) for i in range(0, len(head), 2)}
    rows = np.array([[float(v) for v in ln.split()] for ln in lines[2:] if ln.strip()])
    return meta, rows[:, 0].astype(np.int64), rows[:, 1] + 1j * rows[:, 2]


if __name__ == "__main__":
    # optional: a smaller grid and another output file (a quick check of the script itself)
    if len(sys.argv) == 3:
        main(int(sys.argv[1]), sys.argv[2])
    else:
        main()
