"""The 128^3 configuration of the mixed-precision path against the FP64 oracle, element by element: sixth
order (Eq. scheme6), the seeded 20-bump medium (seeds 1/2, ~10 points per wavelength), TF32 eigenvector
transforms with FP32 accumulation, complex64 stencil and Krylov vectors, FP64 Givens, double-float true
residual, flexible GMRES(30) to rel-res 1e-6.  The oracle (complex128, right-preconditioned GMRES(30) with
EigT, Sec. 4.1) solves the same right-hand side to rel-res 1e-12, which takes about half a minute on the
host cores.  Measured on a GB300: 13 inner iterations, relative solution error 4.2e-7 (2-norm) and 5.3e-7
(max-norm) against the 1e-5 target.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu, pytest.mark.slow]

from oracle.eigt import EigT
from oracle.gmres import gmres
from oracle.grid import Grid
from oracle.operators import Operator
from paper_2602_07711_gb300 import HELM_PREC_TF32, Solver, media


def test_config2_solution_matches_oracle_element_by_element():
    n = 128
    k2, f, k0 = media.bumps(n, 1, 2)
    S = Solver((n, n, n), k2, k0, order=6, precision=HELM_PREC_TF32, flexible=True, rtol=1e-6, restart=30,
               max_iter=300)
    F = S.build_rhs(torch.from_numpy(f).cuda())
    x, info = S.solve(F)
    assert info.status == 0 and info.relres_true <= 1e-6
    g = Grid(n, n, n, staggered=True)
    A = Operator(g, k2, k0, 6)
    Fh = F.cpu().numpy()
    xo, io = gmres(A, EigT(g, k0).apply_Minv, Fh, m=30, rtol=1e-12, max_it=600)
    assert io["relres"] <= 1e-11
    xg = x.cpu().numpy().ravel()
    assert np.linalg.norm(xg - xo) / np.linalg.norm(xo) <= 1e-5
    assert np.abs(xg - xo).max() / np.abs(xo).max() <= 1e-5
    # the GPU's own FP64-accurate residual agrees with the oracle's evaluation of it
    relres = np.linalg.norm(A(xg).ravel() - Fh.ravel()) / np.linalg.norm(Fh)
    assert abs(relres - info.relres_true) <= 1e-3 * relres
    S.close()
