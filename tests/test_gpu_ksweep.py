"""The wavenumber sweep of Sec. 5.1 (Table tab:diff_k_results) on the GPU path: the manufactured test problem
(collocated grid, high-order closure, sixth order) for k0 = k in {10, 20, 50} on the 100^3 grid,
preconditioned by EigT3 (which inverts the same second-order operator as the paper's PFFT3; the oracle pins
PFFT = EigT), FGMRES(20) with TF32 transforms to rel-res 1e-10, against the oracle's FP64 GMRES(20) on the
same three systems.

Checked: the GPU reaches the oracle's solution of every system (and so its discretisation error against the
exact solution, which grows with k h as the sixth-order truncation says); the table's trend, N0 growing with
k on a fixed grid, holds for the FP64 Krylov process.  The GPU's own iteration counts do not follow that
trend: every complex64 restart cycle lowers the double-float true residual by 1e-3 to 1e-4 only, the less
the smaller k h is (the stencil's 1/h^2 terms cancel down to ~k^2, which costs complex64 digits), so the
small wavenumbers need more cycles to reach 1e-10 (14, 12, 15 iterations for k = 10, 20, 50 measured).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu, pytest.mark.slow]

from oracle import manufactured as mf
from oracle.closure import pad_ghost_ho
from oracle.eigt import EigT
from oracle.gmres import gmres
from oracle.grid import Grid
from oracle.operators import Operator
from oracle.rhs import rhs6
from paper_2602_07711_gb300 import HELM_CLOSURE_HIGH_ORDER, HELM_PREC_TF32, Solver, media

N, KS = 100, (10, 20, 50)


def _gpu(n, k):
    d = media.manufactured(n, float(k), 6)
    S = Solver((n, n, n), d["k2"], float(k), order=6, precision=HELM_PREC_TF32, flexible=True, restart=20,
               max_iter=400, rtol=1e-10, staggered=False)
    S.set_closure(HELM_CLOSURE_HIGH_ORDER)
    F = S.closure_rhs(torch.from_numpy(d["faces"]).cuda(), S.build_rhs_fields(torch.from_numpy(d["fields"]).cuda()))
    x, info = S.solve(F)
    assert info.status == 0 and info.relres_true <= 1e-10
    S.close()
    return info, x.cpu().numpy(), d["u"]


def _oracle_system(n, k):
    g = Grid(n, n, n, staggered=False)
    X, Y, Z = g.mesh()
    zero = (np.zeros(g.shape, complex),) * 3
    op = Operator(g, np.full(g.shape, k * k, dtype=complex), k, 6, rule="collocated_ho", dk2=zero,
                  lapk2=np.zeros(g.shape, complex))
    fdiff = lambda X, Y, Z, dd: mf.f_exact(X, Y, Z, k, *dd)
    ghost_f = pad_ghost_ho(np.zeros(g.shape, complex), k, g.h, fdiff=fdiff)
    f, lapf, sum4, mix, df = mf.rhs6_fields(X, Y, Z, k)
    b = (rhs6(f, lapf, sum4, mix, df, np.full(g.shape, k * k, dtype=complex), zero, g.h)
         - op.apply_padded(ghost_f)).ravel()
    return op, EigT(g, k).apply_Minv, b


def test_wavenumber_sweep_on_the_gpu():
    its, errs = [], []
    for k in KS:
        info, xg, u = _gpu(N, k)
        op, M, b = _oracle_system(N, k)
        xo, io = gmres(op, M, b, m=20, rtol=1e-10, max_it=400)
        assert io["converged"]
        its.append(io["iterations"])
        xo = xo.reshape(xg.shape)
        # the GPU's solution is the oracle's (both at rel-res 1e-10)
        assert np.linalg.norm(xg - xo) / np.linalg.norm(xo) <= 1e-7, k
        errs.append(np.linalg.norm(xg - u) / np.linalg.norm(u))
    # the table's trend, on the FP64 Krylov process: N0 grows with the wavenumber
    assert its == sorted(its) and its[0] < its[-1], its
    # sixth-order accuracy degrades with k h on a fixed grid
    assert errs == sorted(errs) and errs[-1] < 1e-3, errs
