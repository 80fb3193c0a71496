"""Parity at the full size of the headline workload, in the launch configuration bench.py times: 256^3,
sixth order, the 20-bump medium of seeds 3/4 (~10 points per wavelength), TF32 EigT, FGMRES(30), rtol
1e-6.  The FP64 oracle is evaluated on the whole field (each evaluation takes seconds on the host cores):
the matvec element by element, the preconditioner in the GPU's own eigenbasis within the TF32 bound, the
right-hand side, and the FP64 residual of the GPU's solution.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle.eigt import EigT
from oracle.grid import Grid
from oracle.operators import Operator, derived_k2_fields
from oracle.rhs import rhs6_sampled
from paper_2602_07711_gb300 import HELM_PREC_TF32, Solver, media

N = 256


@pytest.fixture(scope="module")
def case():
    k2, f, k0 = media.bumps(N, 3, 4)
    S = Solver((N, N, N), k2, k0, order=6, precision=HELM_PREC_TF32, flexible=True, rtol=1e-6, restart=30,
               max_iter=300)
    g = Grid(N, N, N, staggered=True)
    A = Operator(g, k2, k0, 6)
    yield {"k2": k2, "f": f, "k0": k0, "S": S, "g": g, "A": A}
    S.close()


def _rand(shape, seed):
    r = np.random.default_rng(seed)
    return (r.standard_normal(shape) + 1j * r.standard_normal(shape)).astype(np.complex64)


def test_apply_A_full_size(case):
    S, A, g = case["S"], case["A"], case["g"]
    u = _rand(g.shape, 31)
    w = S.apply_A(torch.from_numpy(u).cuda()).cpu().numpy()
    ref = A(u.astype(np.complex128)).reshape(g.shape)
    # complex64 rounding of ~30 terms with cancellation, as at the small sizes
    assert np.abs(w - ref).max() / np.abs(ref).max() < 2e-6
    assert np.linalg.norm(w - ref) / np.linalg.norm(ref) < 1e-6


def test_precond_full_size(case):
    S, g, k0 = case["S"], case["g"], case["k0"]
    e = EigT(g, k0)
    e.Dx, e.Vx, e.Vxi = S.get_eig(0)
    e.Dy, e.Vy, e.Vyi = S.get_eig(1)
    kap = np.linalg.cond(e.Vx) * np.linalg.cond(e.Vy)
    y = _rand(g.shape, 32)
    z = S.apply_precond(torch.from_numpy(y).cuda()).cpu().numpy()
    ref = e.apply_Minv(y.astype(np.complex128)).reshape(g.shape)
    assert np.linalg.norm(z - ref) / np.linalg.norm(ref) < 2e-3 * kap


def test_rhs_and_solution_full_size(case):
    S, A, g = case["S"], case["A"], case["g"]
    k2, f = case["k2"], case["f"]
    F = S.build_rhs(torch.from_numpy(f).cuda())
    Fh = F.cpu().numpy()
    dk2, _ = derived_k2_fields(k2, True, g.h)
    ref = rhs6_sampled(f, k2, dk2, True, g.h).reshape(g.shape)
    assert np.abs(Fh - ref).max() / np.abs(ref).max() < 1e-10
    x, info = S.solve(F)
    assert info.status == 0 and info.relres_true <= 1e-6
    xg = x.cpu().numpy()
    # the FP64 residual of the GPU's solution, evaluated by the oracle on the whole field
    assert np.linalg.norm(A(xg).reshape(-1) - Fh.reshape(-1)) / np.linalg.norm(Fh) <= 1.5e-6
