"""Tensor-core (tcgen05, TF32) eigenvector transforms against the CPU oracle, through the C-ABI.

TF32 keeps 10 explicit mantissa bits (the weights are rounded to nearest, the streamed grid values are
truncated by the tensor core), so each product carries a relative error below 2^-10 and the FP32
accumulation over K = N terms grows it like sqrt(K) in the mean.  Bounds used below (relative):
2-norm error <= 2e-3 * kappa, max-norm error <= 1e-2 * kappa, kappa = cond(V_x) cond(V_y) of the basis.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle.eigt import EigT
from oracle.gmres import gmres
from oracle.grid import Grid
from oracle.operators import Operator
from paper_2602_07711_gb300 import HELM_PREC_FP32, HELM_PREC_TF32, Solver, media


def _dev(a, dtype=torch.complex64):
    return torch.from_numpy(np.ascontiguousarray(a)).to(device="cuda", dtype=dtype)


def _rand(shape, seed):
    r = np.random.default_rng(seed)
    return r.standard_normal(shape) + 1j * r.standard_normal(shape)


def _errs(a, b):
    return (np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()), np.abs(a - b).max() / np.abs(b).max())


@pytest.mark.parametrize("n", [(32, 32, 32), (48, 40, 36), (64, 64, 64), (128, 128, 20), (256, 256, 8)])
def test_tf32_transforms_match_oracle(n):
    g = Grid(*n, staggered=True)
    k0 = 2 * math.pi / (10 * g.h[0])
    k2 = np.full(g.shape, k0 * k0, complex)
    S = Solver(n, k2, k0, order=4, precision=HELM_PREC_TF32, flexible=True)
    e = EigT(g, k0)
    e.Dx, e.Vx, e.Vxi = S.get_eig(0)
    e.Dy, e.Vy, e.Vyi = S.get_eig(1)
    kap = np.linalg.cond(e.Vx) * np.linalg.cond(e.Vy)
    y = _rand(g.shape, 5)
    fwd = S.precond_step(1, _dev(y)).cpu().numpy()
    e2, emax = _errs(fwd, e.forward(y))
    assert e2 < 2e-3 * kap and emax < 1e-2 * kap, (e2, emax, kap)
    inv = S.precond_step(3, _dev(y)).cpu().numpy()
    e2, emax = _errs(inv, e.inverse(y))
    assert e2 < 2e-3 * kap and emax < 1e-2 * kap, (e2, emax, kap)
    z = S.apply_precond(_dev(y)).cpu().numpy()
    e2, emax = _errs(z, e.apply_Minv(y))
    assert e2 < 2e-3 * kap, (e2, kap)


def test_tf32_fgmres_solution_matches_oracle():
    n = 32
    k2, f, k0 = media.single_gaussian(n)
    S = Solver((n, n, n), k2, k0, order=4, precision=HELM_PREC_TF32, flexible=True, rtol=1e-6)
    F = S.build_rhs(torch.from_numpy(f).cuda())
    x, info = S.solve(F)
    g = Grid(n, n, n, staggered=True)
    A = Operator(g, k2, k0, 4)
    Fh = F.cpu().numpy()
    xo, _ = gmres(A, EigT(g, k0).apply_Minv, Fh, m=30, rtol=1e-12, max_it=400)
    xg = x.cpu().numpy().ravel()
    assert info.status == 0 and info.relres_true <= 1e-6
    assert np.linalg.norm(A(xg) - Fh) / np.linalg.norm(Fh) <= 1.5e-6
    assert np.linalg.norm(xg - xo) / np.linalg.norm(xo) <= 1e-5


def test_tf32_and_fp32_paths_agree_on_order6_bumps():
    n = 64
    k2, f, k0 = media.bumps(n, 21, 22)
    Fd = torch.from_numpy(f).cuda()
    out = {}
    for prec in (HELM_PREC_FP32, HELM_PREC_TF32):
        S = Solver((n, n, n), k2, k0, order=6, precision=prec, flexible=True, rtol=1e-6)
        x, info = S.solve(S.build_rhs(Fd))
        assert info.status == 0 and info.relres_true <= 1e-6
        out[prec] = (x.cpu().numpy(), info.iterations)
    d = np.linalg.norm(out[0][0] - out[1][0]) / np.linalg.norm(out[0][0])
    assert d < 2e-5
    assert abs(out[0][1] - out[1][1]) <= 3
