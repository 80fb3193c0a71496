"""Tensor-core (tcgen05, TF32) eigenvector transforms against the CPU oracle, through the C-ABI.

TF32 keeps 10 explicit mantissa bits (the weights are rounded to nearest, the streamed grid values are
truncated by the tensor core), so each product carries a relative error of about 2^-11 and the FP32
accumulation adds little.  The measured relative errors on random complex inputs do not grow with N or with
the conditioning of the bases: 8.0e-4 ... 8.4e-4 (2-norm) and 7.5e-4 ... 9.6e-4 (max-norm) for one
transform, 1.5e-3 ... 1.8e-3 and 1.6e-3 ... 2.0e-3 for the whole preconditioner, from 32^3 to 256 x 256 x 8.
The bounds below are fixed, about 2.5x those measurements; a transposed basis or one shifted by a column
gives relative errors near 1.4 (tests/test_oracle_pins.py plants both in the oracle at 256 x 256 x 8).
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
from paper_2602_07711_gb300 import HELM_PREC_FP32, HELM_PREC_TF32, HELM_PREC_TF32X3, HELM_PRECOND_PFFT, Solver, media
from oracle.pfft import PFFT


# relative error bounds of one TF32 transform (forward or inverse) and of the whole preconditioner
TF32_PASS_2, TF32_PASS_MAX = 2e-3, 2.5e-3
TF32_PRECOND_2, TF32_PRECOND_MAX = 4e-3, 5e-3
# the three-product split (3xTF32): FP32-level transforms, whose error grows with the contraction length like
# FP32 accumulation does; per size about 3x the measured relative errors (pass 2-norm / max-norm, whole
# preconditioner 2-norm / max-norm): 32^3 6.6e-7 / 8.9e-7, 3.1e-6 / 2.7e-6; 48 x 40 x 36 9.8e-7 / 1.2e-6,
# 3.7e-6 / 3.5e-6; 128 x 128 x 20 2.8e-6 / 2.8e-6, 1.3e-5 / 1.3e-5; 256 x 256 x 8 5.7e-6 / 6.5e-6,
# 1.7e-5 / 2.1e-5 (TF32 alone: 8e-4 at every size)
X3_BOUNDS = {(32, 32, 32): (2e-6, 2.7e-6, 9.5e-6, 8.5e-6), (48, 40, 36): (3e-6, 3.6e-6, 1.1e-5, 1.1e-5),
             (128, 128, 20): (8.5e-6, 8.5e-6, 4e-5, 4e-5), (256, 256, 8): (1.7e-5, 2e-5, 5.2e-5, 6.4e-5)}


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
    y = _rand(g.shape, 5)
    fwd = S.precond_step(1, _dev(y)).cpu().numpy()
    e2, emax = _errs(fwd, e.forward(y))
    assert e2 < TF32_PASS_2 and emax < TF32_PASS_MAX, (e2, emax)
    inv = S.precond_step(3, _dev(y)).cpu().numpy()
    e2, emax = _errs(inv, e.inverse(y))
    assert e2 < TF32_PASS_2 and emax < TF32_PASS_MAX, (e2, emax)
    z = S.apply_precond(_dev(y)).cpu().numpy()
    e2, emax = _errs(z, e.apply_Minv(y))
    assert e2 < TF32_PRECOND_2 and emax < TF32_PRECOND_MAX, (e2, emax)


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


@pytest.mark.parametrize("n", list(X3_BOUNDS))
def test_split_tf32_transforms_match_oracle(n):
    """HELM_PREC_TF32X3: hi hi + hi lo + lo hi products of TF32 halves on the tensor cores, as accurate as
    FP32 transforms (the remainders carry the 13 bits TF32 drops)."""
    g = Grid(*n, staggered=True)
    k0 = 2 * math.pi / (10 * g.h[0])
    S = Solver(n, np.full(g.shape, k0 * k0, complex), k0, order=4, precision=HELM_PREC_TF32X3, flexible=True)
    e = EigT(g, k0)
    e.Dx, e.Vx, e.Vxi = S.get_eig(0)
    e.Dy, e.Vy, e.Vyi = S.get_eig(1)
    p2, pmax, q2, qmax = X3_BOUNDS[n]
    y = _rand(g.shape, 5)
    e2, emax = _errs(S.precond_step(1, _dev(y)).cpu().numpy(), e.forward(y))
    assert e2 < p2 and emax < pmax, (e2, emax)
    e2, emax = _errs(S.precond_step(3, _dev(y)).cpu().numpy(), e.inverse(y))
    assert e2 < p2 and emax < pmax, (e2, emax)
    e2, emax = _errs(S.apply_precond(_dev(y)).cpu().numpy(), e.apply_Minv(y))
    assert e2 < q2 and emax < qmax, (e2, emax)


def test_split_tf32_pfft_matches_oracle():
    n, L = (64, 32, 20), (1.0, 0.5, 0.3125)
    g = Grid(*n, lx=L[0], ly=L[1], lz=L[2], staggered=True)
    k0 = 2 * math.pi / (10 * g.h[0])
    S = Solver(n, np.full(g.shape, k0 * k0, complex), k0, order=4, L=L, precond=HELM_PRECOND_PFFT,
               precision=HELM_PREC_TF32X3, flexible=True)
    y = _rand(g.shape, 8)
    z = S.apply_precond(_dev(y)).cpu().numpy()
    ref = PFFT(g, k0, variant="face").apply_Minv(y)
    assert np.linalg.norm(z - ref) / np.linalg.norm(ref) < 1e-4


def test_split_tf32_fgmres_matches_oracle_and_fp32():
    n = 64
    k2, f, k0 = media.bumps(n, 21, 22)
    Fd = torch.from_numpy(f).cuda()
    out = {}
    for prec in (HELM_PREC_FP32, HELM_PREC_TF32X3):
        S = Solver((n, n, n), k2, k0, order=6, precision=prec, flexible=True, rtol=1e-6)
        x, info = S.solve(S.build_rhs(Fd))
        assert info.status == 0 and info.relres_true <= 1e-6
        out[prec] = (x.cpu().numpy(), info.iterations)
    d = np.linalg.norm(out[HELM_PREC_FP32][0] - out[HELM_PREC_TF32X3][0]) / np.linalg.norm(out[HELM_PREC_FP32][0])
    assert d < 2e-5
    assert abs(out[HELM_PREC_FP32][1] - out[HELM_PREC_TF32X3][1]) <= 1
