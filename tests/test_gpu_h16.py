"""The 16-bit transform chains (HELM_PREC_BF16, HELM_PREC_FP16) against the CPU oracle, through the C-ABI.

Every operand of the x- and y-pass MMAs is a 16-bit value and the grids between the passes are stored in
16 bits (the z-solve reads and writes them and computes in FP32).  BF16 keeps an 8-bit significand (round
to nearest even: relative error up to 2^-9), FP16 TF32's 11 bits (up to 2^-11) inside power-of-two stage
scales that rule out overflow (operator bounds from set-up times the norms the passes measure).  The chain carries about six such roundings
where the TF32 chain carries four TF32 truncations (up to 2^-10 each).  The bounds are fixed, at about 2.5x
the errors measured on a GB300 (recorded beside them); a transposed basis or one shifted by a column gives
relative errors near 1.4.
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
from paper_2602_07711_gb300 import HELM_PREC_BF16, HELM_PREC_FP16, HelmError, Solver, helm, media, solve_batched

# relative error bounds (2-norm, max-norm) of the whole preconditioner.  Measured, BF16: 6.0e-3 / 7.2e-3 at
# 32^3, 6.6e-3 / 6.7e-3 at 48 x 40 x 36, 6.5e-3 / 8.8e-3 at 64^3, 7.8e-3 / 1.0e-2 at 128 x 128 x 20, 1.03e-2 /
# 1.58e-2 at 256 x 256 x 8; FP16: 7.3e-4 / 6.8e-4, 8.0e-4 / 8.4e-4, 8.4e-4 / 1.05e-3, 9.7e-4 / 1.32e-3,
# 1.27e-3 / 1.72e-3 (TF32: 1.5e-3 ... 1.8e-3 / 1.6e-3 ... 2.0e-3).
BOUNDS = {HELM_PREC_BF16: (2.6e-2, 4e-2), HELM_PREC_FP16: (3.2e-3, 4.3e-3)}


def _dev(a, dtype=torch.complex64):
    return torch.from_numpy(np.ascontiguousarray(a)).to(device="cuda", dtype=dtype)


def _rand(shape, seed):
    r = np.random.default_rng(seed)
    return r.standard_normal(shape) + 1j * r.standard_normal(shape)


def _errs(a, b):
    a = np.asarray(a, np.complex128)
    b = np.asarray(b, np.complex128)
    return (np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()), np.abs(a - b).max() / np.abs(b).max())


@pytest.mark.parametrize("prec", [HELM_PREC_BF16, HELM_PREC_FP16])
@pytest.mark.parametrize("n", [(32, 32, 32), (48, 40, 36), (64, 64, 64), (128, 128, 20), (256, 256, 8)])
def test_h16_preconditioner_matches_oracle(n, prec):
    g = Grid(*n, staggered=True)
    k0 = 2 * math.pi / (10 * g.h[0])
    k2 = np.full(g.shape, k0 * k0, complex)
    S = Solver(n, k2, k0, order=4, precision=prec, flexible=True)
    e = EigT(g, k0)
    e.Dx, e.Vx, e.Vxi = S.get_eig(0)
    e.Dy, e.Vy, e.Vyi = S.get_eig(1)
    y = _rand(g.shape, 5)
    ref = e.apply_Minv(y).reshape(g.shape)
    z = S.apply_precond(_dev(y)).cpu().numpy()
    e2, emax = _errs(z, ref)
    print("h16 preconditioner", prec, n, e2, emax)
    assert e2 < BOUNDS[prec][0] and emax < BOUNDS[prec][1], (e2, emax)
    # scale invariance over a wide range (FP16 normalises by ||r|| when no Arnoldi scale is given): a power
    # of two leaves every rounding unchanged
    for p2 in (2.0 ** 60, 2.0 ** -60):
        z2 = S.apply_precond(_dev(p2 * y)).cpu().numpy()
        assert _errs(z2, p2 * z.astype(np.complex128))[0] < 1e-6
    # r may alias z
    yy = _dev(y)
    helm.helm_apply_precond(S.ctx, yy, yy)
    assert np.array_equal(yy.cpu().numpy(), z)
    S.close()


@pytest.mark.parametrize("prec", [HELM_PREC_BF16, HELM_PREC_FP16])
def test_h16_fgmres_solution_matches_oracle(prec):
    n = 48
    k2, f, k0 = media.bumps(n, 11, 12)
    S = Solver((n, n, n), k2, k0, order=6, precision=prec, flexible=True, rtol=1e-6, restart=30, max_iter=200)
    F = S.build_rhs(torch.from_numpy(f).cuda())
    x, info = S.solve(F)
    g = Grid(n, n, n, staggered=True)
    A = Operator(g, k2, k0, 6)
    e = EigT(g, k0)
    Fh = F.cpu().numpy()
    xo, _ = gmres(A, e.apply_Minv, Fh, m=30, rtol=1e-12, max_it=400)
    xo = xo.reshape(g.shape)
    xg = x.cpu().numpy()
    S.close()
    assert info.status == 0 and info.relres_true <= 1e-6
    assert np.linalg.norm(A(xg) - Fh) / np.linalg.norm(Fh) <= 1.5e-6
    assert np.linalg.norm(xg - xo) / np.linalg.norm(xo) <= 1e-5


@pytest.mark.parametrize("prec", [HELM_PREC_BF16, HELM_PREC_FP16])
def test_h16_limits(prec):
    # N_x must be a multiple of 4 (16-byte rows of 16-bit pairs for the TMA copies)
    n = (42, 40, 20)
    g = Grid(*n, staggered=True)
    k0 = 2 * math.pi / (10 * g.h[0])
    with pytest.raises(HelmError):
        Solver(n, np.full(g.shape, k0 * k0, complex), k0, order=4, precision=prec)
    # batched solves with a 16-bit chain must be flexible (the chain runs in the group iterations only)
    n = 32
    k2, f, k0 = media.single_gaussian(n)
    S = Solver((n, n, n), k2, k0, order=4, precision=prec, flexible=False)
    B = torch.from_numpy(np.stack([f, f])).cuda()
    with pytest.raises(HelmError):
        solve_batched([S], [B])
    S.close()
    # the FP16 stage bounds assume a constant k0 along z
    kz = np.full(n, k0 * k0)
    kz[n // 2:] *= 1.1
    if prec == HELM_PREC_FP16:
        with pytest.raises(HelmError):
            Solver((n, n, n), k2, k0, order=4, precision=prec, flexible=True, k0z2=kz)
    else:
        Solver((n, n, n), k2, k0, order=4, precision=prec, flexible=True, k0z2=kz).close()


@pytest.mark.parametrize("prec", [HELM_PREC_BF16, HELM_PREC_FP16])
def test_h16_batched_matches_single_solves(prec):
    """Two problems (a 48^3 and a 160^3 bump medium, two right-hand sides each; the 160^3 lanes form a group
    whose chain runs over both vectors at once) in one batched call with the 16-bit chain: every lane
    converges to rtol and matches its single solve (the group's chain scales by the group's norms, so the
    roundings differ from a single solve's)."""
    solvers, bs, singles = [], [], []
    for n, nr, seed in ((48, 2, 21), (160, 2, 23)):
        k2, f, k0 = media.bumps(n, seed, seed + 1)
        S = Solver((n, n, n), k2, k0, order=6, precision=prec, flexible=True, rtol=1e-6, restart=30, max_iter=200)
        F = S.build_rhs(torch.from_numpy(f).cuda())
        rng = np.random.default_rng(seed)
        B = torch.stack([F * complex(np.exp(2j * np.pi * rng.uniform())) * (1 + r) for r in range(nr)]).contiguous()
        solvers.append(S)
        bs.append(B)
        singles.append([S.solve(B[r].contiguous()) for r in range(nr)])
    nrhs = min(b.shape[0] for b in bs)
    bs = [b[:nrhs].contiguous() for b in bs]
    xs, infos = solve_batched(solvers, bs)
    for p, S in enumerate(solvers):
        for r in range(nrhs):
            x1, i1 = singles[p][r]
            assert infos[p][r].status == 0 and infos[p][r].relres_true <= 1e-6
            assert abs(infos[p][r].iterations - i1.iterations) <= 1
            d = (xs[p][r] - x1).abs().max().item() / x1.abs().max().item()
            assert d < 1e-5, (p, r, d)
        S.close()
