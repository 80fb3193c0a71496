"""Parity of the CUDA path (through the C-ABI) with the complex128 CPU oracle, element by element.

Tolerances (relative, max-norm over the output unless stated):
  complex128 kernels (apply_A FP64, eigensetup)                 1e-11
  double-float kernels (build_rhs; ~44-bit arithmetic)          1e-10
  complex64 stencil                                            2e-6   (FP32 rounding of ~27 terms)
  complex64 EigT transforms (FP32)                             1.5e-6
  complex64 z-solve / preconditioner (FP32)                     per case, about 3x the measured error
                                                               (long z-lines amplify rounding: 300 planes
                                                               measured 6.5e-5 against 2.9e-6 at 33)
  GMRES solution at rtol 1e-6 vs oracle solved to 1e-12         1e-5 in the relative 2-norm (the accuracy target)
Sizes span several tiles plus ragged tails (x not a multiple of 32, y not of 8, z not of 32).
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle.eigt import EigT
from oracle.gmres import gmres
from oracle.grid import Grid
from oracle.operators import Operator, derived_k2_fields
from oracle.rhs import rhs4_sampled, rhs6_sampled
from oracle.tridiag import thomas
from paper_2602_07711_gb300 import HELM_PREC_FP32, Solver, media


def _dev(a, dtype=torch.complex128):
    return torch.from_numpy(np.ascontiguousarray(a)).to(device="cuda", dtype=dtype)


def _rel(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    return np.abs(a - b).max() / np.abs(b).max()


def _rand(shape, seed):
    r = np.random.default_rng(seed)
    return r.standard_normal(shape) + 1j * r.standard_normal(shape)


def _medium(n, L, seed=0):
    """Smooth variable k^2 on a staggered grid of n = (nx, ny, nz) over lengths L, k0 ~ 10 ppw."""
    g = Grid(*n, lx=L[0], ly=L[1], lz=L[2], staggered=True)
    X, Y, Z = g.mesh()
    k0 = 2 * math.pi / (10 * g.h[0])
    k2 = k0 * k0 * (1 + 0.25 * np.exp(-((X - .5 * L[0]) ** 2 + (Y - .45 * L[1]) ** 2 + (Z - .55 * L[2]) ** 2) / 0.03)
                    - 0.1 * np.exp(-((X - .3 * L[0]) ** 2 + (Y - .6 * L[1]) ** 2 + (Z - .4 * L[2]) ** 2) / 0.01)) + 0j
    k2 = k2 + 1j * 0.01 * k0 * k0 * np.sin(3 * X)     # complex-valued k (Eq. problem)
    return g, k2, k0


SIZES = {
    2: [((40, 36, 33), (1.0, 0.9, 0.85))],
    4: [((40, 36, 33), (1.0, 0.9, 0.85)), ((32, 32, 32), (1.0, 1.0, 1.0)), ((66, 10, 70), (1.0, 0.2, 0.9))],
    6: [((40, 36, 33), (40 / 40, 36 / 40, 33 / 40)), ((32, 32, 32), (1.0, 1.0, 1.0)),
        ((70, 18, 66), (70 / 70, 18 / 70, 66 / 70))],
}


@pytest.mark.parametrize("order,case", [(o, c) for o in (2, 4, 6) for c in SIZES[o]])
def test_apply_A_matches_oracle(order, case):
    n, L = case
    g, k2, k0 = _medium(n, L)
    S = Solver(n, k2, k0, order=order, L=L)
    x = _rand(g.shape, 1)
    ref = Operator(g, k2, k0, order)(x)
    y128 = S.apply_A(_dev(x)).cpu().numpy()
    assert _rel(y128, ref) < 1e-11
    y64 = S.apply_A(_dev(x, torch.complex64)).cpu().numpy()
    assert _rel(y64, ref) < 2e-6


@pytest.mark.parametrize("order", [4, 6])
@pytest.mark.parametrize("real", [False, True])
def test_every_matvec_variant_matches_oracle(order, real):
    """helm_set_matvec_variant 0-4 (cp.async at four or three CTAs per SM, TMA ring, two outputs per thread,
    two outputs with the order-6 fields formed in the kernel) on a complex and on a real medium (the real
    forms stage k^2 as float; on a complex medium variants 3 and 4 fall back), at two ragged sizes."""
    for n, L in (((40, 36, 33), (1.0, 0.9, 0.825)), ((70, 18, 66), (70 / 70, 18 / 70, 66 / 70))):
        g, k2, k0 = _medium(n, L)
        if real:
            k2 = k2.real + 0j
        S = Solver(n, k2, k0, order=order, L=L)
        x = _rand(g.shape, 3)
        ref = Operator(g, k2, k0, order)(x)
        for v in range(5):
            S.set_matvec_variant(v)
            y64 = S.apply_A(_dev(x, torch.complex64)).cpu().numpy()
            assert _rel(y64, ref) < 2e-6, (n, v)
        with pytest.raises(Exception):
            S.set_matvec_variant(5)
        S.close()


@pytest.mark.parametrize("order", [4, 6])
@pytest.mark.parametrize("real", [False, True])
def test_build_rhs_matches_oracle(order, real):
    """On a real medium the sixth-order right-hand side takes its real form (k^2 from the residual's
    real field, real gradients)."""
    n, L = (40, 36, 33), (1.0, 0.9, 0.825)
    g, k2, k0 = _medium(n, L)
    if real:
        k2 = k2.real + 0j
    f = _rand(g.shape, 2)
    S = Solver(n, k2, k0, order=order, L=L)
    F = S.build_rhs(_dev(f)).cpu().numpy()
    if order == 4:
        ref = rhs4_sampled(f, True, g.h)
    else:
        dk2, _ = derived_k2_fields(k2, True, g.h)
        ref = rhs6_sampled(f, k2, dk2, True, g.h)
    assert _rel(F, ref) < 1e-10
    F2 = S.build_rhs(f).cpu().numpy()          # host input
    assert _rel(F2, ref) < 1e-10


@pytest.mark.parametrize("n", [4, 5, 17, 32, 33, 64, 127, 256, 512])
def test_eigensetup_diagonalises_lambda_bar(n):
    g = Grid(n, 8, 8, staggered=True)
    k0 = 2 * math.pi / (10 * g.h[0])
    S = Solver((n, 8, 8), np.full(g.shape, k0 * k0, complex), k0, order=2)
    D, V, Vi = S.get_eig(0)
    e = EigT(g, k0)
    # same spectrum as LAPACK on the oracle's matrix, and V D V^-1 rebuilds Lambda-bar
    ref = np.sort_complex(e.Dx)
    got = np.sort_complex(D)
    assert np.abs(got - ref).max() < 1e-10
    from oracle.eig1d import lambda_bar
    Lb = lambda_bar(n, e.gx, e.zx)
    assert np.abs(V @ np.diag(D) @ Vi - Lb).max() < 1e-10
    assert np.abs(Vi @ V - np.eye(n)).max() < 1e-10


# FP32 transform passes; the z-solve and the whole preconditioner per case (measured max-norm errors on a
# GB300: 2.9e-6 / 2.3e-6 at 40 x 36 x 33, 6.2e-6 / 5.4e-6 at 64^3, 6.5e-5 / 8.0e-5 at 48 x 40 x 300)
TOL_PASS_FP32 = 1.5e-6


@pytest.mark.parametrize("n,L,tol", [((40, 36, 33), (1.0, 0.9, 0.825), 8e-6), ((64, 64, 64), (1.0, 1.0, 1.0), 1.8e-5),
                                     ((48, 40, 300), (1.0, 1.0, 1.0), 2.4e-4)])
def test_precond_steps_match_oracle(n, L, tol):
    g, k2, k0 = _medium(n, L)
    S = Solver(n, k2, k0, order=4, L=L, precision=HELM_PREC_FP32)
    e = EigT(g, k0)
    # the transformed coordinates depend on the eigenvector basis: check the steps in the GPU's own
    # FP64 basis (the basis itself is pinned by test_eigensetup_diagonalises_lambda_bar)
    e.Dx, e.Vx, e.Vxi = S.get_eig(0)
    e.Dy, e.Vy, e.Vyi = S.get_eig(1)
    y = _rand(g.shape, 3)
    fwd = S.precond_step(1, _dev(y, torch.complex64)).cpu().numpy()
    ref_fwd = e.forward(y)
    assert _rel(fwd, ref_fwd) < TOL_PASS_FP32
    # z-solve on exactly the same input
    sub, diag, sup = e.z_coefficients()
    zs = S.precond_step(2, _dev(ref_fwd, torch.complex64)).cpu().numpy()
    ref_z = thomas(sub, diag, sup, ref_fwd)
    assert _rel(zs, ref_z) < tol
    inv = S.precond_step(3, _dev(ref_z, torch.complex64)).cpu().numpy()
    assert _rel(inv, e.inverse(ref_z)) < TOL_PASS_FP32
    z = S.apply_precond(_dev(y, torch.complex64)).cpu().numpy()
    assert _rel(z, e.apply_Minv(y)) < tol


def _solve_pair(n, order, flexible, seed_m=None):
    if seed_m is None:
        k2, f, k0 = media.single_gaussian(n)
    else:
        k2, f, k0 = media.bumps(n, seed_m, seed_m + 1)
    S = Solver((n, n, n), k2, k0, order=order, flexible=flexible, rtol=1e-6, restart=30, max_iter=200)
    F = S.build_rhs(_dev(f))
    x, info = S.solve(F)
    g = Grid(n, n, n, staggered=True)
    A = Operator(g, k2, k0, order)
    e = EigT(g, k0)
    Fh = F.cpu().numpy()
    xo, io = gmres(A, e.apply_Minv, Fh, m=30, rtol=1e-12, max_it=400)
    xo = xo.reshape(g.shape)
    _, io6 = gmres(A, e.apply_Minv, Fh, m=30, rtol=1e-6, max_it=400, flexible=flexible)
    io["iterations_at_rtol"] = io6["iterations"]
    xg = x.cpu().numpy()
    relerr = np.linalg.norm(xg - xo) / np.linalg.norm(xo)
    relres = np.linalg.norm(A(xg) - Fh) / np.linalg.norm(Fh)
    return info, relerr, relres, io


@pytest.mark.parametrize("flexible", [False, True])
def test_gmres_config1_matches_oracle(flexible):
    """4th order, 32^3, single Gaussian inclusion, EigT, GMRES(30)/FGMRES(30), rtol 1e-6."""
    info, relerr, relres, io = _solve_pair(32, 4, flexible)
    assert info.status == 0 and info.relres_true <= 1e-6
    assert relres <= 1.5e-6            # the oracle's FP64 residual of the GPU solution
    assert relerr <= 1e-5
    # same Krylov process as the oracle; right-preconditioned GMRES forms the update M^-1 (V y) from
    # complex64 vectors, so its first cycle can stop one restart short of the FP64 true residual
    assert -1 <= info.iterations - io["iterations_at_rtol"] <= (1 if flexible else 3)


def test_gmres_order6_bumps_matches_oracle():
    info, relerr, relres, io = _solve_pair(40, 6, True, seed_m=11)
    assert info.status == 0 and info.relres_true <= 1e-6
    assert abs(info.iterations - io["iterations_at_rtol"]) <= 1
    assert relres <= 1.5e-6
    assert relerr <= 1e-5


def test_second_order_operator_converges_in_one_iteration():
    n = 36
    g = Grid(n, n, n, staggered=True)
    k0 = 2 * math.pi / (10 * g.h[0])
    S = Solver((n, n, n), np.full(g.shape, k0 * k0, complex), k0, order=2, rtol=1e-5)
    b = _dev(_rand(g.shape, 9))
    x, info = S.solve(b)
    assert info.iterations == 1 and info.relres_true < 1e-5


@pytest.mark.parametrize("order", [2, 4, 6])
def test_residual_resolves_small_residuals(order):
    """helm_residual (double-float) against the oracle's FP64 F - A x when ||F - A x|| ~ 1e-9 ||F||:
    complex64 arithmetic could not resolve this residual at all."""
    n, L = (32, 32, 32), (1.0, 1.0, 1.0)
    g, k2, k0 = _medium(n, L)
    A = Operator(g, k2, k0, order)
    F = _rand(g.shape, 12)
    x, info = gmres(A, EigT(g, k0).apply_Minv, F, m=30, rtol=1e-13, max_it=600)
    xp = x.reshape(g.shape) + 1e-9 * np.abs(x).max() * _rand(g.shape, 13)
    r_ref = F - A(xp)
    S = Solver(n, k2, k0, order=order, L=L)
    n2, ni = S.residual(_dev(F), _dev(xp))
    ref2 = np.linalg.norm(r_ref)
    assert ref2 < 1e-6 * np.linalg.norm(F)
    assert abs(n2 - ref2) <= 0.02 * ref2, (n2, ref2)
    assert abs(ni - np.abs(r_ref).max()) <= 0.05 * np.abs(r_ref).max()


@pytest.mark.parametrize("order,n,L,complex_k", [
    (6, (40, 36, 33), (1.0, 0.9, 0.825), False),   # real medium: the two-row compensated-sum kernel
    (6, (70, 20, 65), (1.0, 20 / 70, 65 / 70), False),
    (6, (40, 36, 33), (1.0, 0.9, 0.825), True),    # complex medium: the renormalised double-float kernel
    (4, (40, 36, 33), (1.0, 0.9, 0.85), False),
])
def test_residual_vector_matches_oracle_elementwise(order, n, L, complex_k):
    """r = F - A x of helm_residual against the FP64 oracle at every point, for F = A x + d with
    |d| ~ 1e-9 |A x| (so that F - A x cancels nine digits).  x is a plane wave modulated by a smooth envelope
    plus a small random part, nonzero on the boundary (every ghost factor is used).  Bound per point:
    the complex64 rounding of r (2^-23 |r|) plus the double-float error, 1e-11 h^-2 max|x|: ~40 additions
    of error <= 2^-44 of the terms' magnitudes, which sum to about 8.5 h^-2 |x|, plus, at order 6, the FP32
    rounding of the gradient terms (h/20) g_d D_d that both kernels take from the leading parts, 2^-19
    (h/20) sum_d |g_d| max|x| at the point (D_d sums ~10 FP32 terms of size |x|: error ~2^-20.4 |x|).
    FP32 arithmetic for the whole operator would miss the bound by three orders of magnitude (2^-24 x 8.5
    h^-2 |x|).  The norms follow from the same bound by the triangle inequality."""
    g, k2, k0 = _medium(n, L)
    if not complex_k:
        k2 = k2.real + 0j
    X, Y, Z = g.mesh()
    x = np.exp(1j * k0 * (0.6 * X + 0.48 * Y + 0.64 * Z)) * (1 + 0.3 * np.sin(5 * X + 2 * Y) * np.cos(3 * Z))
    x = x + 1e-3 * _rand(g.shape, 21)
    A = Operator(g, k2, k0, order)
    Ax = A(x)
    F = Ax + 1e-9 * np.abs(Ax).max() * _rand(g.shape, 22)
    r_ref = F - A(x)
    S = Solver(n, k2, k0, order=order, L=L)
    r = torch.empty(g.shape, dtype=torch.complex64, device="cuda")
    from paper_2602_07711_gb300 import helm
    n2, ni = helm.helm_residual(S.ctx, _dev(F), _dev(x), r)
    S.close()
    rg = r.cpu().numpy().astype(np.complex128)
    bound = 2.0 ** -23 * np.abs(r_ref) + 1e-11 * np.abs(x).max() / g.h[0] ** 2
    if order == 6:
        dk2, _ = derived_k2_fields(k2, True, g.h)
        bound = bound + 2.0 ** -19 * (g.h[0] / 20) * sum(np.abs(d) for d in dk2) * np.abs(x).max()
    err = np.abs(rg - r_ref)
    assert np.all(err <= bound), (float((err / bound).max()), float(np.abs(r_ref).max()))
    assert abs(n2 - np.linalg.norm(r_ref)) <= np.linalg.norm(bound)
    assert abs(ni - np.abs(r_ref).max()) <= bound.max()


@pytest.mark.parametrize("rtol", [1e-6, 1e-8])
def test_scattering_sphere_matches_oracle(rtol):
    """The single-inclusion scattering problem of Sec. 5.2 (k^2 = 1050 + 2.26i inside r = 0.1 at
    (0.5, 0.5, 0.7), 439.2 outside, f = -(k^2 - k0^2) e^{i k0 z}, staggered grid) at 40^3, sixth order,
    EigT + FGMRES(20) as in the paper's table, mixed precision on the GPU against the FP64 oracle."""
    n = 40
    k2, f, k0 = media.sphere(n)
    S = Solver((n, n, n), k2, k0, order=6, flexible=True, rtol=rtol, restart=20, max_iter=200)
    F = S.build_rhs(_dev(f))
    x, info = S.solve(F)
    g = Grid(n, n, n, staggered=True)
    A = Operator(g, k2, k0, 6)
    e = EigT(g, k0)
    Fh = F.cpu().numpy()
    xo, _ = gmres(A, e.apply_Minv, Fh, m=20, rtol=1e-12, max_it=400)
    xo = xo.reshape(g.shape)
    _, io = gmres(A, e.apply_Minv, Fh, m=20, rtol=rtol, max_it=400, flexible=True)
    xg = x.cpu().numpy()
    assert info.status == 0 and info.relres_true <= rtol
    assert np.linalg.norm(A(xg) - Fh) / np.linalg.norm(Fh) <= 1.5 * rtol   # the oracle's FP64 residual
    assert np.linalg.norm(xg - xo) / np.linalg.norm(xo) <= 10 * rtol
    # the first restart cycle is the oracle's Krylov process until its estimate has fallen by the inner
    # tolerance of a cycle (1e-4); the later cycles restart from the double-float true residual, and a
    # restarted GMRES never needs fewer iterations than an unrestarted one
    _, io4 = gmres(A, e.apply_Minv, Fh, m=20, rtol=1e-4, max_it=400, flexible=True)
    assert abs(info.cycle_its[0] - io4["iterations"]) <= 1
    assert io["iterations"] - 1 <= info.iterations <= io["iterations"] + 5


@pytest.mark.parametrize("order,case", [(4, SIZES[4][0]), (4, SIZES[4][2]), (6, SIZES[6][0]), (6, SIZES[6][2])])
def test_apply_A_real_medium_matches_oracle(order, case):
    """A medium without attenuation (Im k^2 = 0) takes the real-medium complex64 matvec (k^2 staged as
    float, the order-6 fields as one real float4 per point); same oracle and tolerance as the general one."""
    n, L = case
    g, k2, k0 = _medium(n, L)
    k2 = k2.real + 0j
    S = Solver(n, k2, k0, order=order, L=L)
    x = _rand(g.shape, 1)
    ref = Operator(g, k2, k0, order)(x)
    y64 = S.apply_A(_dev(x, torch.complex64)).cpu().numpy()
    assert _rel(y64, ref) < 2e-6


def test_profile_classes_times_only_the_selected_class():
    """helm_profile_classes records events only around the launches of the selected kernel classes (the
    bench times the dominant kernel this way inside its timed region); helm_profile times every class."""
    from paper_2602_07711_gb300 import helm
    n = 32
    k2, f, k0 = media.single_gaussian(n)
    S = Solver((n, n, n), k2, k0, order=4, rtol=1e-6)
    F = S.build_rhs(_dev(f))
    L = helm.lib()
    ms = (helm.C.c_double * 11)()
    ln = (helm.C.c_longlong * 11)()
    dots, stencil = 4, 0
    assert L.helm_profile_classes(S.ctx, 1 << dots) == 0
    _, info = S.solve(F)
    assert L.helm_profile_read(S.ctx, ms, ln, 11, 1) == 0
    # (an iteration enqueued ahead past the end of a cycle runs too)
    assert ln[dots] >= info.iterations and ms[dots] > 0
    assert all(ln[i] == 0 for i in range(11) if i != dots)
    assert L.helm_profile(S.ctx, 1) == 0
    _, info = S.solve(F)
    assert L.helm_profile_read(S.ctx, ms, ln, 11, 1) == 0
    assert ln[dots] >= info.iterations and ln[stencil] >= info.iterations
    assert L.helm_profile(S.ctx, 0) == 0
