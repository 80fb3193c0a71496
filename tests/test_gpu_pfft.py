"""PFFT preconditioner (Sec. 4.2) on the GPU against the oracle, through the C-ABI.

The PFFT solve and the EigT solve both invert the same A_p exactly, so the GPU's PFFT output is checked
against both the oracle's PFFT (face-Dirichlet sine basis) and its EigT.  Fixed relative 2-norm bounds
per case, about 3x the errors measured on a GB300: FP32 sine transforms 1.6e-5 (32 x 32 x 20), 7.7e-5
(64 x 32 x 33), 1.0e-5 (16 x 64 x 8), 4.5e-6 (128 x 128 x 12); TF32 tensor-core sine products 1.4e-3 and
1.5e-3 (as the TF32 EigT transforms).
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle.eigt import EigT
from oracle.grid import Grid
from oracle.pfft import PFFT
from paper_2602_07711_gb300 import HELM_PREC_TF32, HELM_PRECOND_EIGT, HELM_PRECOND_FFT2, HELM_PRECOND_PFFT, Solver, media


def _rand(shape, seed):
    r = np.random.default_rng(seed)
    return r.standard_normal(shape) + 1j * r.standard_normal(shape)


@pytest.mark.parametrize("n,L,tol", [((32, 32, 20), (1.0, 1.0, 0.625), 5e-5), ((64, 32, 33), (1.0, 0.6, 0.5), 2.3e-4),
                                     ((16, 64, 8), (0.25, 1.0, 0.2), 3e-5), ((128, 128, 12), (1.0, 1.0, 0.1), 1.5e-5)])
def test_pfft_preconditioner_matches_oracle(n, L, tol):
    g = Grid(*n, lx=L[0], ly=L[1], lz=L[2], staggered=True)
    k0 = 2 * math.pi / (10 * g.h[0])
    S = Solver(n, np.full(g.shape, k0 * k0, complex), k0, order=4, L=L, precond=HELM_PRECOND_PFFT)
    y = _rand(g.shape, 7)
    z = S.apply_precond(torch.from_numpy(y).to("cuda", torch.complex64)).cpu().numpy()
    e = EigT(g, k0)
    for ref in (PFFT(g, k0, variant="face").apply_Minv(y), e.apply_Minv(y)):
        err = np.linalg.norm(z - ref) / np.linalg.norm(ref)
        assert err < tol, err


def test_pfft_gmres_matches_eigt_gmres():
    n = 64
    k2, f, k0 = media.bumps(n, 31, 32)
    out = {}
    for pc in (HELM_PRECOND_EIGT, HELM_PRECOND_PFFT):
        S = Solver((n, n, n), k2, k0, order=6, precond=pc, flexible=True, rtol=1e-6)
        x, info = S.solve(S.build_rhs(torch.from_numpy(f).cuda()))
        assert info.status == 0 and info.relres_true <= 1e-6
        out[pc] = (x.cpu().numpy(), info.iterations)
    d = np.linalg.norm(out[1][0] - out[2][0]) / np.linalg.norm(out[1][0])
    assert d < 2e-5 and abs(out[1][1] - out[2][1]) <= 1


@pytest.mark.parametrize("n,L", [((32, 32, 20), (1.0, 1.0, 0.625)), ((128, 64, 12), (1.0, 0.5, 0.1))])
def test_pfft_tensor_core_transforms_match_oracle(n, L):
    """TF32 contexts run the sine transforms as tcgen05 products with the sine bases: the TF32 bound of
    the EigT preconditioner applies (4e-3 in the 2-norm)."""
    g = Grid(*n, lx=L[0], ly=L[1], lz=L[2], staggered=True)
    k0 = 2 * math.pi / (10 * g.h[0])
    S = Solver(n, np.full(g.shape, k0 * k0, complex), k0, order=4, L=L, precond=HELM_PRECOND_PFFT,
               precision=HELM_PREC_TF32, flexible=True)
    y = _rand(g.shape, 8)
    z = S.apply_precond(torch.from_numpy(y).to("cuda", torch.complex64)).cpu().numpy()
    ref = PFFT(g, k0, variant="face").apply_Minv(y)
    err = np.linalg.norm(z - ref) / np.linalg.norm(ref)
    assert err < 4e-3, err


def test_pfft_tensor_core_fgmres_converges_like_eigt():
    n = 64
    k2, f, k0 = media.bumps(n, 33, 34)
    out = {}
    for pc in (HELM_PRECOND_EIGT, HELM_PRECOND_PFFT):
        S = Solver((n, n, n), k2, k0, order=6, precond=pc, precision=HELM_PREC_TF32, flexible=True, rtol=1e-6)
        x, info = S.solve(S.build_rhs(torch.from_numpy(f).cuda()))
        assert info.status == 0 and info.relres_true <= 1e-6
        out[pc] = (x.cpu().numpy(), info.iterations)
    d = np.linalg.norm(out[1][0] - out[2][0]) / np.linalg.norm(out[1][0])
    assert d < 1e-5 and abs(out[1][1] - out[2][1]) <= 2


@pytest.mark.parametrize("n,L", [((32, 32, 20), (1.0, 1.0, 0.625)), ((64, 32, 33), (1.0, 0.6, 0.5))])
def test_fft2_preconditioner_matches_oracle(n, L):
    """FFT2 = h_z^2 (A_p^F)^-1 (the Dirichlet sine solve of PFFT's first step) against the oracle's."""
    g = Grid(*n, lx=L[0], ly=L[1], lz=L[2], staggered=True)
    k0 = 2 * math.pi / (10 * g.h[0])
    S = Solver(n, np.full(g.shape, k0 * k0, complex), k0, order=4, L=L, precond=HELM_PRECOND_FFT2)
    y = _rand(g.shape, 9)
    z = S.apply_precond(torch.from_numpy(y).to("cuda", torch.complex64)).cpu().numpy()
    hz = g.h[2]
    ref = hz * hz * PFFT(g, k0, variant="face").solve_F(y).reshape(g.shape)
    # FP32 sine transforms and z-solves; without the absorbing condition the Dirichlet z-systems have no
    # damping and come closer to singular than EigT's, which amplifies the rounding (1.6e-5 measured at 32^3)
    assert np.linalg.norm(z - ref) / np.linalg.norm(ref) < 1e-4


def test_fft2_needs_many_more_iterations_than_eigt():
    """The paper's comparison (Sec. 5): a preconditioner with the absorbing condition (EigT) converges in a
    handful of iterations where the Dirichlet one (FFT2) needs many; both reach the same solution."""
    n = 64
    k2, f, k0 = media.bumps(n, 31, 32)
    out = {}
    for pc in (HELM_PRECOND_EIGT, HELM_PRECOND_FFT2):
        S = Solver((n, n, n), k2, k0, order=6, precond=pc, flexible=True, rtol=1e-6, max_iter=400)
        x, info = S.solve(S.build_rhs(torch.from_numpy(f).cuda()))
        assert info.status == 0 and info.relres_true <= 1e-6
        out[pc] = (x.cpu().numpy(), info.iterations)
    d = np.linalg.norm(out[HELM_PRECOND_EIGT][0] - out[HELM_PRECOND_FFT2][0]) / np.linalg.norm(out[HELM_PRECOND_EIGT][0])
    assert d < 2e-5
    assert out[HELM_PRECOND_FFT2][1] >= 3 * out[HELM_PRECOND_EIGT][1]


# ---- PFFT3: collocated grids (Sec. 4.2 with the three-point ABC: Lbar corner 2 i k0 h, zeta = 2) ------------
# The correction (A_p^F - A_p) then reads the two outer layers of Theta and W; the result must still equal
# the oracle's PFFT and EigT (which invert the same A_p).
@pytest.mark.parametrize("n,L,tol", [((32, 32, 20), (1.0, 1.0, 0.625), 5e-5), ((64, 32, 33), (1.0, 0.6, 0.5), 2.3e-4)])
def test_pfft3_collocated_preconditioner_matches_oracle(n, L, tol):
    g = Grid(*n, lx=L[0], ly=L[1], lz=L[2], staggered=False)
    k0 = 2 * math.pi / (10 * g.h[0])
    S = Solver(n, np.full(g.shape, k0 * k0, complex), k0, order=4, L=L, precond=HELM_PRECOND_PFFT, staggered=False)
    y = _rand(g.shape, 17)
    z = S.apply_precond(torch.from_numpy(y).to("cuda", torch.complex64)).cpu().numpy()
    for ref in (PFFT(g, k0, variant="face").apply_Minv(y), EigT(g, k0).apply_Minv(y)):
        err = np.linalg.norm(z - ref) / np.linalg.norm(ref)
        assert err < tol, err
    # the one-layer correction of PFFT2 is not enough here: dropping the second layer is a visible error
    e = EigT(g, k0)
    P1 = PFFT(g, k0, variant="face")
    zeta_x, zeta_y = P1.eigt.zx, P1.eigt.zy
    P1.eigt.zx = P1.eigt.zy = 1.0          # oracle copy with the second-layer term dropped (planted mistake)
    bad = P1.apply_Minv(y)
    P1.eigt.zx, P1.eigt.zy = zeta_x, zeta_y
    assert np.linalg.norm(bad - e.apply_Minv(y)) / np.linalg.norm(e.apply_Minv(y)) > 100 * tol


def test_pfft3_tensor_core_matches_oracle():
    n, L = (64, 32, 20), (1.0, 0.5, 0.3)
    g = Grid(*n, lx=L[0], ly=L[1], lz=L[2], staggered=False)
    k0 = 2 * math.pi / (10 * g.h[0])
    S = Solver(n, np.full(g.shape, k0 * k0, complex), k0, order=4, L=L, precond=HELM_PRECOND_PFFT,
               precision=HELM_PREC_TF32, flexible=True, staggered=False)
    y = _rand(g.shape, 18)
    z = S.apply_precond(torch.from_numpy(y).to("cuda", torch.complex64)).cpu().numpy()
    ref = EigT(g, k0).apply_Minv(y)
    assert np.linalg.norm(z - ref) / np.linalg.norm(ref) < 4e-3


def test_pfft3_gmres_on_the_manufactured_problem_matches_eigt3():
    """The paper's test problem of Sec. 5.1 (collocated grid, high-order closure, sixth order) with PFFT3 and
    with EigT3: the same iterations (+-1) and the same solution."""
    from paper_2602_07711_gb300 import HELM_CLOSURE_HIGH_ORDER
    n = 64
    k0 = math.sqrt(439.2)
    d = media.manufactured(n, k0, 6)
    out = {}
    for pc in (HELM_PRECOND_EIGT, HELM_PRECOND_PFFT):
        S = Solver((n, n, n), d["k2"], k0, order=6, precond=pc, flexible=True, rtol=1e-10, restart=20, max_iter=200,
                   staggered=False)
        S.set_closure(HELM_CLOSURE_HIGH_ORDER)
        F = S.closure_rhs(torch.from_numpy(d["faces"]).cuda(), S.build_rhs_fields(torch.from_numpy(d["fields"]).cuda()))
        x, info = S.solve(F)
        assert info.status == 0 and info.relres_true <= 1e-10
        out[pc] = (x.cpu().numpy(), info.iterations)
        S.close()
    xe, xp = out[HELM_PRECOND_EIGT][0], out[HELM_PRECOND_PFFT][0]
    assert np.linalg.norm(xe - xp) / np.linalg.norm(xe) < 1e-8
    assert abs(out[HELM_PRECOND_EIGT][1] - out[HELM_PRECOND_PFFT][1]) <= 1
    # and the printed sixth-order accuracy of the scheme is reached (64^3: between the 50^3 and 100^3 rows)
    u = d["u"]
    assert 9.97e-8 < np.linalg.norm(xp - u) / np.linalg.norm(u) < 7.06e-6
