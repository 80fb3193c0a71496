"""Pins of the CPU oracle against what the paper and the mathematics fix (no GPU).

Each test names the passage it checks.  Together they are chosen so that a dropped term, a wrong sign,
a wrong index or a transposed operand anywhere in the oracle fails at least one of them.
"""
import math
import os

import numpy as np
import pytest
import scipy.linalg as sla

from oracle import manufactured as mf
from oracle import metrics
from oracle.closure import pad_ghost_ho
from oracle.eig1d import abc_params, dirichlet_closed_form, eig_decomp, lambda_bar, lambda_dirichlet
from oracle.eigt import EigT
from oracle.gmres import gmres
from oracle.grid import Grid, gamma_two_point
from oracle.model1d import d_r, matrices
from oracle.operators import Operator, apply_A4, apply_A6, derived_k2_fields
from oracle.pfft import PFFT
from oracle.rhs import rhs4_padded, rhs6, rhs6_sampled
from oracle.tridiag import thomas
from paper_tables import high_order_rows, printed_half_unit

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
K0_PAPER = math.sqrt(439.2)


def _rand(shape, seed):
    r = np.random.default_rng(seed)
    return r.standard_normal(shape) + 1j * r.standard_normal(shape)


# ---- grid (Sec. 2.1, Sec. 5.2) -------------------------------------------------------------
def test_unknown_count_and_nodes():
    g = Grid(32, 31, 30, staggered=True)
    assert g.unknowns == 32 * 31 * 30 and g.shape == (30, 31, 32)
    assert np.allclose(g.coords(0), (np.arange(32) + 0.5) / 32)
    c = Grid(17, 17, 17, staggered=False)
    assert c.unknowns == 17 ** 3
    assert np.isclose(c.coords(0)[0], 0.0) and np.isclose(c.coords(0)[-1], 1.0)


def test_gamma_unimodular_and_consistent():
    # |gamma| = 1 for real k0 (the two-point ABC only rotates the phase), and the ghost it predicts
    # approaches the outgoing wave exp(-i k0 x) sampled half a step outside the face as h -> 0.
    k0 = 12.0
    errs = []
    for n in (32, 64, 128):
        h = 1.0 / n
        g = gamma_two_point(k0, h)
        assert abs(abs(g) - 1.0) < 1e-15
        ghost_exact = np.exp(-1j * k0 * (-h / 2)) / np.exp(-1j * k0 * (h / 2))
        errs.append(abs(g - ghost_exact))
    assert errs[0] / errs[1] > 7.5 and errs[1] / errs[2] > 7.5   # third order in h


# ---- 1D matrices and eigenpairs (Sec. 3.1, Sec. 4.1) ---------------------------------------
@pytest.mark.parametrize("N", [2, 5, 16, 33])
def test_dirichlet_eigenpairs_closed_form(N):
    lam, Vc = dirichlet_closed_form(N)
    L = lambda_dirichlet(N)
    assert np.allclose(L @ Vc, Vc * lam[None, :], atol=1e-12)
    assert np.allclose(Vc.T @ Vc, np.eye(N), atol=1e-12)
    D, V, Vi = eig_decomp(N, 0.0, 1.0)
    assert np.allclose(np.sort(D.real), np.sort(lam), atol=1e-12)


@pytest.mark.parametrize("staggered", [True, False])
def test_lambda_bar_structure_and_eigvecs(staggered):
    N, k0, h = 12, 9.0, 1.0 / 12
    g, z = abc_params(k0, h, staggered)
    L = lambda_bar(N, g, z)
    assert L[0, 0] == g and L[-1, -1] == g and L[0, 1] == z and L[-1, -2] == z and L[1, 0] == 1
    D, V, Vi = eig_decomp(N, g, z)
    # Diagonal similarity S = diag(sqrt(z),1..1,sqrt(z)) makes S^-1 L S complex symmetric, so the
    # eigenvectors are complex-orthogonal after that scaling: (S^-1 V)^T (S^-1 V) is diagonal.
    s = np.ones(N, dtype=complex)
    s[0] = s[-1] = np.sqrt(z)
    Q = V / s[:, None]
    G = Q.T @ Q
    assert np.abs(G - np.diag(np.diag(G))).max() < 1e-10 * np.abs(np.diag(G)).min()
    assert np.allclose(L @ V, V * D[None, :], atol=1e-12)


# ---- 1D model problem: Eq. 1DEGV pins d_r and the preconditioner ---------------------------
@pytest.mark.parametrize("r", [2, 3, 4])
def test_1d_spectrum_closed_form(r):
    N, k = 40, 15.0
    h = 1.0 / (N + 1)
    tau = k * h
    A, Ap = matrices(N, k, r)
    ev = np.sort_complex(np.linalg.eigvals(A @ np.linalg.inv(Ap)))
    i = np.arange(1, N + 1)
    num = 2.0 * sum((-1) ** (j - 1) * tau ** (2 * j) / math.factorial(2 * j) for j in range(2, r + 1))
    closed = 1.0 + num / (-4.0 * np.sin(np.pi * h * i / 2) ** 2 + tau * tau)
    # second form of Eq. 1DEGV
    s = sum((-1) ** (l + 1) * tau ** (2 * l) / math.factorial(2 * (l + 2)) for l in range(0, r - 1))
    closed2 = 1.0 - 2.0 * k ** 4 * h * h * s / (4.0 * np.sin(np.pi * h * i / 2) ** 2 / h / h - k * k)
    assert np.allclose(np.sort_complex(closed + 0j), ev, atol=1e-11)
    assert np.allclose(closed, closed2, atol=1e-11)
    assert abs(d_r(tau, r) - math.cos(tau)) < tau ** (2 * r + 2) / math.factorial(2 * r + 2) * 1.01


@pytest.mark.parametrize("r", [2, 3])
def test_1d_gmres_meets_the_theorem_estimate(r):
    """Theorem last_1D_theorem: right-preconditioned GMRES on the order-2r 1D scheme with the second-order
    preconditioner has ||r_n|| <= (2 tau^2/delta0 sum_l k^(2l)/(4^l (2(l+2))!))^n ||r_0||; the iteration
    count falls as N grows (the property stated after the proof)."""
    k = 15.0
    counts = []
    for N in (40, 80, 160):
        h = 1.0 / (N + 1)
        tau = k * h
        A, Ap = matrices(N, k, r)
        i = np.arange(1, N + 1)
        delta0 = np.min(np.abs(4.0 * np.sin(i * np.pi * h / 2) ** 2 / h ** 2 - k * k)) / (k * k)
        q = 2.0 * tau ** 2 / delta0 * sum(k ** (2 * l) / (4 ** l * math.factorial(2 * (l + 2))) for l in range(r - 1))
        assert q < 1.0
        hist = []
        b = np.random.default_rng(N).standard_normal(N) + 0j
        _, info = gmres(lambda v: A @ v, lambda v: np.linalg.solve(Ap, v), b, m=N, rtol=1e-13, max_it=N,
                        history=hist)
        for n, rel in enumerate(hist, start=1):
            if q ** n < 1e-12:
                break
            assert rel <= q ** n * (1 + 1e-9), (N, n, rel, q ** n)
        counts.append(next(n for n, rel in enumerate(hist, start=1) if rel <= 1e-10))
    assert counts[0] >= counts[1] >= counts[2] and counts[0] > counts[2], counts


# ---- Thomas (Eq. Indep_precond_system) --------------------------------------------------------
def test_thomas_vs_banded_solver():
    n, m = 37, 5
    r = np.random.default_rng(3)
    a = r.standard_normal((n, m)) + 1j * r.standard_normal((n, m))
    c = r.standard_normal((n, m)) + 1j * r.standard_normal((n, m))
    b = 4 + r.standard_normal((n, m)) + 1j * r.standard_normal((n, m))
    d = r.standard_normal((n, m)) + 1j * r.standard_normal((n, m))
    x = thomas(a, b, c, d)
    for col in range(m):
        ab = np.zeros((3, n), dtype=complex)
        ab[0, 1:] = c[:-1, col]
        ab[1] = b[:, col]
        ab[2, :-1] = a[1:, col]
        ref = sla.solve_banded((1, 1), ab, d[:, col])
        assert np.allclose(x[:, col], ref, rtol=1e-12, atol=1e-12)


# ---- EigT exactly inverts A_p (Sec. 4.1) ----------------------------------------------------
@pytest.mark.parametrize("staggered", [True, False])
@pytest.mark.parametrize("n", [(8, 8, 8), (8, 7, 6)])
def test_eigt_equals_dense_lu(staggered, n):
    g = Grid(*n, lx=1.0, ly=0.9, lz=1.1, staggered=staggered)
    k0 = 7.3
    prof = k0 * k0 * (1 + 0.1 * np.linspace(0, 1, n[2]))    # depth-dependent K_z of Sec. 4.1
    e = EigT(g, k0, k0z2=prof)
    Y = _rand(g.shape, 1)
    U = e.solve_Ap(Y)
    Ud = sla.lu_solve(sla.lu_factor(e.dense_Ap()), Y.ravel()).reshape(g.shape)
    assert np.abs(U - Ud).max() <= 1e-12 * np.abs(Ud).max()


@pytest.mark.parametrize("staggered", [True, False])
def test_second_order_stencil_is_kronecker_Ap(staggered):
    # The stencil form (Sec. 2, delta^2 + k0^2 with the ghosts eliminated) and the Kronecker form of A_p
    # (Sec. 4.1) are two statements of the same matrix: A_p = h_z^2 A_2.
    g = Grid(6, 5, 7, lx=1.0, ly=0.8, lz=1.2, staggered=staggered)
    k0 = 5.0
    A2 = Operator(g, np.full(g.shape, k0 * k0), k0, 2).dense()
    Ap = EigT(g, k0).dense_Ap()
    hz = g.h[2]
    assert np.abs(A2 * hz * hz - Ap).max() < 1e-13 * np.abs(Ap).max()


@pytest.mark.parametrize("staggered", [True, False])
def test_gmres_one_iteration_on_second_order_operator(staggered):
    g = Grid(10, 9, 8, staggered=staggered)
    k0 = 11.0
    A = Operator(g, np.full(g.shape, k0 * k0), k0, 2)
    e = EigT(g, k0)
    x, info = gmres(A, e.apply_Minv, _rand(g.shape, 2), m=20, rtol=1e-10)
    assert info["iterations"] == 1 and info["relres"] < 1e-12


def _copy_eigt(e):
    c = EigT.__new__(EigT)
    c.__dict__.update(e.__dict__)
    return c


@pytest.mark.parametrize("mistake", ["transposed_Vxi", "row_shifted_Vxi", "transposed_Vyi", "conjugated_Vyi"])
def test_transform_bounds_catch_a_wrong_basis(mistake):
    """The fixed bounds of the GPU transform tests (2e-3 relative in the 2-norm for one TF32 pass, 4e-3 for
    the preconditioner; EigT steps 2 and 4 of Sec. 4.1) lie far below what the plausible kernel mistakes
    give.  Each mistake is planted in a copy of the oracle at the headline's 256 x 256 transform size."""
    g = Grid(256, 256, 8, staggered=True)
    k0 = 2 * math.pi / (10 * g.h[0])
    e = EigT(g, k0)
    y = _rand(g.shape, 5)
    ref = e.forward(y)
    bad = _copy_eigt(e)
    if mistake == "transposed_Vxi":
        bad.Vxi = e.Vxi.T.copy()
    elif mistake == "row_shifted_Vxi":
        bad.Vxi = np.roll(e.Vxi, 1, axis=0)
    elif mistake == "transposed_Vyi":
        bad.Vyi = e.Vyi.T.copy()
    else:
        bad.Vyi = e.Vyi.conj()
    err = np.linalg.norm(bad.forward(y) - ref) / np.linalg.norm(ref)
    assert err > 50 * 4e-3, err
    # and the inverse transform with the same mistake in V
    bad_inv = _copy_eigt(e)
    bad_inv.Vx = e.Vx.T.copy() if "Vxi" in mistake else e.Vx
    bad_inv.Vy = e.Vy.conj() if mistake == "conjugated_Vyi" else (e.Vy.T.copy() if "Vyi" in mistake else e.Vy)
    if mistake == "row_shifted_Vxi":
        bad_inv.Vx = np.roll(e.Vx, 1, axis=0)
    ref_inv = e.inverse(y)
    err = np.linalg.norm(bad_inv.inverse(y) - ref_inv) / np.linalg.norm(ref_inv)
    assert err > 50 * 4e-3, err


# ---- PFFT = EigT (Sec. 4.2) ------------------------------------------------------------------
@pytest.mark.parametrize("variant", ["node", "face"])
@pytest.mark.parametrize("staggered", [True, False])
def test_pfft_equals_eigt(variant, staggered):
    g = Grid(9, 8, 7, lx=1.0, ly=0.9, lz=1.0, staggered=staggered)
    k0 = 6.5
    Y = _rand(g.shape, 4)
    Ue = EigT(g, k0).solve_Ap(Y)
    Up = PFFT(g, k0, variant=variant).solve_Ap(Y)
    assert np.abs(Up - Ue).max() <= 1e-12 * np.abs(Ue).max()


def test_pfft_correction_is_boundary_sparse():
    g = Grid(9, 8, 7)
    p = PFFT(g, 6.5, variant="face")
    R = p.diff_apply(_rand(g.shape, 5))
    inner = R[:, 1:-1, 1:-1]
    assert np.abs(inner).max() == 0.0 and np.abs(R[:, 0, 3]).max() > 0


# ---- golden: Table tab:direct_solve (second-order direct solve errors) ---------------------
def _golden_direct():
    rows = []
    with open(os.path.join(GOLDEN, "direct_solve_table.txt")) as fh:
        for line in fh:
            if line.strip() and not line.startswith("#"):
                n, me, l2 = line.split()
                rows.append((int(n), float(me), float(l2)))
    return rows


@pytest.mark.parametrize("row", _golden_direct())
def test_paper_direct_solve_errors(row):
    N, me_paper, l2_paper = row
    g = Grid(N, N, N, staggered=True)
    X, Y, Z = g.mesh()
    u = mf.u_exact(X, Y, Z, K0_PAPER)
    f = mf.f_exact(X, Y, Z, K0_PAPER)
    U = EigT(g, K0_PAPER).apply_Minv(f)
    me, l2 = metrics.max_err(u, U), metrics.l2_err(u, U)
    assert abs(me - me_paper) <= 0.005 * 10 ** math.floor(math.log10(me_paper))
    assert abs(l2 - l2_paper) <= 0.05 * 10 ** math.floor(math.log10(l2_paper))


# ---- truncation order of the compact schemes (Eqs. scheme4, scheme6) ------------------------
def _smooth_fields():
    sp = pytest.importorskip("sympy")
    X, Y, Z = sp.symbols("x y z", real=True)
    u = sp.exp(sp.I * (1.3 * X + 0.7 * Y - 0.9 * Z)) * (1 + sp.Rational(1, 2) * sp.sin(2 * X + Y)) + sp.cos(1.1 * Y + 0.4 * Z)
    k2 = 20 * (1 + sp.Rational(3, 10) * sp.sin(1.7 * X + 0.6 * Y + 1.1 * Z) + sp.Rational(1, 5) * sp.cos(0.8 * X - 1.3 * Z)) \
        + sp.I * sp.Rational(1, 2) * sp.sin(X + Y)
    f = sp.diff(u, X, 2) + sp.diff(u, Y, 2) + sp.diff(u, Z, 2) + k2 * u
    ex = dict(u=u, k2=k2, f=f,
              lapf=sp.diff(f, X, 2) + sp.diff(f, Y, 2) + sp.diff(f, Z, 2),
              sum4f=sp.diff(f, X, 4) + sp.diff(f, Y, 4) + sp.diff(f, Z, 4),
              mixf=sp.diff(f, X, 2, Y, 2) + sp.diff(f, X, 2, Z, 2) + sp.diff(f, Y, 2, Z, 2),
              fx=sp.diff(f, X), fy=sp.diff(f, Y), fz=sp.diff(f, Z),
              k2x=sp.diff(k2, X), k2y=sp.diff(k2, Y), k2z=sp.diff(k2, Z),
              lapk2=sp.diff(k2, X, 2) + sp.diff(k2, Y, 2) + sp.diff(k2, Z, 2))
    fn = {k: sp.lambdify((X, Y, Z), v, "numpy") for k, v in ex.items()}
    return lambda name, P: np.broadcast_to(np.asarray(fn[name](*P), dtype=complex), P[0].shape)


def _truncation(order, h, ev):
    n = 5
    r = (np.arange(-1, n + 1)) * h + 0.3
    Zm, Ym, Xm = np.meshgrid(r, r, r, indexing="ij")
    P = (Xm, Ym, Zm)
    Up, Kp = ev("u", P), ev("k2", P)
    C = tuple(a[1:-1, 1:-1, 1:-1] for a in P)
    hh = (h, h, h)
    if order == 4:
        AU = apply_A4(Up, Kp, hh)
        F = rhs4_padded(ev("f", P), hh)          # f^(IV) from exact f samples, one layer beyond
        return np.abs(AU - F).max()
    dk2 = (ev("k2x", C), ev("k2y", C), ev("k2z", C))
    AU = apply_A6(Up, Kp, dk2, ev("lapk2", C), hh)
    F = rhs6(ev("f", C), ev("lapf", C), ev("sum4f", C), ev("mixf", C), (ev("fx", C), ev("fy", C), ev("fz", C)),
             ev("k2", C), dk2, hh)
    return np.abs(AU - F).max()


@pytest.mark.parametrize("order", [4, 6])
def test_truncation_order_variable_k(order):
    ev = _smooth_fields()
    e = [_truncation(order, h, ev) for h in (0.08, 0.04, 0.02)]
    slopes = [math.log2(e[i] / e[i + 1]) for i in range(2)]
    assert min(slopes) > order - 0.15, slopes


# ---- global convergence on the manufactured solution (Sec. 5.1) -----------------------------
def _manufactured_rhs(order, g, k0):
    """F of the compact scheme from the analytic f: f^(IV) = (1 + sum h^2/12 delta^2) f with f sampled one
    node outside the grid (Eq. scheme4), or f^(VI) of Eq. scheme6 from the analytic derivatives."""
    X, Y, Z = g.mesh()
    k2 = np.full(g.shape, k0 * k0, dtype=complex)
    zero = (np.zeros(g.shape, complex),) * 3
    if order == 6:
        f, lapf, sum4, mix, df = mf.rhs6_fields(X, Y, Z, k0)
        return rhs6(f, lapf, sum4, mix, df, k2, zero, g.h)
    ax = [np.arange(-1, n + 1) * hd for n, hd in zip(g.n, g.h)]
    Zp, Yp, Xp = np.meshgrid(ax[2], ax[1], ax[0], indexing="ij")
    return rhs4_padded(mf.f_exact(Xp, Yp, Zp, k0), g.h)


def _const_operator(g, k0, order, rule):
    zero = (np.zeros(g.shape, complex),) * 3
    return Operator(g, np.full(g.shape, k0 * k0, dtype=complex), k0, order, rule=rule, dk2=zero,
                    lapk2=np.zeros(g.shape, complex))


def _manufactured_error(order, N):
    k0 = 8.0
    g = Grid(N, N, N, staggered=False)
    X, Y, Z = g.mesh()
    u = mf.u_exact(X, Y, Z, k0)
    op = _const_operator(g, k0, order, "zero")
    # exact ghost values (Dirichlet data of the closure-free test) move to the right-hand side
    ax = np.arange(-1, N + 1) * g.h[0]
    Zp, Yp, Xp = np.meshgrid(ax, ax, ax, indexing="ij")
    ughost = mf.u_exact(Xp, Yp, Zp, k0)
    ughost[1:-1, 1:-1, 1:-1] = 0
    F = _manufactured_rhs(order, g, k0)
    e = EigT(g, k0)
    U, info = gmres(op, e.apply_Minv, (F - op.apply_padded(ughost)).ravel(), m=30, rtol=1e-13, max_it=300)
    return metrics.l2_err(u, U.reshape(g.shape))


@pytest.mark.parametrize("order", [4, 6])
def test_manufactured_convergence_order(order):
    errs = [_manufactured_error(order, N) for N in (9, 17, 33)]
    slope = math.log2(errs[1] / errs[2])
    assert slope > order - 0.3, errs


# ---- high-order ABC closure on collocated grids (oracle/closure.py) --------------------------
def test_closure_without_taylor_terms_is_the_three_point_rule():
    g = Grid(7, 6, 5, staggered=False)
    U = _rand(g.shape, 11)
    ref = Operator(g, np.ones(g.shape), 5.0, 2, rule="collocated3").pad(U)
    assert np.allclose(pad_ghost_ho(U, 5.0, g.h, terms=0), ref, rtol=0, atol=1e-13)


def test_closure_ghosts_of_the_exact_solution_are_seventh_order():
    k0 = 9.0
    fdiff = lambda X, Y, Z, d: mf.f_exact(X, Y, Z, k0, *d)
    errs = []
    for N in (17, 33):
        g = Grid(N, N, N, staggered=False)
        X, Y, Z = g.mesh()
        ax = np.arange(-1, N + 1) * g.h[0]
        Zp, Yp, Xp = np.meshgrid(ax, ax, ax, indexing="ij")
        P = pad_ghost_ho(mf.u_exact(X, Y, Z, k0), k0, g.h, fdiff=fdiff)
        errs.append(np.abs(P - mf.u_exact(Xp, Yp, Zp, k0)).max())
    assert math.log2(errs[0] / errs[1]) > 6.5, errs


@pytest.mark.parametrize("order", [4, 6])
def test_closure_keeps_the_scheme_order(order):
    """With the closure, the global error falls at the scheme's order (4.0 and 6.0 measured) on a resolved
    manufactured problem: the boundary rows do not lower it."""
    k0 = 8.0
    errs = []
    for N in (17, 33):
        g = Grid(N, N, N, staggered=False)
        X, Y, Z = g.mesh()
        op = _const_operator(g, k0, order, "collocated_ho")
        ghost_f = pad_ghost_ho(np.zeros(g.shape, complex), k0, g.h,
                               fdiff=lambda X, Y, Z, d: mf.f_exact(X, Y, Z, k0, *d))
        b = (_manufactured_rhs(order, g, k0) - op.apply_padded(ghost_f)).ravel()
        U, _ = gmres(op, EigT(g, k0).apply_Minv, b, m=30, rtol=1e-13, max_it=300)
        errs.append(metrics.l2_err(mf.u_exact(X, Y, Z, k0), U.reshape(g.shape)))
    assert math.log2(errs[0] / errs[1]) > order - 0.2, errs


@pytest.mark.parametrize("row", [r for r in high_order_rows() if r[1] <= 127], ids=lambda r: f"o{r[0]}n{r[1]}")
def test_paper_high_order_errors_and_iterations(row):
    """Tables tab:fourth_order_results / tab:sixth_order_results: the compact schemes with the high-order
    closure, EigT3-preconditioned GMRES(20) to rel-res 1e-10 from x0 = 0."""
    order, N, me_text, l2_paper, n0_paper = row
    g = Grid(N, N, N, staggered=False)
    X, Y, Z = g.mesh()
    u = mf.u_exact(X, Y, Z, K0_PAPER)
    op = _const_operator(g, K0_PAPER, order, "collocated_ho")
    fdiff = lambda X, Y, Z, d: mf.f_exact(X, Y, Z, K0_PAPER, *d)
    ghost_f = pad_ghost_ho(np.zeros(g.shape, complex), K0_PAPER, g.h, fdiff=fdiff)
    b = (_manufactured_rhs(order, g, K0_PAPER) - op.apply_padded(ghost_f)).ravel()
    U, info = gmres(op, EigT(g, K0_PAPER).apply_Minv, b, m=20, rtol=1e-10, max_it=200)
    U = U.reshape(g.shape)
    assert info["converged"]
    me, l2 = metrics.max_err(u, U), metrics.l2_err(u, U)
    me_paper = float(me_text)
    # the closure is our reading: the L2 error (a volume average) must agree to 2%, the pointwise maximum,
    # which sits next to the boundary, to 5% or the printed rounding
    assert abs(l2 - l2_paper) <= 0.02 * l2_paper, (l2, l2_paper)
    assert abs(me - me_paper) <= max(0.05 * me_paper, printed_half_unit(me_text)), (me, me_paper)
    # N0: the paper counts MATLAB's iterations, we count Arnoldi steps until the true residual is 1e-10
    assert n0_paper <= info["iterations"] <= n0_paper + 5, (info["iterations"], n0_paper)


def test_paper_high_order_iterations_do_not_grow_with_the_grid():
    """The property the paper highlights after the high-order tables: N0 falls as the grid is refined."""
    its = []
    for N in (33, 65):
        g = Grid(N, N, N, staggered=False)
        op = _const_operator(g, K0_PAPER, 4, "collocated_ho")
        fdiff = lambda X, Y, Z, d: mf.f_exact(X, Y, Z, K0_PAPER, *d)
        ghost_f = pad_ghost_ho(np.zeros(g.shape, complex), K0_PAPER, g.h, fdiff=fdiff)
        b = (_manufactured_rhs(4, g, K0_PAPER) - op.apply_padded(ghost_f)).ravel()
        its.append(gmres(op, EigT(g, K0_PAPER).apply_Minv, b, m=20, rtol=1e-10, max_it=200)[1]["iterations"])
    assert its[1] < its[0], its


# ---- high-order operators: GMRES + EigT solves the assembled system (8^3) -------------------
@pytest.mark.parametrize("order", [4, 6])
def test_gmres_matches_dense_solve(order):
    g = Grid(8, 8, 8, staggered=True)
    X, Y, Z = g.mesh()
    k0 = 9.0
    k2 = k0 * k0 * (1 + 0.25 * np.exp(-((X - .5) ** 2 + (Y - .45) ** 2 + (Z - .55) ** 2) / 0.05)) + 0j
    A = Operator(g, k2, k0, order)
    b = _rand(g.shape, 6)
    xd = np.linalg.solve(A.dense(), b.ravel())
    for flexible in (False, True):
        x, info = gmres(A, EigT(g, k0).apply_Minv, b, m=4, rtol=1e-13, max_it=200, flexible=flexible)
        assert info["converged"] and info["iterations"] > 4 and info["restarts"] > 1
        assert np.abs(x - xd).max() <= 1e-10 * np.abs(xd).max()


# ---- sampled-data derivative readings converge (Eq. scheme6 readings) -----------------------
def test_sampled_rhs6_matches_analytic_in_interior():
    k0 = 6.0
    errs = []
    for N in (24, 48):
        g = Grid(N, N, N, staggered=True)
        X, Y, Z = g.mesh()
        k2 = np.full(g.shape, k0 * k0, complex)
        zero = (np.zeros(g.shape, complex),) * 3
        f, lapf, sum4, mix, df = mf.rhs6_fields(X, Y, Z, k0)
        Fa = rhs6(f, lapf, sum4, mix, df, k2, zero, g.h)
        Fs = rhs6_sampled(f, k2, zero, True, g.h)
        s = slice(N // 4, 3 * N // 4)
        errs.append(np.abs(Fa - Fs)[s, s, s].max() / np.abs(Fa).max())
    assert math.log2(errs[0] / errs[1]) > 5.6, errs


# ---- golden: Table tab:scattering_results (EigT2 iteration counts) ------------------------------
def _golden_scatter():
    rows = []
    with open(os.path.join(GOLDEN, "scattering_table.txt")) as fh:
        for line in fh:
            if line.strip() and not line.startswith("#"):
                n, n0 = line.split()
                rows.append((int(n), int(n0)))
    return rows


@pytest.mark.parametrize("row", [r for r in _golden_scatter() if r[0] <= 127])
def test_paper_scattering_iterations(row):
    """The oracle's sixth-order GMRES(20) + EigT2 on the Sec. 5.2 inclusion reaches rel-res 1e-8 in the
    printed number of inner iterations at 100^3 and 127^3 (the larger grids take minutes on a CPU)."""
    N, n0_paper = row
    g = Grid(N, N, N, staggered=True)
    X, Y, Z = g.mesh()
    k02 = 439.2
    inside = (X - 0.5) ** 2 + (Y - 0.5) ** 2 + (Z - 0.7) ** 2 <= 0.1 ** 2
    k2 = np.where(inside, 1050 + 2.26j, k02 + 0j)
    k0 = math.sqrt(k02)
    f = -(k2 - k02) * np.exp(1j * k0 * Z)
    dk2, _ = derived_k2_fields(k2, True, g.h)
    F = rhs6_sampled(f, k2, dk2, True, g.h)
    A = Operator(g, k2, k0, 6)
    x, info = gmres(A, EigT(g, k0).apply_Minv, F, m=20, rtol=1e-8, max_it=100)
    assert info["converged"] and info["iterations"] == n0_paper
    assert np.linalg.norm(A(x.reshape(g.shape)) - F) / np.linalg.norm(F) <= 1e-8
