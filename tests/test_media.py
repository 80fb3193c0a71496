"""The seeded input generators (paper_2602_07711_gb300/media.py) against the problem definitions the paper
fixes and the oracle restates (CPU only).  The generators hold no solver arithmetic; these checks make sure
that the GPU tests and the oracle see the same problems."""
import math

import numpy as np
import pytest

pytest.importorskip("torch")

from oracle import manufactured as mf
from oracle.grid import Grid
from paper_2602_07711_gb300 import media

K0 = math.sqrt(439.2)


@pytest.mark.parametrize("order", [4, 6])
def test_manufactured_problem_matches_the_oracle_definition(order):
    n = 11
    d = media.manufactured(n, K0, order)
    g = Grid(n, n, n, staggered=False)
    X, Y, Z = g.mesh()
    assert np.allclose(d["u"], mf.u_exact(X, Y, Z, K0), rtol=0, atol=1e-12)
    if order == 4:
        ax = np.arange(-1, n + 1) * g.h[0]
        Zp, Yp, Xp = np.meshgrid(ax, ax, ax, indexing="ij")
        assert np.allclose(d["fields"], mf.f_exact(Xp, Yp, Zp, K0), rtol=0, atol=1e-9)
    else:
        f, lapf, s4, mix, df = mf.rhs6_fields(X, Y, Z, K0)
        ref = np.stack([f, lapf, s4, mix, df[0], df[1], df[2]])
        assert np.abs(d["fields"] - ref).max() <= 1e-12 * np.abs(ref).max()


def test_manufactured_solution_satisfies_the_abc_and_the_equation():
    """Sec. 5.1: u = phi(x) phi(y) phi(z) meets du/dn = i k0 u on every face, and lap u + k0^2 u = f."""
    k0 = 7.0
    x = np.linspace(0.0, 1.0, 9)
    eps = 1e-5
    # d phi/dx at x = 0 (outward normal -x) and x = 1 (outward normal +x), by central differences
    phi = lambda t: media._phi(t, k0, 0)
    d0 = (phi(eps) - phi(-eps)) / (2 * eps)
    d1 = (phi(1 + eps) - phi(1 - eps)) / (2 * eps)
    assert abs(-d0 - 1j * k0 * phi(0.0)) < 1e-6 * k0
    assert abs(d1 - 1j * k0 * phi(1.0)) < 1e-6 * k0
    Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
    u = lambda a, b, c: media._phi(a, k0, 0) * media._phi(b, k0, 0) * media._phi(c, k0, 0)
    h = 1e-3
    lap = sum((u(*[X + h * (q == 0), Y + h * (q == 1), Z + h * (q == 2)]) - 2 * u(X, Y, Z)
               + u(*[X - h * (q == 0), Y - h * (q == 1), Z - h * (q == 2)])) / h ** 2 for q in range(3))
    f = media._f_deriv(X, Y, Z, k0, 0, 0, 0)
    assert np.abs(lap + k0 * k0 * u(X, Y, Z) - f).max() <= 1e-4 * np.abs(f).max()


def test_face_data_layout_matches_the_closure():
    """helm_closure_rhs reads, per axis x, y, z and side near/far, three fields over the face: x faces
    N_z x N_y, y faces N_z x (N_x + 2), z faces (N_y + 2) x (N_x + 2)."""
    n = 9
    d = media.manufactured(n, K0, 6)
    per = [n * n, n * (n + 2), (n + 2) * (n + 2)]
    assert d["faces"].size == sum(2 * 3 * p for p in per)
    # first block: f_x on the x = 0 face at interior (z, y) nodes
    g = Grid(n, n, n, staggered=False)
    X, Y, Z = g.mesh()
    fx0 = mf.f_exact(np.zeros_like(X[:, :, 0]), Y[:, :, 0], Z[:, :, 0], K0, 1, 0, 0)
    assert np.allclose(d["faces"][:n * n].reshape(n, n), fx0, rtol=1e-13, atol=0)
