"""The separable test solution of Sec. 5.1: u = phi(x) phi(y) phi(z) on the unit cube,
phi(x) = exp(i k0 (x - a)) + exp(-i k0 (x - b)) - 2, a = 0, b = 1 (k0^2 = 439.2 in the paper).

phi'' = -k0^2 (phi + 2), so f = lap u + k0^2 u = -2 k0^2 [u + phi_y phi_z + phi_x phi_z + phi_x phi_y].
f is written as a sum of separable terms g_x(x) g_y(y) g_z(z) with g in {phi, 1}; its derivatives are
the products of the one-dimensional derivatives (analytic fields for Eq. scheme6).
"""
import numpy as np


def phi_deriv(x, k0, n, a=0.0, b=1.0):
    """n-th derivative of phi."""
    v = (1j * k0) ** n * np.exp(1j * k0 * (x - a)) + (-1j * k0) ** n * np.exp(-1j * k0 * (x - b))
    if n == 0:
        v = v - 2.0
    return v


def _one(x, n):
    return np.ones_like(x, dtype=np.complex128) if n == 0 else np.zeros_like(x, dtype=np.complex128)


def _terms(k0):
    # f = -2 k0^2 [phi phi phi + 1 phi phi + phi 1 phi + phi phi 1]
    P = lambda x, n: phi_deriv(x, k0, n)
    return [(P, P, P), (_one, P, P), (P, _one, P), (P, P, _one)], -2.0 * k0 * k0


def _sep(X, Y, Z, terms, coef, nx, ny, nz):
    out = 0.0
    for gx, gy, gz in terms:
        out = out + gx(X, nx) * gy(Y, ny) * gz(Z, nz)
    return coef * out


def u_exact(X, Y, Z, k0):
    return phi_deriv(X, k0, 0) * phi_deriv(Y, k0, 0) * phi_deriv(Z, k0, 0)


def f_exact(X, Y, Z, k0, dx=0, dy=0, dz=0):
    terms, coef = _terms(k0)
    return _sep(X, Y, Z, terms, coef, dx, dy, dz)


def rhs6_fields(X, Y, Z, k0):
    """(f, lap f, sum of pure 4th derivatives, mixed 4th sum, (f_x, f_y, f_z)) analytically."""
    F = lambda a, b, c: f_exact(X, Y, Z, k0, a, b, c)
    lap = F(2, 0, 0) + F(0, 2, 0) + F(0, 0, 2)
    sum4 = F(4, 0, 0) + F(0, 4, 0) + F(0, 0, 4)
    mix = F(2, 2, 0) + F(2, 0, 2) + F(0, 2, 2)
    return F(0, 0, 0), lap, sum4, mix, (F(1, 0, 0), F(0, 1, 0), F(0, 0, 1))
