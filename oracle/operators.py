"""The high-order operator A of the compact schemes, with the boundary ghosts eliminated.

Plain slice arithmetic on a grid padded with one ghost layer.  Each difference operator is the
central difference of Sec. 2.1 (delta_x, delta_x^2) applied to a padded grid function; products
of operators are products of the one-dimensional weight sets.

Ghost rules (how the layer outside the unknowns is filled):
  'staggered'   Eq. D_bc: U_0 = gamma U_1, U_{N+1} = gamma U_N, per direction; an edge or corner
                ghost therefore carries the product of the gammas (our reading of the corner).
  'collocated3' second-order three-point closure of the ABC on a collocated grid: the central
                difference of du/dn - i k0 u = 0 at the boundary node gives U_0 = U_2 + 2 i k0 h U_1
                (this is the Lambda-bar corner gamma = 2 i k0 h, zeta = 2 of Sec. 4.1).
  'collocated_ho' the high-order closure of oracle/closure.py (manufactured-solution tests, collocated).
  'zero'        the ghost layer stays zero; the caller moves known ghost values to the right-hand side.
Coefficient fields (k^2, f) are extended by mirror symmetry: about the face for staggered grids,
about the boundary node for collocated grids (zero-gradient extension; reading).
"""
import numpy as np

from .closure import pad_ghost_ho


def pad_ghost(U, rule, gammas=None, k0=None, h=None):
    """Return U with one ghost layer on every face, filled per `rule` (x, then y, then z)."""
    nz, ny, nx = U.shape
    P = np.zeros((nz + 2, ny + 2, nx + 2), dtype=np.complex128)
    P[1:-1, 1:-1, 1:-1] = U
    if rule == "staggered":
        gx, gy, gz = gammas
        P[1:-1, 1:-1, 0] = gx * P[1:-1, 1:-1, 1]
        P[1:-1, 1:-1, -1] = gx * P[1:-1, 1:-1, -2]
        P[1:-1, 0, :] = gy * P[1:-1, 1, :]
        P[1:-1, -1, :] = gy * P[1:-1, -2, :]
        P[0, :, :] = gz * P[1, :, :]
        P[-1, :, :] = gz * P[-2, :, :]
    elif rule == "collocated3":
        hx, hy, hz = h
        P[1:-1, 1:-1, 0] = P[1:-1, 1:-1, 2] + 2j * k0 * hx * P[1:-1, 1:-1, 1]
        P[1:-1, 1:-1, -1] = P[1:-1, 1:-1, -3] + 2j * k0 * hx * P[1:-1, 1:-1, -2]
        P[1:-1, 0, :] = P[1:-1, 2, :] + 2j * k0 * hy * P[1:-1, 1, :]
        P[1:-1, -1, :] = P[1:-1, -3, :] + 2j * k0 * hy * P[1:-1, -2, :]
        P[0, :, :] = P[2, :, :] + 2j * k0 * hz * P[1, :, :]
        P[-1, :, :] = P[-3, :, :] + 2j * k0 * hz * P[-2, :, :]
    elif rule == "zero":
        pass
    else:
        raise ValueError(rule)
    return P


def pad_coef(c, staggered, width=1):
    """Mirror extension of a coefficient field (k^2 or f) by `width` layers."""
    mode = "symmetric" if staggered else "reflect"
    return np.pad(np.asarray(c, dtype=np.complex128), width, mode=mode)


def _S(P, a, b, c):
    """Interior view of a one-layer-padded array shifted by (a, b, c) in (x, y, z)."""
    nz, ny, nx = P.shape
    return P[1 + c:nz - 1 + c, 1 + b:ny - 1 + b, 1 + a:nx - 1 + a]


_W2 = {-1: 1.0, 0: -2.0, 1: 1.0}   # delta^2 weights (times 1/h^2)
_W1 = {-1: -0.5, 1: 0.5}           # delta weights   (times 1/h)


def _apply(P, wsets):
    """Sum over offsets of the product of 1D weight sets; wsets = (wx, wy, wz) dicts or None."""
    wx, wy, wz = [w if w is not None else {0: 1.0} for w in wsets]
    out = 0.0
    for a, ca in wx.items():
        for b, cb in wy.items():
            for c, cc in wz.items():
                out = out + (ca * cb * cc) * _S(P, a, b, c)
    return out


def d2(P, axis, h):
    w = [None, None, None]
    w[axis] = _W2
    return _apply(P, w) / h[axis] ** 2


def d2d2(P, ax1, ax2, h):
    w = [None, None, None]
    w[ax1] = _W2
    w[ax2] = _W2
    return _apply(P, w) / (h[ax1] ** 2 * h[ax2] ** 2)


def d2d2d2(P, h):
    return _apply(P, [_W2, _W2, _W2]) / (h[0] * h[1] * h[2]) ** 2


def d1(P, axis, h):
    w = [None, None, None]
    w[axis] = _W1
    return _apply(P, w) / h[axis]


def d1d2(P, axis, ax2, h):
    """delta_axis delta_ax2^2."""
    w = [None, None, None]
    w[axis] = _W1
    w[ax2] = _W2
    return _apply(P, w) / (h[axis] * h[ax2] ** 2)


def apply_A2(P, K2P, h):
    """Second-order operator (delta_x^2 + delta_y^2 + delta_z^2 + k^2) on padded U (P) and k^2 (K2P)."""
    return d2(P, 0, h) + d2(P, 1, h) + d2(P, 2, h) + _S(K2P, 0, 0, 0) * _S(P, 0, 0, 0)


def apply_A4(P, K2P, h):
    """Fourth-order compact scheme, left side of Eq. scheme4.

    (dxx+dyy+dzz)U + (hx^2+hy^2)/12 dxx dyy U + (hx^2+hz^2)/12 dxx dzz U + (hy^2+hz^2)/12 dyy dzz U
    + (1 + hx^2/12 dxx + hy^2/12 dyy + hz^2/12 dzz)(k^2 U), every operator acting on the padded
    grid function; k^2 U at a ghost is k^2(mirror) * U(ghost).
    """
    hx, hy, hz = h
    KU = K2P * P
    out = d2(P, 0, h) + d2(P, 1, h) + d2(P, 2, h)
    out = out + (hx**2 + hy**2) / 12.0 * d2d2(P, 0, 1, h)
    out = out + (hx**2 + hz**2) / 12.0 * d2d2(P, 0, 2, h)
    out = out + (hy**2 + hz**2) / 12.0 * d2d2(P, 1, 2, h)
    out = out + _S(KU, 0, 0, 0)
    out = out + hx**2 / 12.0 * d2(KU, 0, h) + hy**2 / 12.0 * d2(KU, 1, h) + hz**2 / 12.0 * d2(KU, 2, h)
    return out


def apply_A6(P, K2P, dk2, lapk2, h):
    """Sixth-order compact scheme, U-dependent part of the left side of Eq. scheme6 (uniform h).

    L_h[(1 + h^2 k^2/30) U] + h^4/30 dxx dyy dzz U + k^2 U + h^2/6 M_h[(1 + h^2 k^2/15) U]
    + h^2/20 { (lap k^2 - k^4) U + 2 sum_d (k^2)_d ( delta_d[(1 + h^2 k^2/6) U] + h^2/6 delta_d T_d U ) }
    with L_h = sum delta^2, M_h = dxx dyy + dxx dzz + dyy dzz, T_x = dyy + dzz (cyclic).
    Our readings: the difference operators act on the product grid functions k^2 U (the
    notation of Eq. scheme4); the (lap k^2 - k^4) term multiplies U; k^2 f and the f_d parts of
    Delta_h(k^2 U) are U-independent and live in the right-hand side (rhs.rhs6).
    dk2 = (k2_x, k2_y, k2_z) and lapk2 are given at the unknowns.
    """
    hh = h[0]
    assert abs(h[1] - hh) < 1e-14 * hh and abs(h[2] - hh) < 1e-14 * hh, "scheme6 needs uniform h"
    h2 = hh * hh
    Kc = _S(K2P, 0, 0, 0)
    Uc = _S(P, 0, 0, 0)
    P30 = (1.0 + h2 * K2P / 30.0) * P
    P15 = (1.0 + h2 * K2P / 15.0) * P
    P6 = (1.0 + h2 * K2P / 6.0) * P
    out = d2(P30, 0, h) + d2(P30, 1, h) + d2(P30, 2, h)
    out = out + h2 * h2 / 30.0 * d2d2d2(P, h)
    out = out + Kc * Uc
    out = out + h2 / 6.0 * (d2d2(P15, 0, 1, h) + d2d2(P15, 0, 2, h) + d2d2(P15, 1, 2, h))
    grad = 0.0
    for d in range(3):
        o1, o2 = [a for a in range(3) if a != d]
        inner = d1(P6, d, h) + h2 / 6.0 * (d1d2(P, d, o1, h) + d1d2(P, d, o2, h))
        grad = grad + 2.0 * dk2[d] * inner
    out = out + h2 / 20.0 * ((lapk2 - Kc * Kc) * Uc + grad)
    return out


def derived_k2_fields(k2, staggered, h):
    """Sampled-data reading of the continuous derivatives of k^2 in Eq. scheme6 (our reading):
    fourth-order five-point central differences with two mirror layers.  Returns (dk2, lapk2)."""
    Q = pad_coef(k2, staggered, width=2)
    nz, ny, nx = k2.shape

    def sh(a, b, c):
        return Q[2 + c:2 + c + nz, 2 + b:2 + b + ny, 2 + a:2 + a + nx]

    dk2 = []
    lap = 0.0
    for axis in range(3):
        off = [0, 0, 0]

        def at(s):
            o = list(off)
            o[axis] = s
            return sh(*o)

        hd = h[axis]
        dk2.append((-at(2) + 8.0 * at(1) - 8.0 * at(-1) + at(-2)) / (12.0 * hd))
        lap = lap + (-at(2) + 16.0 * at(1) - 30.0 * at(0) + 16.0 * at(-1) - at(-2)) / (12.0 * hd * hd)
    return tuple(dk2), lap


class Operator:
    """A for one problem: grid, k^2 samples, background k0, scheme order, ghost rule."""

    def __init__(self, grid, k2, k0, order, rule=None, dk2=None, lapk2=None):
        self.grid = grid
        self.k2 = np.asarray(k2, dtype=np.complex128)
        self.k0 = k0
        self.order = order
        self.rule = rule or ("staggered" if grid.staggered else "collocated3")
        h = grid.h
        self.gammas = tuple((2.0 + 1j * k0 * hd) / (2.0 - 1j * k0 * hd) for hd in h)
        self.K2P = pad_coef(self.k2, grid.staggered)
        if order == 6:
            if dk2 is None:
                dk2, lapk2 = derived_k2_fields(self.k2, grid.staggered, h)
            self.dk2, self.lapk2 = dk2, lapk2

    def pad(self, U):
        if self.rule == "collocated_ho":
            return pad_ghost_ho(U, self.k0, self.grid.h)
        return pad_ghost(U, self.rule, gammas=self.gammas, k0=self.k0, h=self.grid.h)

    def apply_padded(self, P):
        h = self.grid.h
        if self.order == 2:
            return apply_A2(P, self.K2P, h)
        if self.order == 4:
            return apply_A4(P, self.K2P, h)
        if self.order == 6:
            return apply_A6(P, self.K2P, self.dk2, self.lapk2, h)
        raise ValueError(self.order)

    def __call__(self, U):
        U = np.asarray(U, dtype=np.complex128).reshape(self.grid.shape)
        return self.apply_padded(self.pad(U))

    def dense(self):
        """Assemble A column by column (small grids only)."""
        N = self.grid.unknowns
        M = np.zeros((N, N), dtype=np.complex128)
        e = np.zeros(N, dtype=np.complex128)
        for c in range(N):
            e[:] = 0
            e[c] = 1
            M[:, c] = self(e).ravel()
        return M
