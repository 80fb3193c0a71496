"""Modified right-hand sides of the compact schemes.

rhs4:  f^(IV) = (1 + sum_alpha h_alpha^2/12 delta_alpha^2) f                 (Eq. scheme4)
rhs6:  f^(VI) - h^2/20 [k^2 f - h^2/3 sum_d (k^2)_d f_d]                        (Eq. scheme6)
       f^(VI) = f + h^2/12 lap f + h^4/360 (f_xxxx + f_yyyy + f_zzzz) + h^4/90 (f_xxyy + f_xxzz + f_yyzz)
The k^2 f and f_d parts come from Delta_h(k^2 U) of Eq. scheme6, which do not involve U.
Our reading: "nabla^4 f" of Eq. scheme6 is the sum of pure fourth derivatives; with this
reading (and only with it) the scheme has sixth-order truncation error.
"""

from .operators import pad_coef


def rhs4_padded(FP, h):
    """f^(IV) from f given on the unknowns plus one ghost layer (FP)."""
    c = FP[1:-1, 1:-1, 1:-1]
    out = c.copy()
    for axis in range(3):
        sl_p = [slice(1, -1)] * 3
        sl_m = [slice(1, -1)] * 3
        ax = 2 - axis
        sl_p[ax] = slice(2, None)
        sl_m[ax] = slice(0, -2)
        out = out + h[axis] ** 2 / 12.0 * (FP[tuple(sl_p)] - 2.0 * c + FP[tuple(sl_m)]) / h[axis] ** 2
    return out


def rhs4_sampled(f, staggered, h):
    """f^(IV) from samples of f; the ghost layer is the mirror extension (reading)."""
    return rhs4_padded(pad_coef(f, staggered, 1), h)


def rhs6(f, lapf, sum4f, mixf, df, k2, dk2, h):
    """Right-hand side of Eq. scheme6 from f and its derivative fields (analytic or sampled)."""
    hh = h[0]
    h2 = hh * hh
    F = f + h2 / 12.0 * lapf + h2 * h2 / 360.0 * sum4f + h2 * h2 / 90.0 * mixf
    F = F - h2 / 20.0 * (k2 * f - h2 / 3.0 * (dk2[0] * df[0] + dk2[1] * df[1] + dk2[2] * df[2]))
    return F


def f_derivative_fields(f, staggered, h):
    """Sampled-data reading of the derivatives of f in Eq. scheme6 (our reading): lap f by fourth-order
    five-point differences; pure fourth derivatives by delta^4; mixed ones by delta^2 delta^2;
    f_d by delta_d.  Two mirror layers.  Returns (lapf, sum4f, mixf, (fx, fy, fz))."""
    Q = pad_coef(f, staggered, width=2)
    nz, ny, nx = f.shape

    def sh(a, b, c):
        return Q[2 + c:2 + c + nz, 2 + b:2 + b + ny, 2 + a:2 + a + nx]

    def at(axis, s, axis2=None, s2=0):
        o = [0, 0, 0]
        o[axis] = s
        if axis2 is not None:
            o[axis2] = s2
        return sh(*o)

    lap = 0.0
    sum4 = 0.0
    df = []
    for axis in range(3):
        hd = h[axis]
        lap = lap + (-at(axis, 2) + 16 * at(axis, 1) - 30 * at(axis, 0) + 16 * at(axis, -1) - at(axis, -2)) / (12 * hd * hd)
        sum4 = sum4 + (at(axis, 2) - 4 * at(axis, 1) + 6 * at(axis, 0) - 4 * at(axis, -1) + at(axis, -2)) / hd ** 4
        df.append((at(axis, 1) - at(axis, -1)) / (2 * hd))
    w = {-1: 1.0, 0: -2.0, 1: 1.0}
    mix = 0.0
    for a1, a2 in ((0, 1), (0, 2), (1, 2)):
        acc = 0.0
        for s1, c1 in w.items():
            for s2, c2 in w.items():
                acc = acc + c1 * c2 * at(a1, s1, a2, s2)
        mix = mix + acc / (h[a1] ** 2 * h[a2] ** 2)
    return lap, sum4, mix, tuple(df)


def rhs6_sampled(f, k2, dk2, staggered, h):
    lapf, sum4f, mixf, df = f_derivative_fields(f, staggered, h)
    return rhs6(f, lapf, sum4f, mixf, df, k2, dk2, h)
