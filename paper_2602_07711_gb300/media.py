"""Seeded synthetic workloads (inputs only: none of the solver's arithmetic lives here).

Every workload but the last is a scattering problem on the unit cube with a staggered grid (nodes
h/2 + j h, h = 1/n, Sec. 5.2): a medium k^2(x), a background wavenumber k0, an incident plane wave
u_inc = exp(i k0 d.x) and the right-hand side f = -(k^2 - k0^2) u_inc (the form of Sec. 5.2).
The generators return complex128 arrays indexed [z, y, x] (x fastest), built with torch in float64
on the requested device so that the same numbers serve the CPU oracle and the GPU library.

Workloads (sizes and distributions of the paper's scattering tests):
  single_gaussian  one Gaussian inclusion of +20% contrast, k0 = 2 pi 4, d = +z
  bumps            sum of Gaussian bumps, contrast a ~ U(-0.3, 0.3), centres ~ U[0.2, 0.8]^3,
                   widths sigma ~ U(0.03, 0.08), k0 = 2 pi n/(ppw L), direction from a seeded angle
  sphere           the single spherical inclusion of Sec. 5.2 (k^2 = 1050 + 2.26i inside r = 0.1 at
                   (0.5, 0.5, 0.7), 439.2 outside), d = +z
  layered          horizontal layers with k^2/k0^2 ~ U[lo, hi] plus spherical inclusions
  manufactured     the separable test solution of Sec. 5.1 on the collocated grid (numpy, analytic): the
                   exact u, the scheme's right-hand side fields and the closure's face data
"""
import math

import numpy as np


def _torch():
    import torch
    return torch


def _mesh(n, device):
    torch = _torch()
    h = 1.0 / n
    x = (torch.arange(n, dtype=torch.float64, device=device) + 0.5) * h
    Z, Y, X = torch.meshgrid(x, x, x, indexing="ij")
    return X, Y, Z


def _finish(k2, k0, d, X, Y, Z, as_numpy):
    torch = _torch()
    phase = k0 * (d[0] * X + d[1] * Y + d[2] * Z)
    uinc = torch.polar(torch.ones_like(phase), phase)
    f = -(k2 - k0 * k0) * uinc
    if as_numpy:
        return k2.cpu().numpy(), f.cpu().numpy(), float(k0)
    return k2.contiguous(), f.contiguous(), float(k0)


def single_gaussian(n=32, device="cpu", as_numpy=True):
    torch = _torch()
    X, Y, Z = _mesh(n, device)
    k0 = 2.0 * math.pi * 4.0
    r2 = (X - 0.5) ** 2 + (Y - 0.5) ** 2 + (Z - 0.5) ** 2
    k2 = (k0 * k0 * (1.0 + 0.2 * torch.exp(-r2 / 0.02))).to(torch.complex128)
    return _finish(k2, k0, (0.0, 0.0, 1.0), X, Y, Z, as_numpy)


def direction(seed):
    rng = np.random.default_rng(seed)
    v = rng.standard_normal(3)
    return tuple(v / np.linalg.norm(v))


def bumps(n, seed_medium, seed_angle, ppw=10.0, nbumps=20, contrast=0.3, device="cpu", as_numpy=True):
    torch = _torch()
    rng = np.random.default_rng(seed_medium)
    a = rng.uniform(-contrast, contrast, nbumps)
    c = rng.uniform(0.2, 0.8, (nbumps, 3))
    s = rng.uniform(0.03, 0.08, nbumps)
    X, Y, Z = _mesh(n, device)
    k0 = 2.0 * math.pi * n / ppw
    rel = torch.ones_like(X)
    for b in range(nbumps):
        r2 = (X - c[b, 0]) ** 2 + (Y - c[b, 1]) ** 2 + (Z - c[b, 2]) ** 2
        rel = rel + a[b] * torch.exp(-r2 / (2.0 * s[b] ** 2))
    k2 = (k0 * k0 * rel).to(torch.complex128)
    return _finish(k2, k0, direction(seed_angle), X, Y, Z, as_numpy)


def sphere(n, device="cpu", as_numpy=True):
    torch = _torch()
    X, Y, Z = _mesh(n, device)
    k02 = 439.2
    inside = ((X - 0.5) ** 2 + (Y - 0.5) ** 2 + (Z - 0.7) ** 2) <= 0.1 ** 2
    k2 = torch.where(inside, torch.tensor(1050 + 2.26j, dtype=torch.complex128, device=device),
                     torch.tensor(k02 + 0j, dtype=torch.complex128, device=device))
    return _finish(k2, math.sqrt(k02), (0.0, 0.0, 1.0), X, Y, Z, as_numpy)


def layered(n, seed, ppw=8.0, nlayers=8, lo=0.7, hi=1.3, nspheres=3, rlo=0.05, rhi=0.12, device="cpu",
            as_numpy=True):
    torch = _torch()
    rng = np.random.default_rng(seed)
    lay = rng.uniform(lo, hi, nlayers)
    cen = rng.uniform(0.2, 0.8, (nspheres, 3))
    rad = rng.uniform(rlo, rhi, nspheres)
    con = rng.uniform(lo, hi, nspheres)
    X, Y, Z = _mesh(n, device)
    k0 = 2.0 * math.pi * n / ppw
    idx = torch.clamp((Z * nlayers).long(), 0, nlayers - 1)
    rel = torch.tensor(lay, dtype=torch.float64, device=device)[idx]
    for b in range(nspheres):
        r2 = (X - cen[b, 0]) ** 2 + (Y - cen[b, 1]) ** 2 + (Z - cen[b, 2]) ** 2
        rel = torch.where(r2 <= rad[b] ** 2, torch.full_like(rel, con[b]), rel)
    k2 = (k0 * k0 * rel).to(torch.complex128)
    return _finish(k2, k0, (0.0, 0.0, 1.0), X, Y, Z, as_numpy)


# ---- the manufactured test problem of Sec. 5.1 (collocated grid) ---------------------------------------
def _phi(x, k0, n):
    """n-th derivative of phi(x) = exp(i k0 x) + exp(-i k0 (x - 1)) - 2 (a = 0, b = 1)."""
    v = (1j * k0) ** n * np.exp(1j * k0 * x) + (-1j * k0) ** n * np.exp(-1j * k0 * (x - 1.0))
    return v - 2.0 if n == 0 else v


def _f_deriv(X, Y, Z, k0, dx, dy, dz):
    """Derivative (dx, dy, dz) of f = lap u + k0^2 u for u = phi(x) phi(y) phi(z).  With
    phi'' = -k0^2 (phi + 2): f = -2 k0^2 [phi phi phi + phi_y phi_z + phi_x phi_z + phi_x phi_y]."""
    one = lambda a, n: np.ones_like(a, dtype=np.complex128) if n == 0 else np.zeros_like(a, dtype=np.complex128)
    px, py, pz = _phi(X, k0, dx), _phi(Y, k0, dy), _phi(Z, k0, dz)
    return -2.0 * k0 * k0 * (px * py * pz + one(X, dx) * py * pz + px * one(Y, dy) * pz + px * py * one(Z, dz))


def manufactured(n, k0, order):
    """The separable test problem of Sec. 5.1 on the collocated grid of the unit cube (nodes j h,
    h = 1/(n-1)), as inputs for helm_build_rhs_fields and helm_closure_rhs (numpy, complex128).

    Returns dict(u = exact solution on the grid, k2 = k0^2 everywhere, fields = the right-hand side fields
    of the scheme order (order 4: f on the padded grid; order 6: f, lap f, pure and mixed fourth-derivative
    sums, f_x, f_y, f_z), faces = f_n, f_nnn, lap_T f_n on the six faces in the closure's layout)."""
    h = 1.0 / (n - 1)
    node = np.arange(n) * h
    ext = np.arange(-1, n + 1) * h
    # sparse (broadcasting) meshes: the factors of the separable solution are evaluated on 1D coordinates
    # and multiplied out, which gives the same numbers as full meshes at a fraction of the cost
    Z, Y, X = np.meshgrid(node, node, node, indexing="ij", sparse=True)
    u = _phi(X, k0, 0) * _phi(Y, k0, 0) * _phi(Z, k0, 0)
    F = lambda a, b, c, P=(X, Y, Z): _f_deriv(P[0], P[1], P[2], k0, a, b, c)
    if order == 4:
        Zp, Yp, Xp = np.meshgrid(ext, ext, ext, indexing="ij", sparse=True)
        fields = _f_deriv(Xp, Yp, Zp, k0, 0, 0, 0)
    else:
        fields = np.stack([F(0, 0, 0), F(2, 0, 0) + F(0, 2, 0) + F(0, 0, 2),
                           F(4, 0, 0) + F(0, 4, 0) + F(0, 0, 4), F(2, 2, 0) + F(2, 0, 2) + F(0, 2, 2),
                           F(1, 0, 0), F(0, 1, 0), F(0, 0, 1)])
    faces = []
    for axis in range(3):
        # tangential axes in array order and their extents (ghost columns of earlier directions included)
        ta, tb = (2, 1) if axis == 0 else ((2, 0) if axis == 1 else (1, 0))
        ca = ext if ta < axis else node
        cb = ext if tb < axis else node
        A, B = np.meshgrid(ca, cb, indexing="ij")
        for side in (0, 1):
            coord = [None, None, None]
            coord[axis] = np.full_like(A, 0.0 if side == 0 else 1.0)
            coord[ta], coord[tb] = A, B
            P = tuple(coord)
            d = lambda k, t2=None: tuple((k if q == axis else (2 if q == t2 else 0)) for q in range(3))
            fn = F(*d(1), P=P)
            fnnn = F(*d(3), P=P)
            lt = F(*d(1, ta), P=P) + F(*d(1, tb), P=P)
            faces.extend([fn.ravel(), fnnn.ravel(), lt.ravel()])
    return dict(u=u, k2=np.full(u.shape, k0 * k0, dtype=np.complex128), fields=np.ascontiguousarray(fields),
                faces=np.concatenate(faces), h=h)
