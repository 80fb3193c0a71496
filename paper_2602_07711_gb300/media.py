"""Seeded synthetic workloads (inputs only: none of the solver's arithmetic lives here).

Every workload is a scattering problem on the unit cube with a staggered grid (nodes h/2 + j h,
h = 1/n, Sec. 5.2): a medium k^2(x), a background wavenumber k0, an incident plane wave
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
