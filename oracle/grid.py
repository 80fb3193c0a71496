"""Grid geometry and the two-point Sommerfeld ghost coefficient.

Sec. 2.1 (grid Omega_h, steps h_alpha = L_alpha/(N_alpha - 1)) for collocated grids; Sec. 5.2 (nodes
h/2 + j h, h = L/N) for staggered grids; Eq. D_bc for gamma = (2 + i k0 h)/(2 - i k0 h).
Arrays are indexed [l, j, i] = (z, y, x) with x fastest (the slice ordering U_l of Sec. 4.1).
"""
import numpy as np


class Grid:
    """N_x x N_y x N_z unknowns on [0,Lx]x[0,Ly]x[0,Lz]; boundary nodes are unknowns, ghosts are not."""

    def __init__(self, nx, ny, nz, lx=1.0, ly=1.0, lz=1.0, staggered=True):
        self.n = (int(nx), int(ny), int(nz))
        self.L = (float(lx), float(ly), float(lz))
        self.staggered = bool(staggered)
        if staggered:   # Sec. 5.2: x_j = h/2 + j h, h = L/N
            self.h = tuple(L / n for L, n in zip(self.L, self.n))
        else:           # Sec. 2.1: x_i = (i-1) h, h = L/(N-1)
            self.h = tuple(L / (n - 1) for L, n in zip(self.L, self.n))

    @property
    def shape(self):
        nx, ny, nz = self.n
        return (nz, ny, nx)

    @property
    def unknowns(self):
        nx, ny, nz = self.n
        return nx * ny * nz

    def coords(self, axis):
        n, h = self.n[axis], self.h[axis]
        j = np.arange(n, dtype=np.float64)
        return (0.5 * h + j * h) if self.staggered else j * h

    def mesh(self):
        """Coordinate arrays X, Y, Z of shape (nz, ny, nx)."""
        x, y, z = self.coords(0), self.coords(1), self.coords(2)
        Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
        return X, Y, Z


def gamma_two_point(k0, h):
    """Ghost coefficient of Eq. D_bc: U_0 = gamma U_1 with gamma = (2 + i k0 h)/(2 - i k0 h)."""
    return (2.0 + 1j * k0 * h) / (2.0 - 1j * k0 * h)
