"""PFFT: the three-step solver of A_p U = Y built on a sine-transform solver (Sec. 4.2).

A_p^F (Eq. TFprec) replaces Lbar_x, Lbar_y by Dirichlet matrices whose eigenvectors are sines; z keeps
Lbar_z and K_z.  Eq. PFFT_SOLVER:
  1. A_p^F Theta = Y                       (2D sine transform per slice + z-tridiagonal solves)
  2. A_p W = (A_p^F - A_p) Theta           (EigT; the right side lives on the boundary rows only)
  3. A_p^F U = Y + (A_p^F - A_p)(Theta + W)
The paper's sparse forward/inverse transforms and the reuse of the transformed Y are savings that do
not change the result; this oracle forms every vector in full.

Dirichlet variants (our reading for the grid sizes used here):
  'node'  Lambda of Eq. lambda_mat_definition_new (zero corners): eigenvectors sin(pi i l/(N+1)),
          eigenvalues 2 cos(pi i/(N+1)) (Sec. 3.1), i.e. the DST-I (the paper's FFT grids 2^k - 1).
  'face'  Dirichlet at the staggered face, ghost U_0 = -U_1 (corner -1): eigenvectors
          sin(pi j (l - 1/2)/N), eigenvalues 2 cos(pi j/N), i.e. the DST-II (FFT-friendly for N = 2^k).
(A_p^F - A_p) in x is diag-corner (c - gamma_x) and corner-neighbour (1 - zeta_x) with c = 0 ('node')
or -1 ('face'), times a_x (reading: the matrix difference; the paper's listing of Theta^x shifts the
zeta term one row and drops a_x, which coincide with this for zeta = 1, a_x = 1).
"""
import numpy as np
import scipy.fft as sfft

from .eigt import EigT
from .tridiag import thomas


class PFFT:
    def __init__(self, grid, k0, k0z2=None, variant="face"):
        self.grid = grid
        self.variant = variant
        self.eigt = EigT(grid, k0, k0z2)
        nx, ny, nz = grid.n
        e = self.eigt
        if variant == "node":
            self.dx = 2.0 * np.cos(np.pi * np.arange(1, nx + 1) / (nx + 1))
            self.dy = 2.0 * np.cos(np.pi * np.arange(1, ny + 1) / (ny + 1))
            self.corner = 0.0
        elif variant == "face":
            self.dx = 2.0 * np.cos(np.pi * np.arange(1, nx + 1) / nx)
            self.dy = 2.0 * np.cos(np.pi * np.arange(1, ny + 1) / ny)
            self.corner = -1.0
        else:
            raise ValueError(variant)
        diag = (e.ax * self.dx[None, None, :] + e.ay * self.dy[None, :, None]
                + e.cz[:, None, None]).astype(np.complex128)
        diag[0] += e.gz
        diag[-1] += e.gz
        self.diagF = diag

    def _dst(self, Y, inverse=False):
        t = 1 if self.variant == "node" else 2
        f = sfft.idst if inverse else sfft.dst
        return f(f(Y, type=t, axis=2, norm="ortho"), type=t, axis=1, norm="ortho")

    def solve_F(self, Y):
        """A_p^F Theta = Y."""
        sub, _, sup = self.eigt.z_coefficients()
        That = thomas(sub, self.diagF, sup, self._dst(Y))
        return self._dst(That, inverse=True)

    def diff_apply(self, T):
        """(A_p^F - A_p) T: nonzero on the rows i in {1, N_x} and j in {1, N_y} only (Sec. 4.2)."""
        e = self.eigt
        R = np.zeros_like(T)
        c = self.corner
        R[:, :, 0] += e.ax * ((c - e.gx) * T[:, :, 0] + (1.0 - e.zx) * T[:, :, 1])
        R[:, :, -1] += e.ax * ((c - e.gx) * T[:, :, -1] + (1.0 - e.zx) * T[:, :, -2])
        R[:, 0, :] += e.ay * ((c - e.gy) * T[:, 0, :] + (1.0 - e.zy) * T[:, 1, :])
        R[:, -1, :] += e.ay * ((c - e.gy) * T[:, -1, :] + (1.0 - e.zy) * T[:, -2, :])
        return R

    def solve_Ap(self, Y):
        Y = np.asarray(Y, dtype=np.complex128).reshape(self.grid.shape)
        Theta = self.solve_F(Y)                                   # step 1
        W = self.eigt.solve_Ap(self.diff_apply(Theta))            # step 2
        return self.solve_F(Y + self.diff_apply(Theta + W))       # step 3

    def apply_Minv(self, r):
        hz = self.grid.h[2]
        return hz * hz * self.solve_Ap(r)
