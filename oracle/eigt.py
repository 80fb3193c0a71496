"""EigT: direct solution of the second-order preconditioning system A_p U = Y (Sec. 4.1).

A_p = I_z (x) (a_y Lbar_y (x) I_x + a_x I_y (x) Lbar_x) + (Lbar_z + K_z - 2(a_x + a_y + 1) I_z) (x) I_xy,
a_d = h_z^2/h_d^2, K_z = h_z^2 diag(k0^2(z_l))  (the Kronecker form after Eq. lambda_mat_definition).
A_p is h_z^2 times the second-order operator (delta^2 sum + k0^2) with the ABC ghosts eliminated, so
the preconditioner action is M^{-1} r = h_z^2 A_p^{-1} r.

EigT (Eq. EIG_SOLVER): (1) eigendecompose Lbar_x, Lbar_y; (2) Ybar_l = (V_y^{-1} (x) V_x^{-1}) Y_l,
which for the slice stored as an (N_y, N_x) array is V_y^{-1} Y_l V_x^{-T}; (3) solve the N_x N_y
tridiagonal systems of Eq. Indep_precond_system with diagonal a_x d_{x,i} + a_y d_{y,j} + h_z^2 k0^2(z_l)
- 2(a_x + a_y + 1) (+gamma_z in the end rows; the a's are kept, reading of the diagonal formula),
off-diagonals 1 (zeta_z next to the end rows); (4) U_l = V_y Ubar_l V_x^T.
"""
import numpy as np

from .eig1d import abc_params, eig_decomp, lambda_bar
from .tridiag import thomas


class EigT:
    def __init__(self, grid, k0, k0z2=None):
        self.grid = grid
        nx, ny, nz = grid.n
        hx, hy, hz = grid.h
        self.ax = hz * hz / (hx * hx)
        self.ay = hz * hz / (hy * hy)
        self.k0 = k0
        self.k0z2 = np.full(nz, k0 * k0, dtype=np.complex128) if k0z2 is None else np.asarray(k0z2, np.complex128)
        self.gx, self.zx = abc_params(k0, hx, grid.staggered)
        self.gy, self.zy = abc_params(k0, hy, grid.staggered)
        self.gz, self.zz = abc_params(k0, hz, grid.staggered)
        self.Dx, self.Vx, self.Vxi = eig_decomp(nx, self.gx, self.zx)
        self.Dy, self.Vy, self.Vyi = eig_decomp(ny, self.gy, self.zy)
        self.cz = hz * hz * self.k0z2 - 2.0 * (self.ax + self.ay + 1.0)

    def z_coefficients(self):
        """(sub, diag, super) of the z-systems; diag has shape (nz, ny, nx)."""
        nx, ny, nz = self.grid.n
        diag = (self.ax * self.Dx[None, None, :] + self.ay * self.Dy[None, :, None]
                + self.cz[:, None, None]).astype(np.complex128)
        diag[0] += self.gz
        diag[-1] += self.gz
        sub = np.ones(nz, dtype=np.complex128)
        sup = np.ones(nz, dtype=np.complex128)
        sup[0] = self.zz
        sub[-1] = self.zz
        return sub[:, None, None], diag, sup[:, None, None]

    def forward(self, Y):
        return np.einsum("ab,lbc,dc->lad", self.Vyi, Y, self.Vxi, optimize=True)

    def inverse(self, Ub):
        return np.einsum("ab,lbc,dc->lad", self.Vy, Ub, self.Vx, optimize=True)

    def solve_Ap(self, Y):
        Y = np.asarray(Y, dtype=np.complex128).reshape(self.grid.shape)
        Yb = self.forward(Y)
        sub, diag, sup = self.z_coefficients()
        Ub = thomas(sub, diag, sup, Yb)
        return self.inverse(Ub)

    def apply_Minv(self, r):
        hz = self.grid.h[2]
        return hz * hz * self.solve_Ap(r)

    def dense_Ap(self):
        """The Kronecker form, assembled (small grids only)."""
        nx, ny, nz = self.grid.n
        Lx = lambda_bar(nx, self.gx, self.zx)
        Ly = lambda_bar(ny, self.gy, self.zy)
        Lz = lambda_bar(nz, self.gz, self.zz)
        Ix, Iy, Iz = np.eye(nx), np.eye(ny), np.eye(nz)
        hz = self.grid.h[2]
        Kz = hz * hz * np.diag(self.k0z2)
        horiz = self.ay * np.kron(Ly, Ix) + self.ax * np.kron(Iy, Lx)
        vert = Lz + Kz - 2.0 * (self.ax + self.ay + 1.0) * Iz
        return np.kron(Iz, horiz) + np.kron(vert, np.kron(Iy, Ix))
