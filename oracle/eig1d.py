"""The 1D absorbing-boundary matrix Lambda-bar and its eigendecomposition (Sec. 4.1).

Lambda-bar_nu (Eq. lambda_mat_definition): zero diagonal except the corners gamma_nu, ones off the
diagonal except the corner neighbours zeta_nu.  Staggered two-point ABC: gamma = (2 + i k0 h)/(2 - i k0 h),
zeta = 1 (Eq. D_bc).  Collocated three-point ABC: gamma = 2 i k0 h, zeta = 2 (the row that the ghost
U_0 = U_2 + 2 i k0 h U_1 produces).  EigT step 1 (Eq. EIG_SOLVER): Lambda-bar = V D V^{-1}, here by
LAPACK (numpy.linalg.eig) and numpy.linalg.inv.
"""
import numpy as np


def abc_params(k0, h, staggered):
    if staggered:
        return (2.0 + 1j * k0 * h) / (2.0 - 1j * k0 * h), 1.0
    return 2j * k0 * h, 2.0


def lambda_bar(N, gamma, zeta):
    assert N >= 2
    L = np.zeros((N, N), dtype=np.complex128)
    idx = np.arange(N - 1)
    L[idx, idx + 1] = 1.0
    L[idx + 1, idx] = 1.0
    L[0, 0] = gamma
    L[-1, -1] = gamma
    L[0, 1] = zeta
    L[-1, -2] = zeta
    return L


def lambda_dirichlet(N):
    """Lambda of Eq. lambda_mat_definition_new (zero corners)."""
    return lambda_bar(N, 0.0, 1.0)


def eig_decomp(N, gamma, zeta):
    """(D, V, V^{-1}) with Lambda-bar = V diag(D) V^{-1}."""
    L = lambda_bar(N, gamma, zeta)
    D, V = np.linalg.eig(L)
    return D, V, np.linalg.inv(V)


def dirichlet_closed_form(N):
    """Eigenpairs of Lambda quoted in the proof of the 1D theorem (Sec. 3.1): lambda_i = 2 cos(pi h i),
    (V_i)_l = sqrt(2h) sin(pi h i l), h = 1/(N+1)."""
    h = 1.0 / (N + 1)
    i = np.arange(1, N + 1)
    lam = 2.0 * np.cos(np.pi * h * i)
    V = np.sqrt(2.0 * h) * np.sin(np.pi * h * np.outer(i, i))   # V[l-1, i-1]
    return lam, V
