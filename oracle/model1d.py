"""The 1D model problem of Sec. 3.1: Dirichlet u'' + k^2 u = f on [0,1], h = 1/(N+1).

Eq. vect_eq: U_{i-1} - 2 d U_i + U_{i+1} = F_i, so A = Lambda - 2 d_r I (Eq. A_matrix) with
d_r = sum_{j=0}^r (-1)^j tau^{2j}/(2j)! (Eq. coef_gen), tau = k h; the second-order preconditioner
A_p = Lambda - 2(1 - tau^2/2) I (Eq. precond).
"""
import math

import numpy as np

from .eig1d import lambda_dirichlet


def d_r(tau, r):
    return sum((-1) ** j * tau ** (2 * j) / math.factorial(2 * j) for j in range(r + 1))


def matrices(N, k, r):
    h = 1.0 / (N + 1)
    tau = k * h
    Lam = lambda_dirichlet(N)
    A = Lam - 2.0 * d_r(tau, r) * np.eye(N)
    Ap = Lam - 2.0 * (1.0 - tau * tau / 2.0) * np.eye(N)
    return A, Ap
