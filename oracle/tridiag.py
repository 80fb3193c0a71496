"""Thomas algorithm for the independent z-systems of Eq. Indep_precond_system.

Row l:  a[l] x[l-1] + b[l] x[l] + c[l] x[l+1] = d[l]  (a[0], c[-1] unused).  Axis 0 is the system
index l; all trailing axes are independent systems solved together.  No pivoting (Golub & Van Loan
Alg. 4.3.6, the textbook tridiagonal LU).
"""
import numpy as np


def thomas(a, b, c, d):
    n = d.shape[0]
    b = np.broadcast_to(b, d.shape).astype(np.complex128)
    a = np.broadcast_to(a, d.shape).astype(np.complex128)
    c = np.broadcast_to(c, d.shape).astype(np.complex128)
    cp = np.empty(d.shape, dtype=np.complex128)
    dp = np.empty(d.shape, dtype=np.complex128)
    cp[0] = c[0] / b[0]
    dp[0] = d[0] / b[0]
    for l in range(1, n):
        den = b[l] - a[l] * cp[l - 1]
        cp[l] = c[l] / den if l < n - 1 else 0.0
        dp[l] = (d[l] - a[l] * dp[l - 1]) / den
    x = np.empty(d.shape, dtype=np.complex128)
    x[-1] = dp[-1]
    for l in range(n - 2, -1, -1):
        x[l] = dp[l] - cp[l] * x[l + 1]
    return x
