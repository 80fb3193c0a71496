"""Restarted GMRES(m), right-preconditioned, and flexible GMRES (Sec. 5; the paper cites Saad [s]).

Right preconditioning (Eq. Preconditioned_System): A M^{-1} y = F, U = M^{-1} y; Arnoldi by modified
Gram-Schmidt, the least-squares problem by complex Givens rotations (Saad, Alg. 6.9 and 9.5).
Flexible variant (Saad, Alg. 9.6) stores z_j = M_j^{-1} v_j and updates x with Z y.
Convergence: rel-res = ||F - A U||_2 / ||F - A U^0||_2 (Sec. 5.1) <= rtol, watched on the Givens
estimate and confirmed by the true residual at the end of each cycle.  N0 counts inner steps.
x0 = 0 unless given (reading).
"""
import numpy as np


def _givens(a, b):
    """c (real), s (complex) with [c, s; -conj(s), c] [a; b] = [r; 0]."""
    if b == 0:
        return 1.0, 0.0 + 0j
    if a == 0:
        return 0.0, np.conj(b) / abs(b)
    t = np.hypot(abs(a), abs(b))
    c = abs(a) / t
    s = (a / abs(a)) * np.conj(b) / t
    return c, s


def gmres(apply_A, apply_M, b, x0=None, m=20, rtol=1e-10, max_it=1000, flexible=False, history=None):
    b = np.asarray(b, dtype=np.complex128).ravel()
    x = np.zeros_like(b) if x0 is None else np.asarray(x0, dtype=np.complex128).ravel().copy()
    Av = lambda v: np.asarray(apply_A(v), dtype=np.complex128).ravel()
    Mv = lambda v: np.asarray(apply_M(v), dtype=np.complex128).ravel()
    r = b - Av(x)
    beta0 = np.linalg.norm(r)
    its = 0
    info = {"iterations": 0, "restarts": 0, "converged": False, "beta0": beta0}
    if beta0 == 0:
        info.update(converged=True, relres=0.0)
        return x, info
    while True:
        beta = np.linalg.norm(r)
        if beta / beta0 <= rtol:
            info["converged"] = True
            break
        if its >= max_it:
            break
        V = [r / beta]
        Z = []
        H = np.zeros((m + 1, m), dtype=np.complex128)
        cs = np.zeros(m)
        sn = np.zeros(m, dtype=np.complex128)
        g = np.zeros(m + 1, dtype=np.complex128)
        g[0] = beta
        k = 0
        for j in range(m):
            z = Mv(V[j])
            if flexible:
                Z.append(z)
            w = Av(z)
            for i in range(j + 1):
                H[i, j] = np.vdot(V[i], w)
                w = w - H[i, j] * V[i]
            hnext = np.linalg.norm(w)
            H[j + 1, j] = hnext
            for i in range(j):
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -np.conj(sn[i]) * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            cs[j], sn[j] = _givens(H[j, j], H[j + 1, j])
            H[j, j] = cs[j] * H[j, j] + sn[j] * H[j + 1, j]
            H[j + 1, j] = 0.0
            g[j + 1] = -np.conj(sn[j]) * g[j]
            g[j] = cs[j] * g[j]
            its += 1
            k = j + 1
            if history is not None:
                history.append(abs(g[j + 1]) / beta0)
            if abs(g[j + 1]) / beta0 <= rtol or its >= max_it:
                break
            V.append(w / hnext)
        y = np.linalg.solve(np.triu(H[:k, :k]), g[:k])
        if flexible:
            x = x + sum(y[i] * Z[i] for i in range(k))
        else:
            x = x + Mv(sum(y[i] * V[i] for i in range(k)))
        info["restarts"] += 1
        r = b - Av(x)
    info["iterations"] = its
    info["relres"] = np.linalg.norm(r) / beta0
    return x, info
