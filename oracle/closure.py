"""High-order closure of the Sommerfeld condition on collocated grids (Sec. 2.1, the test-problem passage
after Eq. scheme6; test infrastructure like the rest of oracle/).

The paper states only that its constant-k tests close the fourth- and sixth-order schemes with high-order
approximations of the ABC built on a three-point stencil.  Our reading, written out here:

On a face with outward normal n (coordinate s along n, s = +1 on the far face, -1 on the near one) the
ghost one step outside the boundary node B and the first interior node I lie symmetrically about B, so

    U_ghost = U_I + s * sum_m c_m d_n^(2m+1) u(B),       c_m = 2 h_n^(2m+1) / (2m+1)!.

With the ABC d_n u = s i k0 u along the whole face and the equation d_n^2 u = f - L u, L = k0^2 + lap_T
(lap_T: the two tangential second derivatives; k = k0 on the face), every odd normal derivative reduces to
the face values of u and of f:

    d_n^(2m+1) u = sum_{j<m} (-L)^j d_n^(2(m-j)-1) f + (-1)^m s i k0 L^m u.

The u part of the ghost is therefore U_I + sum_m c_m (-1)^m i k0 L^m U_B (independent of s) and the f part
is s sum_m c_m sum_{j<m} (-L)^j d_n^(2(m-j)-1) f.  We keep m <= 2 (ghost exact to O(h^7)); L acts on U_B
through sixth-order difference matrices along the face (centred seven points where they fit, eight
one-sided points near the face's edges).  m = 0 alone is the second-order three-point rule of the
preconditioner (Lambda-bar with zeta = 2, Sec. 4.1).  The faces are filled x, then y, then z; a later
direction's face covers the ghost columns of the earlier ones, so edge and corner ghosts come from the
closure applied along an already-filled ghost line.

The u part is linear in U (it defines the operator); the f part does not involve U and moves to the
right-hand side: F - A(ghosts of the f part alone).
"""
import math

import numpy as np

TERMS = 2         # highest m kept in the Taylor sum
ACCURACY = 6      # order of the tangential second-derivative matrices


def derivative_matrix(n, h, deriv, acc):
    """n x n matrix of the deriv-th derivative on n equispaced nodes, error O(h^acc).

    Rows use the centred stencil of deriv + acc - 1 nodes where it fits and the deriv + acc nodes nearest
    to the row's node otherwise; weights from the Taylor (Vandermonde) conditions."""
    if n < deriv + acc:
        raise ValueError(f"{n} nodes are too few for a derivative {deriv} of order {acc}")
    r = (deriv + acc - 1) // 2
    D = np.zeros((n, n))
    for i in range(n):
        if i - r >= 0 and i + r <= n - 1:
            idx = np.arange(i - r, i + r + 1)
        else:
            s = deriv + acc
            lo = 0 if i - r < 0 else n - s
            idx = np.arange(lo, lo + s)
        o = (idx - i).astype(np.float64)
        V = np.array([o ** q / math.factorial(q) for q in range(len(o))])
        e = np.zeros(len(o))
        e[deriv] = 1.0
        D[i, idx] = np.linalg.solve(V, e) / h ** deriv
    return D


def _face_coords(axis, value, ca, cb):
    """(X, Y, Z) on the face normal to `axis` at coordinate `value`; (ca, cb) are the coordinates of the
    two tangential axes in the order of the face array (z before y before x)."""
    A, B = np.meshgrid(ca, cb, indexing="ij")
    C = np.full_like(A, value)
    if axis == 0:
        return C, B, A          # face array (z, y)
    if axis == 1:
        return B, C, A          # face array (z, x)
    return B, A, C              # face array (y, x)


def _f_part(fdiff, axis, X, Y, Z, k0, m):
    """sum_{j<m} (-L)^j d_n^(2(m-j)-1) f on a face, L^j expanded by the multinomial theorem over
    (k0^2, d_t1^2, d_t2^2); fdiff(X, Y, Z, (dx, dy, dz)) returns a derivative of f."""
    t1, t2 = [a for a in range(3) if a != axis]
    tot = 0.0
    for j in range(m):
        nd = 2 * (m - j) - 1
        Lj = 0.0
        for a in range(j + 1):
            for b in range(j + 1 - a):
                c = j - a - b
                coef = math.factorial(j) // (math.factorial(a) * math.factorial(b) * math.factorial(c))
                d = [0, 0, 0]
                d[axis], d[t1], d[t2] = nd, 2 * b, 2 * c
                Lj = Lj + coef * k0 ** (2 * a) * fdiff(X, Y, Z, tuple(d))
        tot = tot + (-1) ** j * Lj
    return tot


def pad_ghost_ho(U, k0, h, fdiff=None, origin=(0.0, 0.0, 0.0), terms=TERMS, acc=ACCURACY):
    """U with one ghost layer from the high-order closure.  fdiff None: the u part only (the operator);
    otherwise the f part is added, with f's derivatives from fdiff at the face coordinates
    (collocated nodes origin + j h)."""
    nz, ny, nx = U.shape
    P = np.zeros((nz + 2, ny + 2, nx + 2), dtype=np.complex128)
    P[1:-1, 1:-1, 1:-1] = U
    n = (nx, ny, nz)
    coords = [origin[a] + np.arange(-1, n[a] + 1) * h[a] for a in range(3)]
    for axis in range(3):
        hn = h[axis]
        c = [2.0 * hn ** (2 * m + 1) / math.factorial(2 * m + 1) for m in range(terms + 1)]
        Q = np.moveaxis(P, 2 - axis, 0)            # Q[normal, t_a, t_b], a view of P
        t_a, t_b = [a for a in (2, 1, 0) if a != axis]   # tangential axes in face-array order
        # ghost columns of the directions already filled are part of this face; unfilled ones are not
        ext = [slice(None) if t < axis else slice(1, -1) for t in (t_a, t_b)]
        face = Q[:, ext[0], ext[1]]
        if terms > 0:
            Da = derivative_matrix(face.shape[1], h[t_a], 2, acc)
            Db = derivative_matrix(face.shape[2], h[t_b], 2, acc)
        L = lambda V: k0 * k0 * V + Da @ V + V @ Db.T
        nn = face.shape[0]
        for s, ib, ii, ig in ((-1, 1, 2, 0), (1, nn - 2, nn - 3, nn - 1)):
            V = face[ib].copy()
            g = face[ii].copy()
            for m in range(terms + 1):
                g = g + c[m] * (-1) ** m * 1j * k0 * V
                if m < terms:
                    V = L(V)
            if fdiff is not None:
                X, Y, Z = _face_coords(axis, coords[axis][ib], coords[t_a][ext[0]], coords[t_b][ext[1]])
                for m in range(1, terms + 1):
                    g = g + s * c[m] * _f_part(fdiff, axis, X, Y, Z, k0, m)
            face[ig] = g
    return P
