"""Pins of the learned-correction oracle (no GPU): the hand-written backward agrees with central finite
differences of the loss in float64, and the convolution agrees with a direct sum."""
import numpy as np

from oracle import learned as L


def test_conv3_matches_direct_sum():
    rng = np.random.default_rng(0)
    x = rng.standard_normal((1, 2, 4, 3, 5))
    w = rng.standard_normal((3, 2, 3, 3, 3))
    b = rng.standard_normal(3)
    y = L.conv3(x, w, b)
    # direct evaluation at a few points, zero outside
    for (o, z, yy, xx) in [(0, 0, 0, 0), (2, 3, 2, 4), (1, 1, 1, 2)]:
        s = b[o]
        for i in range(2):
            for dz in range(3):
                for dy in range(3):
                    for dx in range(3):
                        zz, y2, x2 = z + dz - 1, yy + dy - 1, xx + dx - 1
                        if 0 <= zz < 4 and 0 <= y2 < 3 and 0 <= x2 < 5:
                            s += w[o, i, dz, dy, dx] * x[0, i, zz, y2, x2]
        assert abs(y[0, o, z, yy, xx] - s) < 1e-12


def test_backward_matches_finite_differences():
    rng = np.random.default_rng(1)
    P = L.init(3, seed=2)
    for k in P:
        if k.endswith(".b"):
            P[k] = rng.standard_normal(P[k].shape) * 0.1
    x = rng.standard_normal((2, 5, 4, 4, 6))
    t = rng.standard_normal((2, 2, 4, 4, 6))

    def loss(params):
        y, _ = L.forward(params, x)
        return L.mse(y, t)[0]

    y, S = L.forward(P, x)
    _, gy = L.mse(y, t)
    G, _ = L.backward(P, S, gy)
    eps = 1e-6
    for name in ["c1.w", "c3.w", "c5.w", "c6.w", "c2.b", "c4.b"]:
        flat = P[name].reshape(-1)
        for idx in rng.choice(flat.size, size=min(6, flat.size), replace=False):
            old = flat[idx]
            flat[idx] = old + eps
            lp = loss(P)
            flat[idx] = old - eps
            lm = loss(P)
            flat[idx] = old
            fd = (lp - lm) / (2 * eps)
            an = G[name].reshape(-1)[idx]
            assert abs(fd - an) <= 1e-6 * max(1.0, abs(fd)) + 1e-9, (name, idx, fd, an)
