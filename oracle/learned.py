"""Oracle of the learned correction network (not in the paper; an extension of the solver): a small 3D
U-Net evaluated and differentiated by hand in float64 NumPy, for checking the GPU kernels.

Layout: activations [B][C][Z][Y][X]; 3x3x3 convolutions with zero padding and stride 1, weights
[Cout][Cin][3][3][3] plus a bias per output channel.  Architecture (width c):
    a1 = relu(conv(x,  5 -> c))          a2 = relu(conv(a1, c -> c))              (full resolution)
    p  = avgpool2(a2)
    b1 = relu(conv(p,  c -> 2c))         b2 = relu(conv(b1, 2c -> 2c))            (half resolution)
    u  = concat(upsample2(b2), a2)                                                  (3c channels)
    d1 = relu(conv(u, 3c -> c))          y  = conv(d1, c -> 2)                     (linear output)
Backward is written out layer by layer (chain rule); the test checks it against central differences.
"""
import numpy as np

LAYERS = [("c1", 5, 1), ("c2", 1, 1), ("c3", 1, 2), ("c4", 2, 2), ("c5", 3, 1), ("c6", 1, None)]


def shapes(width):
    c = width
    return {"c1": (c, 5), "c2": (c, c), "c3": (2 * c, c), "c4": (2 * c, 2 * c), "c5": (c, 3 * c), "c6": (2, c)}


def init(width, seed=0):
    rng = np.random.default_rng(seed)
    params = {}
    for name, (co, ci) in shapes(width).items():
        std = np.sqrt(2.0 / (27 * ci))
        params[name + ".w"] = rng.standard_normal((co, ci, 3, 3, 3)) * std
        params[name + ".b"] = np.zeros(co)
    return params


def conv3(x, w, b):
    """out[b,o,z,y,x] = bias[o] + sum_{i,t} w[o,i,t] x[b,i,(z,y,x)+t-1], zero padding."""
    B, C, Z, Y, X = x.shape
    xp = np.pad(x, ((0, 0), (0, 0), (1, 1), (1, 1), (1, 1)))
    out = np.zeros((B, w.shape[0], Z, Y, X))
    for dz in range(3):
        for dy in range(3):
            for dx in range(3):
                patch = xp[:, :, dz:dz + Z, dy:dy + Y, dx:dx + X]
                out += np.einsum("oi,bizyx->bozyx", w[:, :, dz, dy, dx], patch)
    return out + b[None, :, None, None, None]


def conv3_backward(x, w, g):
    """Gradients of conv3 w.r.t. x, w and b for the output gradient g."""
    B, C, Z, Y, X = x.shape
    xp = np.pad(x, ((0, 0), (0, 0), (1, 1), (1, 1), (1, 1)))
    gx = np.zeros_like(xp)
    gw = np.zeros_like(w)
    for dz in range(3):
        for dy in range(3):
            for dx in range(3):
                patch = xp[:, :, dz:dz + Z, dy:dy + Y, dx:dx + X]
                gw[:, :, dz, dy, dx] = np.einsum("bozyx,bizyx->oi", g, patch)
                gx[:, :, dz:dz + Z, dy:dy + Y, dx:dx + X] += np.einsum("oi,bozyx->bizyx", w[:, :, dz, dy, dx], g)
    gb = g.sum(axis=(0, 2, 3, 4))
    return gx[:, :, 1:-1, 1:-1, 1:-1], gw, gb


def avgpool2(x):
    B, C, Z, Y, X = x.shape
    return x.reshape(B, C, Z // 2, 2, Y // 2, 2, X // 2, 2).mean(axis=(3, 5, 7))


def upsample2(x):
    return x.repeat(2, axis=2).repeat(2, axis=3).repeat(2, axis=4)


def forward(params, x):
    """Returns the output and the saved activations."""
    P = params
    a1 = np.maximum(conv3(x, P["c1.w"], P["c1.b"]), 0)
    a2 = np.maximum(conv3(a1, P["c2.w"], P["c2.b"]), 0)
    p = avgpool2(a2)
    b1 = np.maximum(conv3(p, P["c3.w"], P["c3.b"]), 0)
    b2 = np.maximum(conv3(b1, P["c4.w"], P["c4.b"]), 0)
    u = np.concatenate([upsample2(b2), a2], axis=1)
    d1 = np.maximum(conv3(u, P["c5.w"], P["c5.b"]), 0)
    y = conv3(d1, P["c6.w"], P["c6.b"])
    return y, dict(x=x, a1=a1, a2=a2, p=p, b1=b1, b2=b2, u=u, d1=d1)


def backward(params, saved, gy):
    """Parameter gradients for the output gradient gy (and the input gradient, for completeness)."""
    P, S = params, saved
    grads = {}
    g, grads["c6.w"], grads["c6.b"] = conv3_backward(S["d1"], P["c6.w"], gy)
    g = g * (S["d1"] > 0)
    gu, grads["c5.w"], grads["c5.b"] = conv3_backward(S["u"], P["c5.w"], g)
    c2 = S["b2"].shape[1]
    gb2 = gu[:, :c2]
    ga2 = gu[:, c2:].copy()
    B, C, Z, Y, X = gb2.shape
    gb2 = gb2.reshape(B, C, Z // 2, 2, Y // 2, 2, X // 2, 2).sum(axis=(3, 5, 7))   # adjoint of upsample2
    gb2 = gb2 * (S["b2"] > 0)
    g, grads["c4.w"], grads["c4.b"] = conv3_backward(S["b1"], P["c4.w"], gb2)
    g = g * (S["b1"] > 0)
    gp, grads["c3.w"], grads["c3.b"] = conv3_backward(S["p"], P["c3.w"], g)
    ga2 = ga2 + upsample2(gp) / 8.0                                                # adjoint of avgpool2
    ga2 = ga2 * (S["a2"] > 0)
    g, grads["c2.w"], grads["c2.b"] = conv3_backward(S["a1"], P["c2.w"], ga2)
    g = g * (S["a1"] > 0)
    gx, grads["c1.w"], grads["c1.b"] = conv3_backward(S["x"], P["c1.w"], g)
    return grads, gx


def mse(y, t):
    """0.5 * mean((y - t)^2) and its gradient."""
    d = y - t
    return 0.5 * np.mean(d * d), d / d.size
