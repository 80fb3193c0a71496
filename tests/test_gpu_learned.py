"""The learned correction's kernels against the CPU oracle (oracle/learned.py), through the C-ABI.

Precision: weights and inputs are given as bfloat16-representable values, so the kernels and the oracle
start from identical numbers; the kernels then store every activation in bfloat16 (unit roundoff 2^-9)
and accumulate in float32.  Seven stored tensors lie between input and output, so the output carries a
relative error of a few times 2^-9 in the 2-norm: the bound used is 2e-2 (4e-2 for gradients, which pass
through the stored activations twice).  A wrong index, tap flip or mask gives errors of order 1.
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import learned as OL
from oracle.eigt import EigT
from oracle.grid import Grid
from paper_2602_07711_gb300 import HELM_PREC_TF32, Net, Solver, helm, learned


def bf16_round(a):
    """Round to the nearest bfloat16 (ties to even), returned as float64."""
    u = np.ascontiguousarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def _rel(a, b):
    return np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel())


def _setup(width, shape, B, seed):
    rng = np.random.default_rng(seed)
    net = Net(width, seed=seed)
    P = OL.init(width, seed=seed)
    for k in P:
        if k.endswith(".b"):
            P[k] = 0.1 * rng.standard_normal(P[k].shape)
        P[k] = bf16_round(P[k])
    net.set_params(net.flatten(P))
    x = bf16_round(rng.standard_normal((B, 5) + shape))
    xd = torch.from_numpy(x.astype(np.float32)).cuda().to(torch.bfloat16)
    return net, P, x, xd


# the convolutions run on the tensor cores (conv_tc.cu): widths that are not multiples of 16 (padded chunks),
# grids narrower and wider than one 128-point row tile (x = 130, 136: a ragged second tile), batches, and the
# width of the ~200K-parameter network (32; its 96-channel data gradient takes two output slices)
@pytest.mark.parametrize("width,shape,B", [(4, (6, 10, 12), 2), (8, (8, 18, 10), 1), (3, (4, 4, 34), 1),
                                           (32, (4, 6, 130), 1), (24, (6, 4, 20), 2)])
def test_forward_matches_oracle(width, shape, B):
    net, P, x, xd = _setup(width, shape, B, 11)
    y = net.forward(xd).cpu().numpy().astype(np.float64)
    yo, _ = OL.forward(P, x)
    assert _rel(y, yo) < 2e-2, _rel(y, yo)


@pytest.mark.parametrize("width,shape,B", [(4, (6, 10, 12), 2), (6, (8, 8, 20), 1), (32, (4, 4, 136), 1)])
def test_backward_matches_oracle(width, shape, B):
    net, P, x, xd = _setup(width, shape, B, 12)
    rng = np.random.default_rng(3)
    t = rng.standard_normal((B, 2) + shape)
    td = torch.from_numpy(t.astype(np.float32)).cuda()
    net.zero_grad()
    y = net.forward(xd)
    gy = torch.empty_like(y)
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    helm.helm_net_mse(y, td, gy, loss)
    net.backward(gy)
    g = net.unflatten(net.get_grads())
    yo, saved = OL.forward(P, x)
    lo, gyo = OL.mse(yo, t)
    assert abs(loss.item() - lo) < 2e-2 * lo
    go, _ = OL.backward(P, saved, gyo)
    for k in go:
        e = _rel(g[k].astype(np.float64), go[k])
        assert e < 4e-2, (k, e)


def test_gradient_accumulates_and_zeroes():
    net, P, x, xd = _setup(4, (4, 6, 8), 1, 13)
    t = torch.randn((1, 2, 4, 6, 8), device="cuda", generator=torch.Generator("cuda").manual_seed(0))
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    net.zero_grad()
    for _ in range(2):
        y = net.forward(xd)
        gy = torch.empty_like(y)
        helm.helm_net_mse(y, t, gy, loss)
        net.backward(gy)
    g2 = net.get_grads()
    net.zero_grad()
    y = net.forward(xd)
    helm.helm_net_mse(y, t, gy, loss)
    net.backward(gy)
    g1 = net.get_grads()
    assert np.allclose(g2, 2 * g1, rtol=1e-4, atol=1e-7 * np.abs(g1).max())


def test_adam_step_matches_formula():
    net, P, x, xd = _setup(4, (4, 6, 8), 1, 14)
    t = torch.zeros((1, 2, 4, 6, 8), device="cuda")
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    w0 = net.get_params().astype(np.float64)
    m = np.zeros_like(w0)
    v = np.zeros_like(w0)
    for step in (1, 2):
        net.zero_grad()
        y = net.forward(xd)
        gy = torch.empty_like(y)
        helm.helm_net_mse(y, t, gy, loss)
        net.backward(gy)
        g = net.get_grads().astype(np.float64)
        net.adam(lr=1e-2, beta1=0.9, beta2=0.999, eps=1e-8)
        m = 0.9 * m + 0.1 * g
        v = 0.999 * v + 0.001 * g * g
        w0 = w0 - 1e-2 * (m / (1 - 0.9 ** step)) / (np.sqrt(v / (1 - 0.999 ** step)) + 1e-8)
        w = net.get_params().astype(np.float64)
        assert np.abs(w - w0).max() < 1e-5 * max(1.0, np.abs(w0).max()), step
        w0 = w


def _problem(n, seed=0):
    k2, f, k0 = learned.high_contrast(n, seed)
    return k2, f, k0


def test_features_and_target_follow_their_definitions():
    n = 16
    k2, f, k0 = _problem(n)
    S = Solver((n, n, n), k2, k0, order=6, precision=HELM_PREC_TF32, flexible=True)
    net = Net(2)
    rng = np.random.default_rng(5)
    v = rng.standard_normal((n, n, n)) + 1j * rng.standard_normal((n, n, n))
    vd = torch.from_numpy(v).cuda().to(torch.complex64)
    mv = S.apply_precond(vd)
    X = S.features(net, vd, mv).float().cpu().numpy().astype(np.float64)
    vv = vd.cpu().numpy().astype(np.complex128)
    mm = mv.cpu().numpy().astype(np.complex128)
    rv = np.sqrt(np.mean(np.abs(vv) ** 2))
    rm = np.sqrt(np.mean(np.abs(mm) ** 2))
    k2h = k2.cpu().numpy()
    ref = np.stack([vv.real / rv, vv.imag / rv, mm.real / rm, mm.imag / rm, k2h.real / k0 ** 2 - 1])
    assert np.abs(X - ref).max() <= 2 ** -8 * np.abs(ref).max()
    xs = torch.from_numpy(rng.standard_normal((n, n, n)) + 1j * rng.standard_normal((n, n, n))).cuda()
    xk = torch.from_numpy(rng.standard_normal((n, n, n)) + 1j * rng.standard_normal((n, n, n))).cuda()
    T = S.target(net, xs, xk, mv).cpu().numpy().astype(np.float64)
    d = (xs.cpu().numpy() - xk.cpu().numpy() - mm) / rm
    assert _rel(T, np.stack([d.real, d.imag])) < 1e-6


def test_attached_net_takes_the_minimal_residual_step_after_eigt():
    n = 16
    k2, f, k0 = _problem(n)
    S = Solver((n, n, n), k2, k0, order=6, precision=HELM_PREC_TF32, flexible=True)
    net = Net(4, seed=3)
    rng = np.random.default_rng(6)
    vd = torch.from_numpy(rng.standard_normal((n, n, n)) + 1j * rng.standard_normal((n, n, n))).cuda().to(torch.complex64)
    z0 = S.apply_precond(vd)
    X = S.features(net, vd, z0)
    y = net.forward(X[None].contiguous())[0]
    zz = z0.cpu().numpy().astype(np.complex128)
    s = np.sqrt(np.mean(np.abs(zz) ** 2))
    c = s * (y[0].cpu().numpy().astype(np.float64) + 1j * y[1].cpu().numpy().astype(np.float64))
    cd = torch.from_numpy(c).cuda().to(torch.complex64)
    Az0 = S.apply_A(z0).cpu().numpy().astype(np.complex128)
    Ac = S.apply_A(cd).cpu().numpy().astype(np.complex128)
    v = vd.cpu().numpy().astype(np.complex128)
    rho = v - Az0
    alpha = np.vdot(Ac, rho) / np.vdot(Ac, Ac).real
    S.attach(net)
    z1 = S.apply_precond(vd).cpu().numpy().astype(np.complex128)
    assert _rel(z1, zz + alpha * c) < 1e-5
    st = net.stats()
    assert st[3] == 0 and st[4] == 1 and abs(st[2] - abs(alpha)) < 1e-4 * abs(alpha)
    r1 = np.linalg.norm(v - S.apply_A(torch.from_numpy(z1).cuda().to(torch.complex64)).cpu().numpy())
    assert r1 <= np.linalg.norm(rho) * (1 + 1e-5)
    assert abs(st[5] - (r1 / np.linalg.norm(rho)) ** 2) < 1e-3
    # EigT part against the oracle: M^-1 v of the constant-k0 second-order operator
    e = EigT(Grid(n, n, n, staggered=True), k0)
    assert _rel(zz, e.apply_Minv(v)) < 1e-2
    # a network whose output is not finite is dropped: z = M^-1 v exactly
    P = net.unflatten(net.get_params())
    P["c6.b"][:] = np.nan
    net.set_params(net.flatten(P))
    z2 = S.apply_precond(vd).cpu().numpy().astype(np.complex128)
    assert np.array_equal(z2, zz)
    assert net.stats()[3] == 1
    S.attach(None)
    with pytest.raises(helm.HelmError):
        Solver((n, n, n), k2, k0, order=6, precision=HELM_PREC_TF32, flexible=False).attach(net)


def test_training_lowers_the_loss_and_learned_fgmres_converges():
    n = 32
    X, T = learned.generate_pairs(n=n, seeds=range(2), iters=(0, 3, 8), arnoldi=2, order=6)
    assert X.shape == (10, 5, n, n, n) and T.shape == (10, 2, n, n, n)
    assert torch.isfinite(T).all()
    net = Net(6, seed=1)
    l0, base = learned.evaluate(net, X, T)
    log = learned.train(net, X, T, steps=80, batch=2, lr=3e-3, lr_final=1e-3)
    l1, _ = learned.evaluate(net, X, T)
    assert l1 < 0.9 * l0, (l0, l1, base, log)
    r = learned.compare(net, n, seed=7, rtol=1e-6, repeats=1)
    assert r["learned"]["status"] == 0 and r["learned"]["relres_true"] <= 1e-6, r
    assert r["plain"]["status"] == 0
    assert r["solution_rel_diff"] < 1e-5, r
    print("learned vs plain at %d^3:" % n, r)
