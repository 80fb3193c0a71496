"""Training data, training loop and comparison runs of the learned correction (helm_net_* of the C-ABI).

Every arithmetic step runs in libhelm's kernels: solves, residuals, M^-1, the network's input features and
targets, forward, loss, backward and Adam.  Torch only holds the device buffers and stacks minibatches.

Pairs come from the solver's own runs.  For a medium and right-hand side b, x* is the flexible-GMRES
solution at a tight tolerance and x_k the iterate after k iterations (a run with max_iter = k from
x_0 = 0).  The residual v = b - A x_k then has the exact preconditioned image A^-1 v = x* - x_k, and the
network learns the part that M^-1 misses, relative to the size of M^-1 v:
    target = (x* - x_k - M^-1 v) / RMS(M^-1 v).
"""
import time

import numpy as np

from . import helm, media


def high_contrast(n, seed, ppw=8.0, device="cuda"):
    """Layered medium with k^2/k0^2 ~ U[0.5, 1.8] plus 5 spherical inclusions, ~ppw points per wavelength."""
    return media.layered(n, seed, ppw=ppw, nlayers=8, lo=0.5, hi=1.8, nspheres=5, device=device, as_numpy=False)


def _solver(n, k2, k0, order, max_iter, rtol, precision=helm.HELM_PREC_TF32):
    return helm.Solver((n, n, n), k2, k0, order=order, precond=helm.HELM_PRECOND_EIGT, precision=precision,
                       restart=30, max_iter=max_iter, rtol=rtol, flexible=True)


def bumps_medium(n, seed, ppw=10.0, device="cuda"):
    """Sum of 20 Gaussian bumps of contrast U(-0.3, 0.3), ~ppw points per wavelength, seeded direction."""
    return media.bumps(n, seed, seed + 1000, ppw=ppw, device=device, as_numpy=False)


def generate_pairs(n=96, seeds=range(6), iters=(0, 2, 4, 7, 11, 16), arnoldi=6, order=6, ppw=8.0, rtol_star=1e-9,
                   medium=high_contrast, net=None):
    """Features X (bfloat16 [P][5][n][n][n]) and targets T (float32 [P][2][n][n][n]) on the GPU.

    Two kinds of pairs per medium:
      residual pairs   v = b - A x_k for the iterates x_k of the solver's own run (k in `iters`), with
                       A^-1 v = x* - x_k; used only when the reference solve x* reached rtol_star.
      Krylov pairs     v_0 = b, z_j = M^-1 v_j, w_j = A z_j, v_{j+1} = w_j (j < `arnoldi`): the vectors A z_j
                       that right-preconditioned GMRES orthogonalises, with the exact image A^-1 w_j = z_j.
    """
    import torch
    if net is None:
        net = helm.Net(1)   # only its statistics scratch is used by the feature and target kernels
    Xs, Ts = [], []
    for seed in seeds:
        k2, f, k0 = medium(n, seed, ppw=ppw)
        S = _solver(n, k2, k0, order, 600, rtol_star)
        b = S.build_rhs(f)
        if iters:
            xs, info = S.solve(b, check=False)
            if info.status == 0:
                for k in iters:
                    if k == 0:
                        xk = torch.zeros_like(b)
                    else:
                        Sk = _solver(n, k2, k0, order, k, 1e-14)
                        xk, _ = Sk.solve(b, check=False)
                        Sk.close()
                    v = torch.empty(S.shape, dtype=torch.complex64, device=b.device)
                    helm.helm_residual(S.ctx, b, xk, v)
                    mv = S.apply_precond(v)
                    Xs.append(S.features(net, v, mv))
                    Ts.append(S.target(net, xs, xk, mv))
        v = b.to(torch.complex64)
        zero = torch.zeros_like(b)
        for j in range(arnoldi):
            z = S.apply_precond(v)
            w = S.apply_A(z)
            mw = S.apply_precond(w)
            Xs.append(S.features(net, w, mw))
            Ts.append(S.target(net, z.to(torch.complex128), zero, mw))
            v = w
        S.close()
    torch.cuda.synchronize()
    return torch.stack(Xs), torch.stack(Ts)


def train(net, X, T, steps=300, batch=2, lr=2e-3, lr_final=2e-4, seed=0, log_every=25):
    """Adam on 0.5 mean((N(x) - t)^2) over random minibatches; returns the logged (step, loss) pairs."""
    import torch
    rng = np.random.default_rng(seed)
    P = X.shape[0]
    loss = torch.zeros(1, dtype=torch.float64, device=X.device)
    gy = None
    log = []
    acc, cnt = 0.0, 0
    for it in range(steps):
        idx = torch.as_tensor(rng.choice(P, size=min(batch, P), replace=False), device=X.device)
        xb = X.index_select(0, idx).contiguous()
        tb = T.index_select(0, idx).contiguous()
        net.zero_grad()
        y = net.forward(xb)
        if gy is None or gy.shape != y.shape:
            gy = torch.empty_like(y)
        loss.zero_()
        helm.helm_net_mse(y, tb, gy, loss)
        net.backward(gy)
        a = it / max(1, steps - 1)
        net.adam(lr=float(lr * (lr_final / lr) ** a))
        acc += float(loss.item())
        cnt += 1
        if (it + 1) % log_every == 0 or it == steps - 1:
            log.append((it + 1, acc / cnt))
            acc, cnt = 0.0, 0
    return log


def evaluate(net, X, T, batch=2):
    """Mean loss over a set, and the loss of the zero correction (0.5 mean t^2) for scale."""
    import torch
    loss = torch.zeros(1, dtype=torch.float64, device=X.device)
    tot, base = 0.0, 0.0
    for i in range(0, X.shape[0], batch):
        xb, tb = X[i:i + batch].contiguous(), T[i:i + batch].contiguous()
        y = net.forward(xb)
        gy = torch.empty_like(y)
        loss.zero_()
        helm.helm_net_mse(y, tb, gy, loss)
        tot += float(loss.item()) * xb.shape[0]
        loss.zero_()
        helm.helm_net_mse(torch.zeros_like(tb), tb, gy, loss)
        base += float(loss.item()) * xb.shape[0]
    return tot / X.shape[0], base / X.shape[0]


def compare(net, n, seed, order=6, ppw=8.0, rtol=1e-6, max_iter=600, medium=high_contrast, repeats=2):
    """FGMRES(30) with EigT, with and without the network: iterations, time, true relative residual."""
    import torch
    k2, f, k0 = medium(n, seed, ppw=ppw)
    out = {}
    sols = {}
    for name in ("plain", "learned"):
        S = _solver(n, k2, k0, order, max_iter, rtol)
        if name == "learned":
            S.attach(net)
        b = S.build_rhs(f)
        best = None
        st0 = net.stats()
        for _ in range(repeats):
            x = torch.zeros_like(b)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            _, info = S.solve(b, x0=x, check=False)
            torch.cuda.synchronize()
            dt = time.perf_counter() - t0
            best = dt if best is None else min(best, dt)
        out[name] = {"iterations": info.iterations, "seconds": best, "relres_true": info.relres_true,
                     "status": info.status}
        sols[name] = x
        if name == "learned":
            st = net.stats() - st0
            out[name]["dropped"] = float(st[3])
            out[name]["applied"] = float(st[4])
            out[name]["mean_residual_ratio"] = float(st[5] / max(st[4], 1.0))
            S.attach(None)
        S.close()
    d = (sols["learned"] - sols["plain"]).abs().pow(2).sum().sqrt() / sols["plain"].abs().pow(2).sum().sqrt()
    out["solution_rel_diff"] = float(d)
    return out


def forward_timing(n, width, reps=5, seed=1):
    """CUDA-event milliseconds of one network forward on a single n^3 field (a fresh network of the given
    width; the five input channels random)."""
    import torch
    net = helm.Net(width, seed=seed)
    x = torch.randn((1, 5, n, n, n), device="cuda").to(torch.bfloat16)
    net.forward(x)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    for _ in range(reps):
        net.forward(x)
    e1.record()
    torch.cuda.synchronize()
    net.close()
    return e0.elapsed_time(e1) / reps


if __name__ == "__main__":
    # python -m paper_2602_07711_gb300.learned N WIDTH [REPS]: time the network's forward on one N^3 field
    import sys
    n_, w_ = int(sys.argv[1]), int(sys.argv[2])
    reps_ = int(sys.argv[3]) if len(sys.argv) > 3 else 5
    print("width %d, %d^3: %.3f ms per forward" % (w_, n_, forward_timing(n_, w_, reps_)))
