"""helm_gmres_solve with the right-hand side and the iterate in host memory.

Device buffers are used in place; page-locked host memory that is mapped into the device address space
(torch's pin_memory) is read and written by the conversion kernels directly; other host memory (a numpy
array) is staged through device buffers of the context.  All three must run the same iteration on the same
values, so the solutions agree bit for bit, with the same iteration counts, and a nonzero x0 given in host
memory is honoured (the same nonzero x0 on the device and in mapped host memory gives the same solve).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2602_07711_gb300 import HELM_PREC_TF32, Solver, helm, media


def test_host_and_device_buffers_give_the_same_solve():
    n = 48
    k2, f, k0 = media.bumps(n, 7, 8)
    S = Solver((n, n, n), k2, k0, order=6, precision=HELM_PREC_TF32, flexible=True, rtol=1e-6)
    F = S.build_rhs(torch.from_numpy(f).cuda())
    runs = {}
    # device
    xd = torch.zeros_like(F)
    code, inf = helm.helm_gmres_solve(S.ctx, F, xd)
    assert code == 0
    runs["device"] = (xd.cpu().numpy(), inf.iterations)
    # page-locked, mapped host memory
    Fp = F.cpu().pin_memory()
    xp = torch.zeros(F.shape, dtype=F.dtype).pin_memory()
    code, inf = helm.helm_gmres_solve(S.ctx, Fp, xp)
    assert code == 0
    runs["pinned"] = (xp.numpy().copy(), inf.iterations)
    # pageable host memory (numpy)
    Fn = np.ascontiguousarray(F.cpu().numpy())
    xn = np.zeros_like(Fn)
    code, inf = helm.helm_gmres_solve(S.ctx, Fn, xn)
    assert code == 0
    runs["pageable"] = (xn.copy(), inf.iterations)
    ref, its = runs["device"]
    for name, (x, it) in runs.items():
        assert it == its, (name, it, its)
        assert np.array_equal(x, ref), name
    # a nonzero x0 (half the solution plus a perturbation) given on the device and in mapped host memory
    x0 = 0.5 * ref + 1e-3 * np.random.default_rng(3).standard_normal(ref.shape)
    xd = torch.from_numpy(x0.copy()).cuda()
    code, inf_d = helm.helm_gmres_solve(S.ctx, F, xd)
    assert code == 0
    xp = torch.from_numpy(x0.copy()).pin_memory()
    code, inf_p = helm.helm_gmres_solve(S.ctx, Fp, xp)
    assert code == 0 and inf_p.iterations == inf_d.iterations
    assert np.array_equal(xp.numpy(), xd.cpu().numpy())
    S.close()
