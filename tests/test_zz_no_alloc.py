"""helm_residual_noalloc: the residual for callers that cannot allocate device memory while they run (an
application whose memory pool owns the device after warm-up, a runtime that forbids cudaMalloc/cudaFree
between its steps).  It must work on a context that has never allocated its Krylov workspace, leave the
device's free memory unchanged, agree with helm_residual (the entry point that allocates its workspace) on
two consecutive calls (the shared static scratch keeps the previous call's contents), and reject problems
above its stated limit.  Collected last so that a failure here does not hide other results."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2602_07711_gb300 import Solver, helm


def _rand(shape, seed):
    r = np.random.default_rng(seed)
    return r.standard_normal(shape) + 1j * r.standard_normal(shape)


def _dev(a, dtype=torch.complex128):
    return torch.from_numpy(np.ascontiguousarray(a)).to(device="cuda", dtype=dtype)


def _medium(n):
    h = 1.0 / n
    k0 = 2 * math.pi / (10 * h)
    g = np.arange(n) * h + h / 2
    Z, Y, X = np.meshgrid(g, g, g, indexing="ij")
    k2 = k0 * k0 * (1 + 0.2 * np.exp(-((X - .5) ** 2 + (Y - .5) ** 2 + (Z - .5) ** 2) / 0.02)) + 0j
    return k2, k0


def test_noalloc_residual_matches_allocating_entry_point():
    n = 48
    k2, k0 = _medium(n)
    F = _dev(_rand(k2.shape, 1))
    r_na = torch.empty(k2.shape, dtype=torch.complex64, device="cuda")
    # the first call on the device may load the library's device code and look up the array's address
    warm = Solver((n, n, n), k2, k0, order=6)
    code, _, _ = helm.helm_residual_noalloc(warm.ctx, F, F, r_na)
    assert code == 0
    warm.close()
    # a fresh context, whose Krylov workspace has never been allocated: the no-alloc call comes first
    S = Solver((n, n, n), k2, k0, order=6)
    xs = [_dev(_rand(k2.shape, 10 + call)) for call in range(2)]
    got = []
    for x in xs:
        code, n2, ni = helm.helm_residual_noalloc(S.ctx, F, x, r_na)
        assert code == 0
        got.append((n2, ni, r_na.clone()))
    # the allocating entry point on the same inputs, after the no-alloc calls
    for x, (n2, ni, r_got) in zip(xs, got):
        r_ref = torch.empty(k2.shape, dtype=torch.complex64, device="cuda")
        n2_ref, ni_ref = helm.helm_residual(S.ctx, F, x, r_ref)
        assert abs(n2 - n2_ref) <= 1e-12 * n2_ref and abs(ni - ni_ref) <= 1e-12 * ni_ref
        assert torch.equal(r_got, r_ref)
    # and once more the other way round: no-alloc after helm_residual on the same context
    code, n2, ni = helm.helm_residual_noalloc(S.ctx, F, xs[0], r_na)
    assert code == 0 and n2 == got[0][0] and ni == got[0][1] and torch.equal(r_na, got[0][2])
    S.close()


def test_noalloc_leaves_free_memory_unchanged():
    n = 40
    k2, k0 = _medium(n)
    F = _dev(_rand(k2.shape, 2))
    x = _dev(_rand(k2.shape, 3))
    r = torch.empty(k2.shape, dtype=torch.complex64, device="cuda")
    S = Solver((n, n, n), k2, k0, order=4)
    code, _, _ = helm.helm_residual_noalloc(S.ctx, F, x, r)     # loads the device code if not loaded yet
    assert code == 0
    S.close()
    S = Solver((n, n, n), k2, k0, order=4)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(2):
        code, _, _ = helm.helm_residual_noalloc(S.ctx, F, x, r)
        assert code == 0
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    S.close()


def test_noalloc_rejects_problems_above_its_limit():
    n = (130, 130, 130)            # 2,197,000 points > 2^21
    k0 = 10.0
    S = Solver(n, np.full((130, 130, 130), k0 * k0, complex), k0, order=2)
    b = torch.zeros((130, 130, 130), dtype=torch.complex128, device="cuda")
    r = torch.empty((130, 130, 130), dtype=torch.complex64, device="cuda")
    code, _, _ = helm.helm_residual_noalloc(S.ctx, b, b, r)
    assert code == 1                # HELM_ERR_ARG
    S.close()
