"""helm_residual_noalloc: the allocation-free residual for callers that cannot call cudaMalloc (graph
capture, frozen memory pools).  It must agree with helm_residual, the entry point that allocates its
workspace, on consecutive calls (the shared static scratch keeps the previous call's contents), and reject
problems above its stated limit.  Collected last so that a failure here does not hide other results."""
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


def test_noalloc_residual_matches_allocating_entry_point():
    n = 48
    h = 1.0 / n
    k0 = 2 * math.pi / (10 * h)
    g = np.arange(n) * h + h / 2
    Z, Y, X = np.meshgrid(g, g, g, indexing="ij")
    k2 = k0 * k0 * (1 + 0.2 * np.exp(-((X - .5) ** 2 + (Y - .5) ** 2 + (Z - .5) ** 2) / 0.02)) + 0j
    S = Solver((n, n, n), k2, k0, order=6)
    F = _dev(_rand(k2.shape, 1))
    for call in range(2):
        x = _dev(_rand(k2.shape, 10 + call))
        r_ref = torch.empty(k2.shape, dtype=torch.complex64, device="cuda")
        r_na = torch.empty(k2.shape, dtype=torch.complex64, device="cuda")
        n2_ref, ni_ref = helm.helm_residual(S.ctx, F, x, r_ref)
        code, n2, ni = helm.helm_residual_noalloc(S.ctx, F, x, r_na)
        assert code == 0
        assert abs(n2 - n2_ref) <= 1e-12 * n2_ref and abs(ni - ni_ref) <= 1e-12 * ni_ref
        assert torch.equal(r_na, r_ref)


def test_noalloc_rejects_problems_above_its_limit():
    n = (130, 130, 130)            # 2,197,000 points > 2^21
    k0 = 10.0
    S = Solver(n, np.full((130, 130, 130), k0 * k0, complex), k0, order=2)
    b = torch.zeros((130, 130, 130), dtype=torch.complex128, device="cuda")
    r = torch.empty((130, 130, 130), dtype=torch.complex64, device="cuda")
    code, _, _ = helm.helm_residual_noalloc(S.ctx, b, b, r)
    assert code == 1                # HELM_ERR_ARG
