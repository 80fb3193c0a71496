"""Failure detection through the C-ABI, in forms that fault, trap or hang no GPU: bad data injected on the
host (a NaN in the right-hand side), a solve capped at max_iter, and the bounded mbarrier waits of the
tensor-core transforms (and, with the FP16 Krylov basis, of the inner products staged by bulk copies) made
to run out by a limit of one poll (the waits return, the kernels drain what they have in flight, free
their tensor memory and report HELM_ERR_ITER_LIMIT; the context stays usable).
"""
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2602_07711_gb300 import HELM_PREC_FP16, HELM_PREC_TF32, Solver, media

HELM_ERR_NAN, HELM_ERR_NOT_CONVERGED, HELM_ERR_ITER_LIMIT = 6, 8, 9


def _problem(n=32):
    k2, f, k0 = media.single_gaussian(n)
    return k2, torch.from_numpy(f).cuda(), k0


@pytest.mark.parametrize("where", ["rhs", "x0"])
def test_nan_in_the_input_returns_helm_err_nan(where):
    n = 32
    k2, f, k0 = _problem(n)
    S = Solver((n, n, n), k2, k0, order=4, rtol=1e-6)
    F = S.build_rhs(f)
    x0 = torch.zeros_like(F)
    if where == "rhs":
        F[5, 6, 7] = complex(float("nan"), 0.0)
    else:
        x0[1, 2, 3] = complex(0.0, float("nan"))
    _, info = S.solve(F, x0=x0, check=False)
    assert info.status == HELM_ERR_NAN
    S.close()


def test_solve_capped_at_max_iter_returns_not_converged_with_the_last_iterate():
    n = 32
    k2, f, k0 = _problem(n)
    S = Solver((n, n, n), k2, k0, order=4, rtol=1e-12, restart=30, max_iter=3)
    F = S.build_rhs(f)
    x, info = S.solve(F, check=False)
    assert info.status == HELM_ERR_NOT_CONVERGED
    assert info.iterations == 3 and 0 < info.relres_true < 1
    # x holds the iterate the reported residual belongs to
    n2, _ = S.residual(F, x)
    assert abs(n2 / info.beta0 - info.relres_true) <= 1e-6 * info.relres_true
    assert torch.count_nonzero(x) == x.numel()
    # the same iterate as an uncapped solver's after its first three steps (the cap ends the cycle there)
    S3 = Solver((n, n, n), k2, k0, order=4, rtol=1e-12, restart=3, max_iter=3)
    x3, info3 = S3.solve(F, check=False)
    assert info3.iterations == 3
    assert torch.allclose(x, x3, rtol=0, atol=1e-12 * float(x3.abs().max()))
    S.close()
    S3.close()


@pytest.mark.parametrize("prec", [HELM_PREC_TF32, HELM_PREC_FP16])
def test_expired_tensor_core_waits_return_iter_limit_and_leave_the_context_usable(prec):
    n = 64
    k2, f, k0 = media.bumps(n, 21, 22)
    fd = torch.from_numpy(f).cuda()
    S = Solver((n, n, n), k2, k0, order=6, precision=prec, flexible=True, rtol=1e-6, max_iter=4)
    F = S.build_rhs(fd)
    S.set_wait_limit(1)        # one poll: the epilogue cannot see a whole tile finished in one poll
    _, info = S.solve(F, check=False)
    assert info.status == HELM_ERR_ITER_LIMIT
    # back to the default bound: the same context solves, and agrees with a fresh one
    S.set_wait_limit(0)
    ref = Solver((n, n, n), k2, k0, order=6, precision=prec, flexible=True, rtol=1e-6, max_iter=300)
    xr, ir = ref.solve(F)
    S2 = Solver((n, n, n), k2, k0, order=6, precision=prec, flexible=True, rtol=1e-6, max_iter=300)
    S2.set_wait_limit(1)
    S2.solve(F, check=False)
    S2.set_wait_limit(0)
    x2, i2 = S2.solve(F)
    assert i2.status == 0 and i2.iterations == ir.iterations
    assert torch.equal(x2, xr)
    for s in (S, S2, ref):
        s.close()


def test_wait_limit_rejects_negative_values():
    from paper_2602_07711_gb300 import helm
    n = 16
    k2, f, k0 = _problem(n)
    S = Solver((n, n, n), k2, k0, order=4)
    with pytest.raises(helm.HelmError):
        S.set_wait_limit(-1)
    S.close()
