"""Batched solves (helm_gmres_solve_batched): many problems of uneven size times several right-hand sides in
one CUDA graph with device-side control.  Every (problem, right-hand side) pair must give what the single
solve of the same pair gives: the same kernels run on the same data in the same order, so iteration counts
are equal and the solutions agree to rounding; the single solve itself is checked against the oracle in
test_gpu_parity.py, and the true residual of every batched solution is checked here as well.
"""
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2602_07711_gb300 import (HELM_PREC_FP32, HELM_PREC_TF32, HELM_PRECOND_PFFT, Batch, Solver, helm, media,
                                    solve_batched)


def _problem(n, seed, ppw, nrhs, order, precision, flexible, restart=30, max_iter=300, rtol=1e-6):
    fs = []
    for r in range(nrhs):
        k2, f, k0 = media.bumps(n, seed, 100 + 7 * seed + r, ppw=ppw, device="cuda", as_numpy=False)
        fs.append(f)
    S = Solver((n, n, n), k2, k0, order=order, precision=precision, flexible=flexible, restart=restart,
               max_iter=max_iter, rtol=rtol)
    B = torch.stack([S.build_rhs(f) for f in fs]).contiguous()
    return S, B


def _rel(a, b):
    return float((a - b).abs().pow(2).sum().sqrt() / b.abs().pow(2).sum().sqrt())


def _check_against_single(Ss, Bs, xs, infos):
    for S, B, X, inf in zip(Ss, Bs, xs, infos):
        for r in range(B.shape[0]):
            x1, i1 = S.solve(B[r].contiguous(), check=False)
            assert inf[r].status == i1.status == 0, (inf[r].as_dict(), i1.as_dict())
            assert inf[r].iterations == i1.iterations and inf[r].restarts == i1.restarts
            assert inf[r].cycle_its[:i1.restarts] == i1.cycle_its[:i1.restarts]
            assert _rel(X[r], x1) < 1e-9, _rel(X[r], x1)
            n2, _ = S.residual(B[r].contiguous(), X[r].contiguous())
            b2, _ = S.residual(B[r].contiguous(), torch.zeros_like(X[r]))
            assert n2 / b2 <= S.options.rtol * 1.001


def test_uneven_batch_matches_single_solves():
    Ss, Bs = [], []
    for (n, order, prec, flex, ppw) in [(24, 4, HELM_PREC_FP32, False, 8.0), (36, 6, HELM_PREC_TF32, True, 10.0),
                                        (40, 6, HELM_PREC_FP32, True, 6.0), (32, 4, HELM_PREC_TF32, True, 12.0)]:
        S, B = _problem(n, n, ppw, 2, order, prec, flex)
        Ss.append(S)
        Bs.append(B)
    xs, infos = solve_batched(Ss, Bs)
    _check_against_single(Ss, Bs, xs, infos)


def test_batch_with_restarts_warm_start_and_mixed_outcomes():
    S1, B1 = _problem(32, 3, 8.0, 3, 6, HELM_PREC_TF32, True, restart=5, max_iter=200)
    S2, B2 = _problem(28, 4, 8.0, 3, 4, HELM_PREC_FP32, False, restart=2, max_iter=3)   # cannot converge in 3
    B1[1].zero_()                                   # a zero right-hand side: nothing to do
    x0 = torch.zeros_like(B2)
    x0[2], _ = S2.solve(B2[2].contiguous(), check=False)   # warm start from 3 iterations
    xs, infos = solve_batched([S1, S2], [B1, B2], x0s=[torch.zeros_like(B1), x0.clone()])
    assert infos[0][1].status == 0 and infos[0][1].iterations == 0
    assert float(xs[0][1].abs().max()) == 0.0
    for r in (0, 2):
        assert infos[0][r].status == 0 and infos[0][r].restarts >= 2
    for r in range(3):
        assert infos[1][r].status == 8 and infos[1][r].iterations == 3   # HELM_ERR_NOT_CONVERGED
    # each lane equals the single solve from the same start
    for r in (0, 2):
        x1, i1 = S1.solve(B1[r].contiguous(), check=False)
        assert i1.iterations == infos[0][r].iterations and _rel(xs[0][r], x1) < 1e-9
    for r in range(3):
        x1, i1 = S2.solve(B2[r].contiguous(), x0=x0[r].clone(), check=False)
        assert i1.iterations == infos[1][r].iterations
        assert _rel(xs[1][r], x1) < 1e-9


def test_batch_plan_runs_repeatedly_and_matches_the_one_shot_call():
    Ss, Bs = [], []
    for (n, order, prec, flex, ppw) in [(24, 6, HELM_PREC_TF32, True, 8.0), (32, 4, HELM_PREC_FP32, True, 10.0)]:
        S, B = _problem(n, n + 1, ppw, 3, order, prec, flex)
        Ss.append(S)
        Bs.append(B)
    Xs = [torch.zeros_like(B) for B in Bs]
    plan = Batch(Ss, Bs, Xs)
    _, inf1 = plan.run()
    x1 = [X.clone() for X in Xs]
    for X in Xs:
        X.zero_()
    _, inf2 = plan.run()
    xs, inf3 = solve_batched(Ss, Bs)
    for p in range(2):
        assert torch.equal(Xs[p], x1[p])
        assert _rel(xs[p], Xs[p]) < 1e-12
        for r in range(3):
            assert inf1[p][r].iterations == inf2[p][r].iterations == inf3[p][r].iterations
            assert inf1[p][r].status == 0
    # new right-hand sides in the same buffers
    Bs[0][0].mul_(2.0)
    for X in Xs:
        X.zero_()
    _, inf4 = plan.run()
    assert _rel(Xs[0][0], 2.0 * x1[0][0]) < 1e-5 and inf4[0][0].status == 0
    plan.close()


def test_batch_rejects_bad_arguments():
    S, B = _problem(16, 1, 8.0, 1, 4, HELM_PREC_FP32, False)
    X = torch.zeros_like(B)
    code, _ = helm.helm_gmres_solve_batched([S.ctx, S.ctx], [B, B], [X, X], 1)
    assert code == 1
    k2, f, k0 = media.bumps(16, 1, 2, ppw=8.0, device="cuda", as_numpy=False)
    P = Solver((16, 16, 16), k2, k0, order=4, precond=HELM_PRECOND_PFFT, flexible=True)
    code, _ = helm.helm_gmres_solve_batched([P.ctx], [B], [X], 1)
    assert code == 10
    code = helm.lib().helm_gmres_solve_batched(None, 1, None, None, 1, None, None)
    assert code == 1


def test_autotune_picks_a_count_and_keeps_the_solution():
    S, B = _problem(48, 5, 8.0, 1, 6, HELM_PREC_TF32, True)
    x0, i0 = S.solve(B[0].contiguous())
    nb, var, dv = S.autotune()
    # matvec variants 0-4 (include/helm.h: helm_set_matvec_variant), inner-product variants 0-2
    assert nb > 0 and var in range(5) and dv in (0, 1, 2) and (nb, var, dv) == S.autotune()
    x1, i1 = S.solve(B[0].contiguous())
    assert abs(i1.iterations - i0.iterations) <= 1
    assert _rel(x1, x0) < 1e-5
