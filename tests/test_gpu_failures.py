"""Failure paths of the solver, driven from the host (no GPU fault).

* A bounded device wait that runs out: the CD sweep's grid barrier is told to
  wait for one arrival more than the grid holds, with a short limit, so every
  wait runs to its limit; the kernel returns early, the call reports
  GLASSO_ETIMEOUT and the context stays usable.
* Section 6.1.2's backtracking running out of trials: a knob rejects every
  line-search trial, giving GLASSO_ELINESEARCH.
* The cycle limit: max_cycles = 1 with a tolerance the first cycle cannot
  reach gives GLASSO_EMAXITER, with the iterate returned.
"""
import numpy as np
import pytest

import oracle
from paper_1607_00315_gb300 import synth

pytestmark = pytest.mark.gpu

N, M, LAM, SEED = 200, 400, 0.1, 41


@pytest.fixture(scope="module")
def problem():
    p = synth.random_problem(N, M, LAM, SEED, gen="sparse")
    S = oracle.form_S(p.X)
    A_ref, _, info_ref, _ = oracle.solve(S, LAM, tol=1e-10)
    assert info_ref["status"] == 0
    return S, A_ref, info_ref


def _context(precision):
    import torch

    from paper_1607_00315_gb300 import build, glasso

    build.build()
    torch.cuda.init()
    return glasso.Context(0, precision=glasso.MIXED if precision == "mixed" else glasso.FP64)


def _solve_ok(ctx, S, A_ref, info_ref):
    A, _, info = ctx.solve(S, LAM, tol=1e-10)
    assert info["status"] == 0
    assert np.abs(A - A_ref).max() <= 1e-7
    _, F = oracle.objective(S, A, LAM)
    assert abs(F - info_ref["objective"]) <= 1e-9 * abs(info_ref["objective"])


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_cd_barrier_wait_runs_out(problem, precision):
    from paper_1607_00315_gb300 import glasso

    S, A_ref, info_ref = problem
    ctx = _context(precision)
    try:
        # about 1 ms of SM cycles per wait, on a count that nothing completes
        ctx.set_debug(glasso.DEBUG_WAIT_CYCLES, 2_000_000)
        ctx.set_debug(glasso.DEBUG_WAIT_UNREACHABLE, 1)
        prof0 = ctx.get_profile(reset=True)["paths"]
        assert isinstance(prof0, dict)
        A_out = np.full((N, N), 7.0)
        _, _, info = ctx.solve(S, LAM, tol=1e-10, A_out=A_out, check=False)
        assert info["status"] == glasso.ETIMEOUT, info
        assert "grid-barrier wait expired" in ctx.L.glasso_last_error(ctx.h).decode()
        assert np.all(A_out == 7.0)  # A_out is not written on a timeout
        paths = ctx.get_profile()["paths"]
        assert paths["cd_lag2"] + paths["cd_persist32"] + paths["cd_chain64"] >= 1
        # the step-level sweep reports the same
        _, L = oracle.cholesky(np.diag(1.0 / (np.diag(S) + LAM)))
        W = oracle.inverse_from_chol(L)
        A0 = np.diag(1.0 / (np.diag(S) + LAM))
        fi, fj = oracle.free_set(S, W, A0, LAM)
        import torch

        dev = [torch.from_numpy(np.ascontiguousarray(x)).cuda() for x in (S, W, A0)]
        pi = torch.from_numpy(fi).cuda()
        pj = torch.from_numpy(fj).cuda()
        D = torch.zeros(len(fi), dtype=torch.float64, device="cuda")
        U = torch.zeros((N, N), dtype=torch.float64, device="cuda")
        with pytest.raises(glasso.GlassoError) as e:
            ctx.cd_sweeps(*dev, LAM, pi, pj, 1, D, U)
        assert e.value.status == glasso.ETIMEOUT
        # back to the default limit: the same context solves to the oracle's bar
        ctx.set_debug(glasso.DEBUG_WAIT_UNREACHABLE, 0)
        ctx.set_debug(glasso.DEBUG_WAIT_CYCLES, 0)
        _solve_ok(ctx, S, A_ref, info_ref)
    finally:
        ctx.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_line_search_runs_out_of_trials(problem, precision):
    from paper_1607_00315_gb300 import glasso

    S, A_ref, info_ref = problem
    ctx = _context(precision)
    try:
        ctx.set_debug(glasso.DEBUG_LS_REJECT, 1)
        A, _, info = ctx.solve(S, LAM, tol=1e-10, check=False)
        assert info["status"] == glasso.ELINESEARCH, info
        # the first relaxation's search took all of its trials and stopped the solve
        assert info["ls_trials"] == 30 and info["relaxations"] >= 1
        # the returned iterate is the starting point, untouched
        assert np.array_equal(A, np.diag(1.0 / (np.diag(S) + LAM)))
        if precision == "fp64":
            # the step-level search: every trial rejected
            import torch

            A0 = np.diag(1.0 / (np.diag(S) + LAM))
            _, L = oracle.cholesky(A0)
            W = oracle.inverse_from_chol(L)
            fi, fj = oracle.free_set(S, W, A0, LAM)
            D, _ = oracle.cd_sweeps(S, W, A0, LAM, fi, fj, 1)
            _, F0 = oracle.objective(S, A0, LAM)
            dev = [torch.from_numpy(np.ascontiguousarray(x)).cuda() for x in (S, W, A0)]
            s, _, al, tr = ctx.line_search(*dev, LAM, torch.from_numpy(fi).cuda(),
                                           torch.from_numpy(fj).cuda(), torch.from_numpy(D).cuda(),
                                           F0, max_trials=12)
            assert s == glasso.ELINESEARCH and tr == 12 and al == 0.0
            assert np.array_equal(dev[2].cpu().numpy(), A0)  # A unchanged
        ctx.set_debug(glasso.DEBUG_LS_REJECT, 0)
        _solve_ok(ctx, S, A_ref, info_ref)
    finally:
        ctx.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_cycle_limit(problem, precision):
    from paper_1607_00315_gb300 import glasso

    S, A_ref, info_ref = problem
    ctx = _context(precision)
    try:
        A, _, info = ctx.solve(S, LAM, tol=1e-14, max_cycles=1, check=False)
        assert info["status"] == glasso.EMAXITER, info
        assert info["cycles"] == 1
        # the oracle's own single cycle stops the same way, at the same point
        A1, _, info1, _ = oracle.solve(S, LAM, tol=1e-14, max_cycles=1)
        assert info1["status"] == oracle.EMAXITER and info1["relaxations"] == info["relaxations"]
        # FP64: the same steps up to rounding; mixed: FP32 sweeps give a nearby iterate
        assert np.abs(A - A1).max() <= (1e-6 if precision == "fp64" else 1e-3)
        # the iterate returned is positive definite and its objective is below F(A0)
        assert oracle.cholesky(A)[0] == 0
        _, F0 = oracle.objective(S, np.diag(1.0 / (np.diag(S) + LAM)), LAM)
        assert info["objective"] < F0
        assert info["rel_kkt"] > 1e-14
    finally:
        ctx.close()


def test_unknown_knob_is_rejected():
    from paper_1607_00315_gb300 import glasso

    ctx = _context("fp64")
    try:
        with pytest.raises(glasso.GlassoError) as e:
            ctx.set_debug(99, 1)
        assert e.value.status == glasso.EINVAL
        with pytest.raises(glasso.GlassoError) as e:
            ctx.set_debug(glasso.DEBUG_WAIT_CYCLES, -1)
        assert e.value.status == glasso.EINVAL
    finally:
        ctx.close()
