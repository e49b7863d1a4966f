"""GPU parity of the PCD-CG Newton-direction solver (glasso_pcd) and of whole
solves with it as the inner solver, against the oracle (orc_pcd,
orc_solve(..., inner = PCD-CG)).

The GPU carries b = G + (W Delta W) across iterations (adding t (W P W) and the
exact zeros' corrections) where the oracle recomputes it from U = Delta W, so
the two agree to rounding: on the FP64 path Delta and U to 1e-9 of their
largest entry and the iteration counts exactly.  On the mixed path the
products with W are FP32 sums of n terms (relative error up to about
n 2^-24 each), held to 1e-4 of the largest entry after a few iterations.
"""
import numpy as np
import pytest

import oracle
from paper_1607_00315_gb300 import synth

pytestmark = pytest.mark.gpu


def _context(precision):
    import torch

    from paper_1607_00315_gb300 import build, glasso

    build.build()
    torch.cuda.init()
    return glasso.Context(0, precision=glasso.MIXED if precision == "mixed" else glasso.FP64)


@pytest.fixture(scope="module")
def ctx():
    c = _context("fp64")
    yield c
    c.close()


@pytest.fixture(scope="module")
def mctx():
    c = _context("mixed")
    yield c
    c.close()


def _state(n, m, lam, seed, gen="sparse", cycles=1):
    """An iterate after `cycles` oracle ML-cycles (or A0 for cycles = 0), its
    inverse and its level-0 free set."""
    p = synth.random_problem(n, m, lam, seed, gen=gen)
    S = oracle.form_S(p.X)
    if cycles > 0:
        A, _, _, _ = oracle.solve(S, lam, tol=1e-14, max_cycles=cycles)
    else:
        A = np.diag(1.0 / (np.diag(S) + lam))
    _, L = oracle.cholesky(A)
    W = oracle.inverse_from_chol(L)
    fi, fj = oracle.free_set(S, W, A, lam)
    return S, W, A, fi, fj


def _same_stop(S, W, A, lam, fi, fj, k, k_ref, D, U, scale):
    """Equal iteration counts -- except once the LASSO is solved to rounding,
    where the stopping rule (d = 0, or a zero step) is decided by rounding
    noise: the oracle's own direction at the GPU's Delta then vanishes to
    rounding."""
    if k != k_ref:
        d_chk, _ = oracle.pcd_direction(S, W, A, lam, fi, fj, D=D, U=U)
        assert np.abs(d_chk).max() <= 1e-12 * scale, (k, k_ref)


def _dev(*xs):
    import torch

    return [torch.from_numpy(np.ascontiguousarray(x)).cuda() for x in xs]


CASES = [
    (60, 120, 0.1, 11, "sparse", 0),
    (150, 300, 0.1, 12, "sparse", 1),
    (257, 200, 0.08, 13, "sparse", 2),   # m < n, a ragged tail of the 32 x 128 SpMM blocks
    (100, 200, 0.2, 14, "tridiag", 1),
]


@pytest.mark.parametrize("iters", [1, 3, 12])
@pytest.mark.parametrize("n,m,lam,seed,gen,cycles", CASES)
def test_pcd_cg_matches_oracle(ctx, n, m, lam, seed, gen, cycles, iters):
    import torch

    S, W, A, fi, fj = _state(n, m, lam, seed, gen, cycles)
    D_ref, U_ref, k_ref = oracle.pcd(S, W, A, lam, fi, fj, iters, cg=True)
    Sd, Wd, Ad, pi, pj = _dev(S, W, A, fi, fj)
    D = torch.zeros(len(fi), dtype=torch.float64, device="cuda")
    U = torch.full((n, n), np.nan, dtype=torch.float64, device="cuda")  # not read
    k = ctx.pcd(Sd, Wd, Ad, lam, pi, pj, iters, D, U, cg=True)
    D, U = D.cpu().numpy(), U.cpu().numpy()
    _same_stop(S, W, A, lam, fi, fj, k, k_ref, D, U, np.abs(D_ref).max())
    scale = max(np.abs(D_ref).max(), 1e-300)
    assert np.abs(D - D_ref).max() <= 1e-9 * scale
    assert np.abs(U - U_ref).max() <= 1e-9 * max(np.abs(U_ref).max(), 1e-300)
    # exact zeros (A + Delta = 0) agree where the oracle has them
    z_ref = (A[fi, fj] + D_ref) == 0.0
    z = (A[fi, fj] + D) == 0.0
    assert np.array_equal(z, z_ref)


@pytest.mark.parametrize("n,m,lam,seed,gen,cycles", CASES[:2])
def test_plain_pcd_and_precision_stop_match_oracle(ctx, n, m, lam, seed, gen, cycles):
    import torch

    S, W, A, fi, fj = _state(n, m, lam, seed, gen, cycles)
    Sd, Wd, Ad, pi, pj = _dev(S, W, A, fi, fj)
    for cg, iters, rtol in ((False, 6, 0.0), (True, 500, 1e-4)):
        D_ref, U_ref, k_ref = oracle.pcd(S, W, A, lam, fi, fj, iters, cg=cg, rtol=rtol)
        D = torch.zeros(len(fi), dtype=torch.float64, device="cuda")
        U = torch.empty((n, n), dtype=torch.float64, device="cuda")
        k = ctx.pcd(Sd, Wd, Ad, lam, pi, pj, iters, D, U, cg=cg, rtol=rtol)
        Dh = D.cpu().numpy()
        _same_stop(S, W, A, lam, fi, fj, k, k_ref, Dh, U.cpu().numpy(), np.abs(D_ref).max())
        assert np.abs(Dh - D_ref).max() <= 1e-9 * np.abs(D_ref).max()


def test_pcd_continues_from_a_nonzero_delta(ctx):
    """b starts from (W Delta W) of the given Delta: one CD sweep, then PCD-CG."""
    import torch

    n, lam = 150, 0.1
    S, W, A, fi, fj = _state(n, 300, lam, 12, "sparse", 1)
    D0, U0 = oracle.cd_sweeps(S, W, A, lam, fi, fj, 1)
    D_ref, U_ref, k_ref = oracle.pcd(S, W, A, lam, fi, fj, 5, cg=True, D=D0, U=U0)
    Sd, Wd, Ad, pi, pj, D = _dev(S, W, A, fi, fj, D0)
    U = torch.empty((n, n), dtype=torch.float64, device="cuda")
    k = ctx.pcd(Sd, Wd, Ad, lam, pi, pj, 5, D, U, cg=True)
    assert k == k_ref
    assert np.abs(D.cpu().numpy() - D_ref).max() <= 1e-9 * np.abs(D_ref).max()
    assert np.abs(U.cpu().numpy() - U_ref).max() <= 1e-9 * np.abs(U_ref).max()


def test_pcd_empty_pair_list(ctx):
    import torch

    n = 40
    S = np.eye(n)
    Sd, Wd, Ad = _dev(S, S, S)
    pi = torch.empty(0, dtype=torch.int32, device="cuda")
    D = torch.empty(0, dtype=torch.float64, device="cuda")
    U = torch.full((n, n), 3.0, dtype=torch.float64, device="cuda")
    assert ctx.pcd(Sd, Wd, Ad, 0.1, pi, pi, 10, D, U) == 0
    assert float(U.abs().max()) == 0.0


@pytest.mark.parametrize("n,m,lam,seed,gen,cycles", CASES[1:3])
def test_mixed_pcd_matches_oracle(mctx, n, m, lam, seed, gen, cycles):
    import torch

    S, W, A, fi, fj = _state(n, m, lam, seed, gen, cycles)
    D_ref, U_ref, k_ref = oracle.pcd(S, W, A, lam, fi, fj, 3, cg=True)
    Sd, Wd, Ad, pi, pj = _dev(S, W, A, fi, fj)
    D = torch.zeros(len(fi), dtype=torch.float64, device="cuda")
    U = torch.empty((n, n), dtype=torch.float64, device="cuda")
    k = mctx.pcd(Sd, Wd, Ad, lam, pi, pj, 3, D, U, cg=True)
    assert k == k_ref
    assert np.abs(D.cpu().numpy() - D_ref).max() <= 1e-4 * np.abs(D_ref).max()
    assert np.abs(U.cpu().numpy() - U_ref).max() <= 1e-4 * np.abs(U_ref).max()


SOLVES = [
    ("sparse", 120, 240, 0.1, 21),
    ("tridiag", 90, 180, 0.2, 22),
    ("sparse", 300, 150, 0.08, 23),
]


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("gen,n,m,lam,seed", SOLVES)
def test_solve_with_pcd_cg_inner_matches_oracle(request, precision, gen, n, m, lam, seed):
    """Whole ML-cycle solves with PCD-CG as the Newton-direction solver (to
    Section 8's relative precision 1e-4) against the oracle's run of the same
    method.  To rel. KKT 1e-6 the FP64 path takes the oracle's relaxations and
    ends at its objective.  To 1e-10 both paths reach the unique minimiser
    (entries 1e-7, support up to the lambda border, objective 1e-9; the mixed
    path's reported objective 1e-7, its A's objective 1e-9).  The relaxation
    count to 1e-10 is not compared: near the minimiser the inner solver's
    relative stopping rule can leave a coordinate a rounding-sized step past
    its kink, and how many relaxations its removal takes depends on rounding."""
    c = request.getfixturevalue("mctx" if precision == "mixed" else "ctx")
    p = synth.random_problem(n, m, lam, seed, gen=gen)
    S = oracle.form_S(p.X)
    if precision == "fp64":
        A6, _, i6, _ = oracle.solve(S, lam, tol=1e-6, inner="pcd_cg")
        B6, _, g6 = c.solve(S, lam, tol=1e-6, inner="pcd_cg")
        assert g6["status"] == 0 and g6["relaxations"] == i6["relaxations"], (g6, i6)
        assert abs(g6["objective"] - i6["objective"]) <= 1e-9 * abs(i6["objective"])
    A_ref, W_ref, info_ref, _ = oracle.solve(S, lam, tol=1e-10, inner="pcd_cg")
    assert info_ref["status"] == 0
    A, _, info = c.solve(S, lam, tol=1e-10, inner="pcd_cg")
    assert info["status"] == 0, info
    assert info["inner_iters"] > 0 and info["rel_kkt"] <= 1e-10
    assert np.abs(A - A_ref).max() <= 1e-7
    border = np.abs(np.abs(S - W_ref) - lam) <= 1e-7
    assert not np.any(((A != 0) != (A_ref != 0)) & ~border)
    F_ref = info_ref["objective"]
    rtol = 1e-9 if precision == "fp64" else 1e-7
    assert abs(info["objective"] - F_ref) <= rtol * abs(F_ref)
    _, F = oracle.objective(S, A, lam)
    assert abs(F - F_ref) <= 1e-9 * abs(F_ref)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_solve_with_auto_inner_reaches_the_minimiser(request, precision):
    """inner = auto: each relaxation takes CD sweeps or PCD-CG by the length of
    the CD chain (pairs x sweeps against GLASSO_AUTO_PCD_WORK).  n = 400 with
    a small lambda: the coarse levels' small free sets and the level-0 dense
    one.  Whatever the mix, the solve ends at the oracle's unique minimiser
    (entries 1e-7, support up to the lambda border, objective 1e-9 / 1e-7)."""
    c = request.getfixturevalue("mctx" if precision == "mixed" else "ctx")
    p = synth.random_problem(400, 800, 0.04, 31, gen="sparse")
    S = oracle.form_S(p.X)
    A_ref, W_ref, info_ref, _ = oracle.solve(S, p.lam, tol=1e-10)
    assert info_ref["status"] == 0
    A, _, info = c.solve(S, p.lam, tol=1e-10, inner="auto")
    assert info["status"] == 0, info
    assert info["rel_kkt"] <= 1e-10
    assert np.abs(A - A_ref).max() <= 1e-7
    border = np.abs(np.abs(S - W_ref) - p.lam) <= 1e-7
    assert not np.any(((A != 0) != (A_ref != 0)) & ~border)
    F_ref = info_ref["objective"]
    rtol = 1e-9 if precision == "fp64" else 1e-7
    assert abs(info["objective"] - F_ref) <= rtol * abs(F_ref)
