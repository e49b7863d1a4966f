"""GPU parity of the fused batched solver (glasso_solve_batch_fused: every
solve of a batch in one persistent launch, one CTA per lambda path, all
decisions on the device) against the FP64 oracle.

Bar (as for the FP64 solve): relative objective within 1e-9, max entry error
within 1e-7, identical support except pairs whose |(S - W)_ij| lies within
1e-7 of lambda, with both sides at a tight tolerance.  The sizes span several
16-column panels of the factorisation with ragged tails, up to the maximum
n = 512 (one thread per column).
"""
import numpy as np
import pytest

import oracle
from paper_1607_00315_gb300 import synth

pytestmark = pytest.mark.gpu

LAMS = list(synth.LAMBDA_PATH)


@pytest.fixture(scope="module")
def ctx():
    import torch

    from paper_1607_00315_gb300 import build, glasso

    build.build()
    torch.cuda.init()
    c = glasso.Context(0, precision=glasso.MIXED)
    yield c
    c.close()


def _compare(A, A_ref, S, lam, F, F_ref, obj_rtol=1e-9):
    assert abs(F - F_ref) <= obj_rtol * abs(F_ref), (F, F_ref)
    assert np.abs(A - A_ref).max() <= 1e-7, np.abs(A - A_ref).max()
    W = np.linalg.inv(A_ref)
    border = np.abs(np.abs(S - W) - lam) <= 1e-7
    diff = (A != 0) != (A_ref != 0)
    assert not np.any(diff & ~border)


def _paths(ctx, insts, tol, **kw):
    from paper_1607_00315_gb300 import glasso

    probs, outs, meta = [], [], []
    for p in insts:
        S = oracle.form_S(p.X)
        for lam in LAMS:
            probs.append(glasso.Context.problem(S, lam, tol, **kw))
            outs.append(np.empty((p.n, p.n)))
            meta.append((S, lam))
    s, infos = ctx.solve_batch_fused(probs, outs, warm_from_prev=True)
    return s, infos, outs, meta


def test_fused_paths_match_oracle(ctx):
    """Warm-started lambda paths of uneven sizes in one launch; each result is
    the oracle's minimiser, and the relaxation count is the oracle's along the
    same warm-started path (the same steps in the same order, FP64)."""
    shapes = [(7, "sparse"), (33, "tridiag"), (64, "sparse"), (100, "tridiag"), (130, "sparse"),
              (257, "sparse")]
    insts = [synth.random_problem(n, 2 * n, 0.1, 400 + k, gen=g) for k, (n, g) in enumerate(shapes)]
    s, infos, outs, meta = _paths(ctx, insts, 1e-10)
    assert s == 0, [i["status"] for i in infos]
    prev = {}
    for (S, lam), A, inf in zip(meta, outs, infos):
        assert inf["status"] == 0 and inf["rel_kkt"] <= 1e-10, inf
        key = id(S)
        A_ref, _, info_ref, _ = oracle.solve(S, lam, tol=1e-10, A0=prev.get(key))
        assert info_ref["status"] == 0
        prev[key] = A_ref
        _compare(A, A_ref, S, lam, inf["objective"], info_ref["objective"])
        assert abs(inf["relaxations"] - info_ref["relaxations"]) <= 1, (inf, info_ref)
        assert inf["seconds"] > 0.0


def test_fused_full_size_n512(ctx):
    """The largest problem a fused launch takes (n = 512, the batched
    workload's upper end), from samples X on the host."""
    from paper_1607_00315_gb300 import glasso

    p = synth.random_problem(512, 1024, 0.1, 4242, gen="sparse")
    S = oracle.form_S(p.X)
    prob = glasso.Context.problem(p.X, 0.1, 1e-9, samples=True)
    out = np.empty((512, 512))
    s, infos = ctx.solve_batch_fused([prob], [out])
    assert s == 0, infos
    A_ref, _, info_ref, _ = oracle.solve(S, 0.1, tol=1e-10)
    _compare(out, A_ref, S, 0.1, infos[0]["objective"], info_ref["objective"])


def test_fused_degenerate_cases(ctx):
    """n = 1 (closed form 1 / (S + lambda)), lambda above every |S_ij| (a
    diagonal minimiser), and an explicit warm start A0."""
    from paper_1607_00315_gb300 import glasso

    S1 = np.array([[2.5]])
    p1 = synth.random_problem(40, 80, 0.1, 77, gen="sparse")
    S2 = oracle.form_S(p1.X)
    big = float(np.abs(S2 - np.diag(np.diag(S2))).max()) * 1.5
    A0 = oracle.solve(S2, 0.2, tol=1e-10)[0]
    probs = [glasso.Context.problem(S1, 0.3, 1e-12), glasso.Context.problem(S2, big, 1e-12),
             glasso.Context.problem(S2, 0.1, 1e-10, A0=A0)]
    outs = [np.empty((1, 1)), np.empty((40, 40)), np.empty((40, 40))]
    s, infos = ctx.solve_batch_fused(probs, outs)
    assert s == 0, infos
    assert abs(outs[0][0, 0] - 1.0 / 2.8) <= 1e-15
    # the minimiser is diag(1 / (S_ii + lambda)); both solvers may take steps
    # of rounding size from it
    closed = np.diag(1.0 / (np.diag(S2) + big))
    assert np.abs(outs[1] - closed).max() <= 1e-14 * np.abs(closed).max()
    assert np.count_nonzero(outs[1] - np.diag(np.diag(outs[1]))) == 0
    A_big, _, info_big, _ = oracle.solve(S2, big, tol=1e-12)
    _compare(outs[1], A_big, S2, big, infos[1]["objective"], info_big["objective"])
    A_ref, _, info_ref, _ = oracle.solve(S2, 0.1, tol=1e-10, A0=A0)
    _compare(outs[2], A_ref, S2, 0.1, infos[2]["objective"], info_ref["objective"])
    assert abs(infos[2]["relaxations"] - info_ref["relaxations"]) <= 1


def test_fused_same_alone_and_in_the_mix(ctx):
    """A CTA's solve reads nothing of the others: a path gives bit-identical
    results alone and among other paths, wherever the queue places it."""
    insts = [synth.random_problem(n, 2 * n, 0.1, 900 + n, gen="sparse") for n in (90, 200, 35, 150)]
    _, _, outs_mix, _ = _paths(ctx, insts, 1e-6)
    _, _, outs_alone, _ = _paths(ctx, insts[2:3], 1e-6)
    k = 2 * len(LAMS)
    for A, B in zip(outs_mix[k:k + len(LAMS)], outs_alone):
        assert np.array_equal(A, B)


def test_fused_statuses_and_rejections(ctx):
    from paper_1607_00315_gb300 import glasso

    p = synth.random_problem(50, 100, 0.1, 5, gen="sparse")
    S = oracle.form_S(p.X)
    # a cycle bound below what the tolerance needs: GLASSO_EMAXITER, A still a valid iterate
    out = np.empty((50, 50))
    s, infos = ctx.solve_batch_fused([glasso.Context.problem(S, 0.05, 1e-14, max_cycles=1)], [out])
    assert s == glasso.EMAXITER and infos[0]["status"] == glasso.EMAXITER
    assert np.all(np.linalg.eigvalsh(out) > 0)
    # n above the fused bound, screening, PCD-CG: rejected before any work
    big = np.eye(glasso.FUSED_MAX_N + 1)
    for prob, o in [(glasso.Context.problem(big, 0.1), np.empty(big.shape)),
                    (glasso.Context.problem(S, 0.1, screen=True), np.empty((50, 50))),
                    (glasso.Context.problem(S, 0.1, inner="pcd_cg"), np.empty((50, 50)))]:
        s, infos = ctx.solve_batch_fused([prob], [o])
        assert s == glasso.EINVAL and infos[0]["status"] == glasso.EINVAL
    # an initial iterate that is not positive definite
    Sneg = -np.eye(3)
    s, infos = ctx.solve_batch_fused([glasso.Context.problem(Sneg, 0.5)], [np.empty((3, 3))])
    assert s == glasso.ENOTPD


def test_fused_is_one_launch(ctx):
    """The solves run inside one kernel launch (the inputs here are S on the
    host, whose symmetry check takes two small kernels per path)."""
    insts = [synth.random_problem(n, 2 * n, 0.1, 60 + n, gen="tridiag") for n in (48, 96, 120)]
    ctx.set_profiling(True)
    ctx.get_profile(reset=True)  # counts from here on
    s, infos, _, _ = _paths(ctx, insts, 1e-6)
    after = ctx.get_profile()
    ctx.set_profiling(False)
    assert s == 0
    assert after["paths"]["fused"] == len(insts) * len(LAMS)
    assert after["kernels"] == 2 * len(insts) + 1
    # the kernel's own clocks per step: every class ran, and together they
    # cover the solves' device time
    cls = [after[k]["ms"] for k in ("cholesky", "inverse", "scan", "cd_sweeps", "ls_cholesky")]
    assert all(c > 0 for c in cls), cls
    per_solve = sum(i["seconds"] for i in infos) * 1e3
    assert abs(sum(cls) - per_solve) <= 0.05 * per_solve, (sum(cls), per_solve)
