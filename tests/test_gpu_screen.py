"""GPU parity of exact screening: the component labelling of the thresholded
covariance graph (bit-exact against the oracle's breadth-first search) and the
screened solve (isolated vertices in closed form, the rest as one
sub-problem), whose result must be the unscreened oracle's minimiser."""
import numpy as np
import pytest

import oracle
from paper_1607_00315_gb300 import synth

pytestmark = pytest.mark.gpu

MIXED_OBJ_RTOL = 1e-7


@pytest.fixture(scope="module")
def ctx():
    import torch

    from paper_1607_00315_gb300 import build, glasso

    build.build()
    torch.cuda.init()
    c = glasso.Context(0)
    yield c
    c.close()


@pytest.fixture(scope="module")
def mctx():
    import torch

    from paper_1607_00315_gb300 import build, glasso

    build.build()
    torch.cuda.init()
    c = glasso.Context(0, precision=glasso.MIXED)
    yield c
    c.close()


def _label_cases():
    rng = np.random.default_rng(81)
    out = []
    for gen, n, lam in (("sparse", 120, 0.2), ("sparse", 300, 0.1), ("sparse", 500, 0.3),
                        ("tridiag", 257, 0.2), ("tridiag", 100, 0.6)):
        p = synth.random_problem(n, 2 * n, lam, 91, gen=gen)
        out.append((oracle.form_S(p.X), lam))
    S = np.eye(7) * 2.0
    for i, j, v in ((0, 3, 0.5), (3, 5, -0.4), (1, 4, 0.3), (2, 6, 0.05), (0, 6, -0.1)):
        S[i, j] = S[j, i] = v
    out.append((S, 0.2))
    out.append((np.array([[1.5]]), 0.1))
    X = rng.standard_normal((40, 33))
    out.append((X.T @ X / 40, 1e-6))  # complete graph
    # a long path in scrambled vertex order: many links, deep trees
    n = 700
    perm = rng.permutation(n)
    S = np.eye(n)
    for a, b in zip(perm[:-1], perm[1:]):
        S[a, b] = S[b, a] = 0.3
    out.append((S, 0.2))
    p = synth.config_problem(2)  # the n = 2000 workload at its own lambda
    out.append((oracle.form_S(p.X), p.lam))
    return out


def test_components_match_oracle(ctx):
    import torch

    for S, lam in _label_cases():
        ref, kref = oracle.components(S, lam)
        Sd = torch.from_numpy(S).cuda()
        comp = torch.full((S.shape[0],), -7, dtype=torch.int32, device="cuda")
        k = ctx.components(Sd, lam, comp)
        assert k == kref
        assert np.array_equal(comp.cpu().numpy(), ref)


SOLVE_CASES = [
    ("sparse", 120, 0.2, 101),   # mostly isolated vertices, several small blocks
    ("sparse", 150, 0.1, 102),   # a giant component and a few isolated vertices
    ("tridiag", 90, 0.2, 103),   # nothing isolated: the sub-problem is the whole problem
    ("sparse", 60, 0.6, 104),    # everything isolated: no sub-problem
]


@pytest.mark.parametrize("gen,n,lam,seed", SOLVE_CASES)
def test_screened_solve_matches_oracle(ctx, mctx, gen, n, lam, seed):
    """Screening changes the work, not the minimiser: the screened solve
    (both paths) returns the unscreened oracle's A, objective and support,
    and reports the oracle's component count and largest component."""
    p = synth.random_problem(n, 2 * n, lam, seed, gen=gen)
    S = oracle.form_S(p.X)
    comp, k = oracle.components(S, lam)
    sizes = np.bincount(comp, minlength=n)
    A_ref, W_ref, info_ref, _ = oracle.solve(S, lam, tol=1e-11)
    assert info_ref["status"] == 0
    W = np.empty((n, n))
    A, W, info = ctx.solve(S, lam, tol=1e-11, screen=True, W_out=W)
    assert info["status"] == 0, info
    assert abs(info["objective"] - info_ref["objective"]) <= 1e-9 * abs(info_ref["objective"])
    assert np.abs(A - A_ref).max() <= 1e-7
    assert np.abs(W - W_ref).max() <= 1e-7 * max(1.0, np.abs(W_ref).max())
    assert info["components"] == k and info["max_block"] == sizes.max()
    assert info["nnz"] == np.count_nonzero(A)
    assert info["rel_kkt"] <= 1e-11
    Am, _, infom = mctx.solve(S, lam, tol=1e-11, screen=True)
    assert infom["status"] == 0, infom
    assert abs(infom["objective"] - info_ref["objective"]) <= MIXED_OBJ_RTOL * abs(info_ref["objective"])
    assert np.abs(Am - A_ref).max() <= 1e-7
    assert infom["components"] == k


def test_screened_lambda_path_batch(ctx):
    """A warm-started lambda path with screening through the batch entry: each
    solve starts from the previous (screened, assembled) solution and meets
    the oracle bar at its own lambda."""
    from paper_1607_00315_gb300 import glasso

    p = synth.random_problem(100, 200, 0.4, 111, gen="sparse")
    S = oracle.form_S(p.X)
    lams = list(synth.LAMBDA_PATH)
    probs = [glasso.Context.problem(S, lam, 1e-10, screen=True) for lam in lams]
    outs = [np.empty((100, 100)) for _ in lams]
    s, infos = ctx.solve_batch(probs, outs, warm_from_prev=True)
    assert s == 0
    for lam, A, inf in zip(lams, outs, infos):
        A_ref, _, info_ref, _ = oracle.solve(S, lam, tol=1e-10)
        assert abs(inf["objective"] - info_ref["objective"]) <= 1e-9 * abs(info_ref["objective"])
        assert np.abs(A - A_ref).max() <= 1e-7
        assert inf["components"] == oracle.components(S, lam)[1]
