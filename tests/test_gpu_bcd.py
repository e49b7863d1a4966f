"""GPU parity of BCD-IC's Schur-complement line-search log det
(glasso_bcd_logdet; Section 6, eq. logdet_blocks, eq. Schurs_PDness) against
the oracle's orc_bcd_logdet, which the CPU suite pins to numpy's dense
slogdet.  Bar: the same code (positive definite or which block is not) and the
log det within 1e-10 relative; the block sizes cover one index, a block of
several 16-row panels of the factorisations with ragged tails, and every
index.
"""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import torch

    from paper_1607_00315_gb300 import build, glasso

    build.build()
    torch.cuda.init()
    c = glasso.Context(0)
    yield c
    c.close()


def _spd(n, seed):
    r = np.random.default_rng(seed)
    M = r.standard_normal((n, n))
    return M @ M.T / n + 0.5 * np.eye(n)


def _block_delta(n, I, seed, scale):
    r = np.random.default_rng(seed)
    inI = np.zeros(n, dtype=np.uint8)
    inI[I] = 1
    pi, pj, D = [], [], []
    for i in range(n):
        for j in range(i, n):
            if (inI[i] or inI[j]) and r.random() < 0.5:
                pi.append(i)
                pj.append(j)
                D.append(scale * r.standard_normal())
    return inI, np.array(pi, dtype=np.int32), np.array(pj, dtype=np.int32), np.array(D)


def _dev(*arrs):
    import torch

    return [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in arrs]


@pytest.mark.parametrize("n,I,scale", [
    (70, [7], 0.3),
    (60, list(range(5, 23)), 0.3),
    (150, list(range(33)) + [148, 149], 0.2),
    (40, list(range(40)), 0.3),
    (300, list(range(0, 300, 5)), 0.1),
    (50, [1, 2, 3], 4.0),  # large enough to leave the positive-definite set
])
def test_bcd_logdet_matches_oracle(ctx, n, I, scale):
    A = _spd(n, n + len(I))
    inI, pi, pj, D = _block_delta(n, I, 3 * n, scale)
    dA, dpi, dpj, dD, dI = _dev(A, pi, pj, D, inI)
    codes = set()
    for alpha in (4.0, 1.0, 0.5, 0.125, 1e-3):
        code, ld = ctx.bcd_logdet(dA, dpi, dpj, dD, dI, alpha)
        rc, ld_ref = oracle.bcd_logdet(A, pi, pj, D, inI, alpha)
        assert code == rc, (alpha, code, rc)
        if code == 0:
            assert abs(ld - ld_ref) <= 1e-10 * max(1.0, abs(ld_ref)), (alpha, ld, ld_ref)
        codes.add(code)
    if scale > 1.0:
        assert codes == {0, 2}


def test_bcd_logdet_other_codes(ctx):
    from paper_1607_00315_gb300 import glasso

    n = 30
    A = _spd(n, 5)
    inI, pi, pj, D = _block_delta(n, [2, 3, 4], 6, 0.3)
    # A_22 not positive definite
    B = A.copy()
    B[20, 20] = -1.0
    dB, dpi, dpj, dD, dI = _dev(B, pi, pj, D, inI)
    assert ctx.bcd_logdet(dB, dpi, dpj, dD, dI, 0.5)[0] == oracle.bcd_logdet(B, pi, pj, D, inI, 0.5)[0] == 1
    # a nonzero of Delta outside the block's rows and columns
    pi2, pj2, D2 = np.append(pi, 10).astype(np.int32), np.append(pj, 12).astype(np.int32), np.append(D, 0.1)
    dA, dpi2, dpj2, dD2 = _dev(A, pi2, pj2, D2)
    assert ctx.bcd_logdet(dA, dpi2, dpj2, dD2, dI, 0.5)[0] == -1
    # a pair index outside [0, n): refused, the context stays usable
    pi3 = pi.copy()
    pi3[0] = n + 5
    (dpi3,) = _dev(pi3)
    with pytest.raises(glasso.GlassoError):
        ctx.bcd_logdet(dA, dpi3, dpj, dD, dI, 0.5)
    code, ld = ctx.bcd_logdet(dA, dpi, dpj, dD, dI, 0.5)
    assert code == 0 and abs(ld - oracle.bcd_logdet(A, pi, pj, D, inI, 0.5)[1]) <= 1e-10 * abs(ld)


def _problem(n, lam, seed):
    from paper_1607_00315_gb300 import synth

    p = synth.random_problem(n, 2 * n, lam, seed, gen="sparse")
    return oracle.form_S(p.X)


@pytest.mark.parametrize("n,block,nsweeps,rule", [(40, 40, 2, "armijo"), (40, 7, 1, "paper"),
                                                  (130, 33, 2, "paper"), (64, 1, 1, "paper")])
def test_bcd_iteration_matches_oracle(ctx, n, block, nsweeps, rule):
    """Two BCD-IC iterations with CD sweeps, step by step against the oracle's
    orc_bcd_iteration: the same blocks moved, the same samples, the iterate to
    1e-10 (a single block with the Armijo rule is the dense relaxation)."""
    lam = 0.1
    S = _problem(n, lam, 500 + n + block)
    A_ref = np.diag(1.0 / (np.diag(S) + lam))
    dS, dA = _dev(S, A_ref)
    for _ in range(2):
        rc, A_ref, F_ref, tr_ref, mv_ref = oracle.bcd_iteration(S, A_ref, lam, block, inner="cd",
                                                                nsweeps=nsweeps, rule=rule)
        F, mv, tr = ctx.bcd_iteration(dS, dA, lam, block, "cd", nsweeps, rule)
        assert rc == 0
        A = dA.cpu().numpy()
        assert np.abs(A - A_ref).max() <= 1e-10, np.abs(A - A_ref).max()
        assert abs(F - F_ref) <= 1e-10 * abs(F_ref)
        assert (mv, tr) == (mv_ref, tr_ref)


def test_bcd_iterations_with_pcd_cg_reach_the_minimiser(ctx):
    """BCD-IC alone (PCD-CG in each block, the paper's step rule) iterated on
    the device reaches the oracle's minimiser."""
    n, lam = 40, 0.1
    S = _problem(n, lam, 11)
    A_ref = oracle.solve(S, lam, tol=1e-11)[0]
    dS, dA = _dev(S, np.diag(1.0 / (np.diag(S) + lam)))
    F_prev = np.inf
    for _ in range(8):
        F, _, _ = ctx.bcd_iteration(dS, dA, lam, 10, "pcd_cg")
        assert F <= F_prev + 1e-12 * abs(F)
        F_prev = F
    A = dA.cpu().numpy()
    assert np.abs(A - A_ref).max() <= 1e-7
    assert oracle.rel_kkt(S, np.linalg.inv(A), A, lam)[0] <= 1e-8


def test_ml_bcd_matches_oracle(ctx):
    """ML-BCD (the ML-cycle over BCD-IC iterations, PCD-CG in the blocks) on
    the device against the oracle's orc_solve_bcd: the minimiser to the FP64
    bar.  PCD-CG stops at a relative precision, and the device's and the
    oracle's inner solves may stop an iteration apart, so the two trajectories
    differ (measured: 9 relaxations against 11); the count is held to a
    quarter of the oracle's."""
    n, block, lam = 40, 10, 0.1
    S = _problem(n, lam, 700 + n)
    A_ref, info_ref = oracle.solve_bcd(S, lam, tol=1e-10, block=block, inner="pcd_cg")
    assert info_ref["status"] == 0
    (dS,) = _dev(S)
    s, dA, info = ctx.solve_bcd(dS, lam, 1e-10, block, "pcd_cg")
    assert s == 0 and info["status"] == 0 and info["rel_kkt"] <= 1e-10, info
    A = dA.cpu().numpy()
    assert np.abs(A - A_ref).max() <= 1e-7
    assert abs(info["objective"] - info_ref["objective"]) <= 1e-9 * abs(info_ref["objective"])
    assert abs(info["relaxations"] - info_ref["relaxations"]) <= max(2, info_ref["relaxations"] // 4)
