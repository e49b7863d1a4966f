"""Pins of the oracle's BCD-IC (Section 6, Algorithm 2) and ML-BCD: CPU only.

What they rest on, besides the oracle itself:
* eq. logdet_blocks (the Schur complement) against numpy's dense slogdet,
  and eq. Schurs_PDness against numpy's Cholesky;
* a block holding every index is the dense relaxation (Section 6.2: QUIC is
  BCD-IC with a single block): with the Armijo rule the iteration equals the
  composed dense steps (free set, CD sweeps, line search) of the oracle;
* the paper's step rule returns the best of its samples, recomputed here by
  evaluating the dense objective at every sample;
* every block step decreases F, and ML-BCD and BCD-IC alone reach the
  minimiser of the dense ML-cycle (the minimiser is unique).
"""
import numpy as np
import pytest

import oracle
from paper_1607_00315_gb300 import synth


def _spd(n, seed):
    r = np.random.default_rng(seed)
    M = r.standard_normal((n, n))
    return M @ M.T / n + 0.5 * np.eye(n)


def _block_delta(n, I, seed, scale=0.3):
    """A symmetric Delta on the pairs with a row or column in I."""
    r = np.random.default_rng(seed)
    inI = np.zeros(n, dtype=np.uint8)
    inI[I] = 1
    pi, pj, D = [], [], []
    for i in range(n):
        for j in range(i, n):
            if (inI[i] or inI[j]) and r.random() < 0.6:
                pi.append(i)
                pj.append(j)
                D.append(scale * r.standard_normal())
    return inI, np.array(pi), np.array(pj), np.array(D)


def _dense(n, pi, pj, D):
    X = np.zeros((n, n))
    X[pi, pj] = D
    X[pj, pi] = D
    return X


@pytest.mark.parametrize("n,I", [(9, [2, 3, 4]), (12, [0, 11]), (15, list(range(15))), (8, [5])])
def test_schur_logdet_matches_dense(n, I):
    A = _spd(n, n)
    inI, pi, pj, D = _block_delta(n, I, 7 + n)
    Dl = _dense(n, pi, pj, D)
    for alpha in (1.0, 0.5, 0.125, 1e-3):
        sign, ref = np.linalg.slogdet(A + alpha * Dl)
        rc, ld = oracle.bcd_logdet(A, pi, pj, D, inI, alpha)
        if sign > 0 and np.all(np.linalg.eigvalsh(A + alpha * Dl) > 0):
            assert rc == 0 and abs(ld - ref) <= 1e-12 * max(1.0, abs(ref)), (alpha, ld, ref)
        else:
            assert rc == 2


def test_schur_pd_test_and_rejections():
    n = 10
    A = _spd(n, 3)
    inI, pi, pj, D = _block_delta(n, [1, 2, 3], 5, scale=4.0)
    Dl = _dense(n, pi, pj, D)
    seen = set()
    for alpha in (4.0, 2.0, 1.0, 0.5, 0.25, 0.01):
        pd = bool(np.all(np.linalg.eigvalsh(A + alpha * Dl) > 0))
        rc, _ = oracle.bcd_logdet(A, pi, pj, D, inI, alpha)
        assert (rc == 0) == pd and (pd or rc == 2)
        seen.add(pd)
    assert seen == {True, False}  # the scale gives both cases
    # A_22 not positive definite
    B = A.copy()
    B[7, 7] = -1.0
    assert oracle.bcd_logdet(B, pi, pj, D, inI, 0.1)[0] == 1
    # Delta on the 22 block is not a block direction
    bad = oracle.bcd_logdet(A, np.append(pi, 6), np.append(pj, 8), np.append(D, 0.1), inI, 0.1)
    assert bad[0] == -1


def test_whole_index_set_is_the_plain_log_det():
    n = 11
    A = _spd(n, 21)
    inI, pi, pj, D = _block_delta(n, list(range(n)), 22)
    L = oracle.cholesky(A + 0.5 * _dense(n, pi, pj, D))[1]
    rc, ld = oracle.bcd_logdet(A, pi, pj, D, inI, 0.5)
    assert rc == 0 and abs(ld - oracle.logdet_from_chol(L)) <= 1e-14 * abs(ld)


def _problem(n=30, lam=0.1, seed=3):
    p = synth.random_problem(n, 2 * n, lam, seed, gen="sparse")
    return oracle.form_S(p.X), lam


def test_one_block_with_armijo_is_the_dense_relaxation():
    S, lam = _problem()
    n = S.shape[0]
    A = np.diag(1.0 / (np.diag(S) + lam))
    # a few dense relaxations first, so that the step tested is not the first
    for _ in range(2):
        A, _, _, _ = oracle.solve(S, lam, tol=0.0, max_cycles=1, A0=A, one_level=True)
    L = oracle.cholesky(A)[1]
    W = oracle.inverse_from_chol(L)
    F0 = oracle.objective(S, A, lam)[1]
    pi, pj = oracle.free_set(S, W, A, lam)[:2]
    D, _ = oracle.cd_sweeps(S, W, A, lam, pi, pj, 2)
    rc_ref, A_ref, F_ref, _, _ = oracle.line_search(S, W, A, lam, pi, pj, D, F0)
    rc, A_bcd, F_bcd, _, moved = oracle.bcd_iteration(S, A, lam, n, inner="cd", nsweeps=2, rule="armijo")
    assert rc == rc_ref == 0 and moved == 1
    assert np.abs(A_bcd - A_ref).max() <= 1e-13
    assert abs(F_bcd - F_ref) <= 1e-12 * abs(F_ref)


def test_paper_rule_takes_the_best_sample():
    S, lam = _problem(24, 0.15, 9)
    n = S.shape[0]
    A = np.diag(1.0 / (np.diag(S) + lam))
    L = oracle.cholesky(A)[1]
    W = oracle.inverse_from_chol(L)
    pi, pj = oracle.free_set(S, W, A, lam)[:2]
    D, _, _ = oracle.pcd(S, W, A, lam, pi, pj, 500, cg=True, rtol=1e-4)
    Dl = _dense(n, pi, pj, D)
    best, a_best = np.inf, None
    for t in range(30):
        a = 0.5 ** t
        info, F = oracle.objective(S, A + a * Dl, lam)
        if info == 0 and F < best:
            best, a_best = F, a
    rc, A_bcd, F_bcd, trials, _ = oracle.bcd_iteration(S, A, lam, n, inner="pcd_cg", rule="paper")
    assert rc == 0
    assert np.abs(A_bcd - (A + a_best * Dl)).max() <= 1e-13
    assert abs(F_bcd - best) <= 1e-12 * abs(best)
    assert trials == round(-np.log2(a_best)) + 2  # up to the first sample after the best


@pytest.mark.parametrize("block", [1, 5, 13])
def test_block_steps_decrease_F(block):
    S, lam = _problem(26, 0.1, 17)
    A = np.diag(1.0 / (np.diag(S) + lam))
    F = oracle.objective(S, A, lam)[1]
    for _ in range(3):
        rc, A, F_new, _, _ = oracle.bcd_iteration(S, A, lam, block, inner="pcd_cg")
        assert rc == 0 and F_new <= F + 1e-12 * abs(F)
        assert abs(F_new - oracle.objective(S, A, lam)[1]) <= 1e-12 * abs(F_new)
        F = F_new


@pytest.mark.parametrize("block,inner,one_level", [(7, "pcd_cg", False), (10, "cd", False),
                                                   (40, "pcd_cg", False), (9, "pcd_cg", True)])
def test_ml_bcd_reaches_the_minimiser(block, inner, one_level):
    S, lam = _problem(40, 0.1, 11)
    A_ref, _, info_ref, _ = oracle.solve(S, lam, tol=1e-10)
    A, info = oracle.solve_bcd(S, lam, tol=1e-10, block=block, inner=inner, one_level=one_level)
    assert info["status"] == 0 and info["rel_kkt"] <= 1e-10
    assert np.abs(A - A_ref).max() <= 1e-7
    assert abs(info["objective"] - info_ref["objective"]) <= 1e-9 * abs(info_ref["objective"])
    W = np.linalg.inv(A_ref)
    border = np.abs(np.abs(S - W) - lam) <= 1e-7
    assert not np.any(((A != 0) != (A_ref != 0)) & ~border)


def _sparse_spd(n, seed, density=0.15):
    """A positive definite A whose off-diagonal support is a random pattern C."""
    r = np.random.default_rng(seed)
    C = np.triu(r.random((n, n)) < density, 1)
    C = C | C.T
    A = np.where(C, r.uniform(-0.3, 0.3, (n, n)), 0.0)
    A = (A + A.T) / 2
    A[np.arange(n), np.arange(n)] = np.abs(A).sum(1) + 0.5
    return A, C


@pytest.mark.parametrize("n,I,seed", [(20, [3, 4, 5, 6], 1), (30, [0, 29], 2), (25, list(range(10, 22)), 3)])
def test_reduced_inversion_from_the_neighbourhood(n, I, seed):
    """The appendix's W_11 = A_11^{-1}(I - A_12 W_21) from the neighbourhood's
    columns of W alone equals the corresponding block of the dense inverse."""
    A, C = _sparse_spd(n, seed)
    inI = np.zeros(n, dtype=np.uint8)
    inI[I] = 1
    inN = np.zeros(n, dtype=np.uint8)
    for k in range(n):
        if not inI[k] and C[np.array(I), k].any():
            inN[k] = 1
    W = np.linalg.inv(A)
    WN = np.full((n, n), np.nan)  # only the neighbourhood's columns are available
    WN[:, inN.astype(bool)] = W[:, inN.astype(bool)]
    rc, W11 = oracle.bcd_w11(A, inI, inN, WN)
    assert rc == 0
    assert np.abs(W11 - W[np.ix_(I, I)]).max() <= 1e-12 * np.abs(W).max()
    # a support outside C (A_12 nonzero outside N) is refused
    out = next(k for k in range(n) if not inI[k] and not inN[k])
    B = A.copy()
    B[I[0], out] = B[out, I[0]] = 0.01
    assert oracle.bcd_w11(B, inI, inN, WN)[0] == -1


@pytest.mark.parametrize("n,seed,one_level", [(30, 3, False), (45, 8, False), (30, 3, True)])
def test_one_block_ml_bcd_is_the_dense_ml_cycle(n, seed, one_level):
    """With a single block holding every index, CD sweeps and the Armijo rule,
    ML-BCD takes exactly the steps of the dense ML-cycle (Section 6.2's
    equivalence of QUIC with single-block BCD-IC, over whole solves): the same
    cycles, relaxations and trials, and the same iterate bit for bit."""
    S, lam = _problem(n, 0.1, seed)
    A1, _, i1, _ = oracle.solve(S, lam, tol=1e-10, one_level=one_level)
    A2, i2 = oracle.solve_bcd(S, lam, tol=1e-10, block=n, inner="cd", rule="armijo", one_level=one_level)
    assert (i1["cycles"], i1["relaxations"], i1["ls_trials"]) == (i2["cycles"], i2["relaxations"], i2["ls_trials"])
    assert np.array_equal(A1, A2)
