"""Pins of the FP64 oracle against things other than itself.

Each test checks one oracle function against a closed form, a library routine,
brute force on a tiny input, a hand-derived fixture (tests/golden) or an
optimality condition of the paper, chosen so that a dropped term, a wrong sign
or index, or a transposed operand in the oracle fails at least one of them.
"""
import itertools
import json
import os

import numpy as np
import pytest

import oracle
from paper_1607_00315_gb300 import synth

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _spd(n, seed, cond=10.0):
    rng = np.random.default_rng(seed)
    q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    ev = np.exp(rng.uniform(0, np.log(cond), n))
    return (q * ev) @ q.T


def _S(n, m, seed):
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((m, n)) @ np.linalg.cholesky(_spd(n, seed + 1)).T
    return X.T @ X / m


# ---------------------------------------------------------------- generators
def test_sparse_theta_structure():
    rng = np.random.Generator(np.random.PCG64(7))
    n = 57
    t = synth.sparse_theta(n, rng)
    off = t - np.diag(np.diag(t))
    assert np.array_equal(off, off.T)
    assert np.count_nonzero(np.triu(off, 1)) == (5 * n) // 2
    a = np.abs(off[off != 0])
    assert a.min() >= 0.1 and a.max() <= 0.3
    assert np.allclose(np.diag(t), np.abs(off).sum(1) + 0.5)
    assert np.linalg.eigvalsh(t).min() > 0


def test_gaussian_samples_covariance():
    rng = np.random.Generator(np.random.PCG64(3))
    t = synth.tridiag_theta(6)
    X = synth.gaussian_samples(t, 200000, rng)
    emp = X.T @ X / X.shape[0]
    assert np.abs(emp - np.linalg.inv(t)).max() < 0.03


# ---------------------------------------------------------------- a1: S
def test_form_S_matches_library_product():
    rng = np.random.default_rng(0)
    X = rng.standard_normal((37, 11))
    assert np.allclose(oracle.form_S(X), X.T @ X / 37, rtol=0, atol=1e-14)
    # centring: the biased sample covariance (denominator m), eq. cov_estimate
    assert np.allclose(oracle.form_S(X, center=True), np.cov(X, rowvar=False, bias=True),
                       rtol=0, atol=1e-14)


# ---------------------------------------------------------------- a2/a3
@pytest.mark.parametrize("n", [1, 2, 7, 33])
def test_cholesky_logdet_inverse_match_library(n):
    A = _spd(n, n)
    info, L = oracle.cholesky(A)
    assert info == 0
    assert np.allclose(L, np.linalg.cholesky(A), rtol=0, atol=1e-12)
    assert np.allclose(np.triu(L, 1), 0)
    assert abs(oracle.logdet_from_chol(L) - np.linalg.slogdet(A)[1]) < 1e-11
    assert np.allclose(oracle.inverse_from_chol(L), np.linalg.inv(A), rtol=1e-10, atol=1e-12)


def test_cholesky_info_is_first_nonpositive_leading_minor():
    A = _spd(9, 5)
    A[5, 5] -= 50.0  # makes some leading minor from index 5 on non-positive
    info, _ = oracle.cholesky(A)
    # Sylvester: the first k with det(A[:k+1, :k+1]) <= 0 is the failing pivot
    k = next(k for k in range(9) if np.linalg.det(A[: k + 1, : k + 1]) <= 0)
    assert info == k + 1


# ---------------------------------------------------------------- objective
def test_objective_diagonal_closed_form():
    rng = np.random.default_rng(1)
    n = 5
    S = _S(n, 40, 2)
    a = rng.uniform(0.5, 2.0, n)
    lam = 0.3
    info, F = oracle.objective(S, np.diag(a), lam)
    assert info == 0
    expect = np.sum(-np.log(a) + np.diag(S) * a + lam * a)
    assert abs(F - expect) < 1e-12


def test_objective_reports_not_pd():
    info, _ = oracle.objective(np.eye(3), -np.eye(3), 0.1)
    assert info == 1


# ---------------------------------------------------------------- a4 free set
def test_free_set_is_where_a_single_cd_step_moves():
    """Section 5.2: variables outside the free set stay at zero when the Newton
    LASSO is solved over them alone.  At Delta = 0 the 1-D model of pair
    (i, j) is found by brute force (dense numpy model), independently of the
    oracle's CD formula and of the free-set formula."""
    n, lam = 8, 0.15
    S = _S(n, 12, 3)
    rng = np.random.default_rng(4)
    A = np.diag(1.0 / (np.diag(S) + lam))
    A[1, 2] = A[2, 1] = 0.05  # one off-diagonal nonzero
    A += 0.0 * rng.standard_normal((n, n))
    W = np.linalg.inv(A)
    fi, fj = oracle.free_set(S, W, A, lam)
    free = set(zip(fi.tolist(), fj.tolist()))
    G = S - W
    grid = np.linspace(-2, 2, 40001)
    for i in range(n):
        for j in range(i, n):
            E = np.zeros((n, n))
            E[i, j] = E[j, i] = 1.0
            # model(mu) = tr(mu E G) + 1/2 mu^2 tr(E W E W) + lam ||A + mu E||_1
            lin = np.trace(E @ G)
            quad = 0.5 * np.trace(E @ W @ E @ W)
            l1 = np.abs(A[None, :, :] + grid[:, None, None] * E[None]).sum(axis=(1, 2))
            model = lin * grid + quad * grid ** 2 + lam * l1
            mu = grid[np.argmin(model)]
            moves = abs(mu) > 1e-3
            if A[i, j] != 0:
                assert (i, j) in free
            else:
                assert ((i, j) in free) == moves, (i, j, mu)


def test_free_set_restricted_to_candidates_keeps_order():
    n, lam = 6, 0.05
    S = _S(n, 9, 5)
    A = np.diag(1.0 / (np.diag(S) + lam))
    W = np.linalg.inv(A)
    fi, fj = oracle.free_set(S, W, A, lam)
    cand = (fi[::-1].copy(), fj[::-1].copy())
    ci, cj = oracle.free_set(S, W, A, lam, cand=cand)
    assert np.array_equal(ci, cand[0]) and np.array_equal(cj, cand[1])
    assert all(i <= j for i, j in zip(fi, fj))
    # row-major order of the upper triangle
    keys = fi.astype(np.int64) * n + fj
    assert np.all(np.diff(keys) > 0)


# ---------------------------------------------------------------- KKT residual
def test_rel_kkt_hand_derived_fixture():
    g = json.load(open(os.path.join(GOLD, "kkt_2x2.json")))
    r, mx = oracle.rel_kkt(np.array(g["S"]), np.array(g["W"]), np.array(g["A"]), g["lambda"])
    assert abs(r - g["rel_kkt"]) < 1e-15 and abs(mx - g["max_kkt"]) < 1e-15


# ---------------------------------------------------------------- a5 hierarchy
def test_hierarchy_hand_derived_sizes():
    g = json.load(open(os.path.join(GOLD, "hierarchy_sizes.json")))
    rng = np.random.default_rng(6)
    for case in g["cases"]:
        nf, ns = case["nf"], case["ns"]
        insupp = np.zeros(nf, dtype=np.uint8)
        insupp[rng.choice(nf, ns, replace=False)] = 1
        absg = rng.uniform(0, 1, nf)
        tag, L = oracle.hierarchy(absg, insupp)
        assert L == case["L"]
        counts = {str(t): int((tag == t).sum()) for t in np.unique(tag)}
        assert counts == case["count_by_tag"]


def test_hierarchy_ranking_matches_library_sort_with_ties():
    rng = np.random.default_rng(8)
    nf = 301
    insupp = (rng.random(nf) < 0.2).astype(np.uint8)
    absg = rng.integers(0, 25, nf).astype(np.float64) / 7.0  # many exact ties
    tag, L = oracle.hierarchy(absg, insupp)
    ns = int(insupp.sum())
    # independent ranking: numpy lexsort by (-|G|, position)
    idx = np.flatnonzero(insupp == 0)
    order = idx[np.lexsort((idx, -absg[idx]))]
    sizes = [None, max((nf + 1) // 2, ns)]
    while sizes[-1] > ns:
        sizes.append(max((sizes[-1] + 1) // 2, ns))
    assert L == len(sizes) - 1
    assert np.all(tag[insupp == 1] == L)
    for l in range(1, L + 1):
        in_l = set(np.flatnonzero(insupp).tolist()) | set(order[: sizes[l] - ns].tolist())
        assert in_l == set(np.flatnonzero(tag >= l).tolist())
        assert len(in_l) == sizes[l]


# ---------------------------------------------------------------- a6 CD sweeps
def _model(G, W, A, D, lam):
    """Newton LASSO objective of eq. Quad_MLE_l1_prior without f(A)."""
    return np.trace(D @ G) + 0.5 * np.trace(D @ W @ D @ W) + lam * np.abs(A + D).sum()


def _dense(n, pi, pj, d):
    D = np.zeros((n, n))
    D[pi, pj] = d
    D[pj, pi] = d
    return D


def test_cd_single_coordinate_is_exact_1d_minimiser():
    n, lam = 7, 0.1
    S = _S(n, 10, 9)
    A = np.diag(1.0 / (np.diag(S) + lam))
    A[0, 3] = A[3, 0] = -0.02
    W = np.linalg.inv(A)
    G = S - W
    rng = np.random.default_rng(10)
    pairs = [(0, 3), (1, 1), (2, 5), (4, 6)]
    # start from a nonzero Delta so that b includes (W Delta W)_ij
    pi0 = np.array([p[0] for p in pairs], dtype=np.int32)
    pj0 = np.array([p[1] for p in pairs], dtype=np.int32)
    d0 = rng.uniform(-0.05, 0.05, len(pairs))
    U0 = _dense(n, pi0, pj0, d0) @ W
    for k, (i, j) in enumerate(pairs):
        d, U = oracle.cd_sweeps(S, W, A, lam, pi0[k:k + 1], pj0[k:k + 1], 1, D=d0[k:k + 1], U=U0)
        D_before = _dense(n, pi0, pj0, d0)
        E = np.zeros((n, n))
        E[i, j] = E[j, i] = 1.0
        grid = d0[k] + np.linspace(-1, 1, 200001)
        vals = [_model(G, W, A, D_before + (g - d0[k]) * E, lam) for g in grid[::100]]
        g0 = grid[::100][int(np.argmin(vals))]
        fine = g0 + np.linspace(-1e-3, 1e-3, 2001)
        vals = [_model(G, W, A, D_before + (g - d0[k]) * E, lam) for g in fine]
        best = fine[int(np.argmin(vals))]
        assert abs(d[0] - best) < 2e-6, (i, j, d[0], best)
        # U stays Delta W (library matmul)
        Dn = D_before + (d[0] - d0[k]) * E
        assert np.allclose(U, Dn @ W, atol=1e-13)


def test_cd_sweeps_converge_to_lasso_kkt():
    """Many sweeps solve the restricted Newton LASSO: its subgradient
    (G + W Delta W + lambda sign) vanishes on the pair list."""
    n, lam = 12, 0.08
    S = _S(n, 30, 11)
    A = np.diag(1.0 / (np.diag(S) + lam))
    W = np.linalg.inv(A)
    fi, fj = oracle.free_set(S, W, A, lam)
    d, U = oracle.cd_sweeps(S, W, A, lam, fi, fj, 400)
    D = _dense(n, fi, fj, d)
    assert np.allclose(U, D @ W, atol=1e-12)
    R = (S - W) + W @ D @ W
    T = A + D
    for i, j in zip(fi, fj):
        if T[i, j] != 0:
            assert abs(R[i, j] + lam * np.sign(T[i, j])) < 1e-9
        else:
            assert abs(R[i, j]) <= lam + 1e-9


def test_cd_decreases_model():
    n, lam = 10, 0.1
    S = _S(n, 15, 12)
    A = np.diag(1.0 / (np.diag(S) + lam))
    W = np.linalg.inv(A)
    fi, fj = oracle.free_set(S, W, A, lam)
    prev = _model(S - W, W, A, np.zeros((n, n)), lam)
    d = None
    U = None
    for _ in range(5):
        d, U = oracle.cd_sweeps(S, W, A, lam, fi, fj, 1, D=d, U=U)
        cur = _model(S - W, W, A, _dense(n, fi, fj, d), lam)
        assert cur <= prev + 1e-14
        prev = cur


# ---------------------------------------------------------------- a7 line search
def test_line_search_first_armijo_alpha():
    n, lam = 9, 0.05
    S = _S(n, 20, 13)
    A = np.diag(1.0 / (np.diag(S) + lam))
    W = np.linalg.inv(A)
    fi, fj = oracle.free_set(S, W, A, lam)
    d, _ = oracle.cd_sweeps(S, W, A, lam, fi, fj, 3)
    d = d * 40.0  # an overlong step forces backtracking
    _, F0 = oracle.objective(S, A, lam)
    rc, A1, F1, alpha, trials = oracle.line_search(S, W, A, lam, fi, fj, d, F0)
    assert rc == 0 and trials > 1
    D = _dense(n, fi, fj, d)
    delta = np.sum((S - W) * D) + lam * (np.abs(A + D).sum() - np.abs(A).sum())

    def F(M):
        s, ld = np.linalg.slogdet(M)
        if s <= 0 or np.linalg.eigvalsh(M).min() <= 0:
            return None
        return -ld + np.sum(S * M) + lam * np.abs(M).sum()

    epsF = 1e-12 * max(abs(F0), n)  # the rounding allowance of the acceptance test
    for t in range(trials):
        a = 0.5 ** t
        val = F(A + a * D)
        ok = val is not None and val <= F0 + 1e-4 * a * delta + epsF
        assert ok == (t == trials - 1)
    assert abs(alpha - 0.5 ** (trials - 1)) == 0
    assert np.allclose(A1, A + alpha * D, atol=1e-15)
    assert abs(F1 - F(A1)) < 1e-10


# ---------------------------------------------------------------- a8 solve
def _kkt_ok(S, A, lam, tol):
    W = np.linalg.inv(A)
    G = S - W
    on = A != 0
    assert np.abs(G[on] + lam * np.sign(A[on])).max() < tol
    if (~on).any():
        assert np.abs(G[~on]).max() <= lam + tol
    assert np.allclose(np.diag(W), np.diag(S) + lam, atol=tol)


def test_solve_diagonal_S_closed_form():
    d = np.array([0.5, 1.0, 2.0, 3.5])
    lam = 0.2
    A, W, info, _ = oracle.solve(np.diag(d), lam, tol=1e-12)
    assert info["status"] == 0
    assert np.allclose(A, np.diag(1.0 / (d + lam)), atol=1e-14)


def test_solve_large_lambda_gives_diagonal():
    S = _S(8, 20, 14)
    lam = np.abs(S - np.diag(np.diag(S))).max() + 1e-3
    A, W, info, _ = oracle.solve(S, lam, tol=1e-12)
    assert np.count_nonzero(A - np.diag(np.diag(A))) == 0
    assert np.allclose(np.diag(A), 1.0 / (np.diag(S) + lam), atol=1e-13)


@pytest.mark.parametrize("s12", [0.7, -0.45, 0.05])
def test_solve_n2_closed_form(s12):
    S = np.array([[1.3, s12], [s12, 0.8]])
    lam = 0.1
    A, _, info, _ = oracle.solve(S, lam, tol=1e-13)
    Wx = np.array([[1.3 + lam, np.sign(s12) * max(abs(s12) - lam, 0.0)],
                   [0.0, 0.8 + lam]])
    Wx[1, 0] = Wx[0, 1]
    assert np.allclose(A, np.linalg.inv(Wx), atol=1e-11)


def _brute_force(S, lam):
    """Enumerate the sign patterns of the off-diagonal entries; for each, solve
    the smooth restricted problem (fixed support, fixed signs) by Newton's
    method and keep the patterns whose solution satisfies the optimality
    conditions of eq. subgradient1.  Independent of the oracle's method."""
    n = S.shape[0]
    offs = [(i, j) for i in range(n) for j in range(i + 1, n)]
    sols = []
    for pat in itertools.product((-1, 0, 1), repeat=len(offs)):
        act = [(i, i, 0) for i in range(n)] + [(i, j, s) for (i, j), s in zip(offs, pat) if s != 0]
        Es = []
        for i, j, _ in act:
            E = np.zeros((n, n))
            E[i, j] = E[j, i] = 1.0
            Es.append(E)
        lin = np.array([np.sum((S + lam * (np.eye(n) if i == j else s * (1 - np.eye(n)))) * E)
                        for (i, j, s), E in zip(act, Es)])

        def fval(x):
            M = sum(xk * E for xk, E in zip(x, Es))
            if np.linalg.eigvalsh(M).min() <= 0:
                return np.inf
            return -np.linalg.slogdet(M)[1] + lin @ x

        x = np.array([1.0 / (S[i, i] + lam) if i == j else 0.0 for i, j, _ in act])
        ok = False
        for _ in range(200):
            M = sum(xk * E for xk, E in zip(x, Es))
            Wm = np.linalg.inv(M)
            g = lin - np.array([np.sum(Wm * E) for E in Es])
            H = np.array([[np.trace(Wm @ Ep @ Wm @ Eq) for Eq in Es] for Ep in Es])
            step = np.linalg.solve(H, -g)
            dec = -g @ step
            if dec < 1e-26:
                ok = True
                break
            t, f0 = 1.0, fval(x)
            while fval(x + t * step) > f0 - 0.25 * t * dec and t > 1e-12:
                t *= 0.5
            x = x + t * step
            if np.abs(x).max() > 1e8:
                break
        if not ok:
            continue
        M = sum(xk * E for xk, E in zip(x, Es))
        Wm = np.linalg.inv(M)
        G = S - Wm
        good = True
        for (i, j), s in zip(offs, pat):
            if s == 0:
                good &= abs(G[i, j]) <= lam + 1e-10
            else:
                good &= M[i, j] * s > -1e-12
        if good:
            sols.append(M)
    return sols


@pytest.mark.parametrize("n,seed", [(2, 21), (3, 22), (3, 23), (4, 24)])
def test_solve_matches_brute_force(n, seed):
    S = _S(n, 2 * n, seed)
    off = np.abs(S - np.diag(np.diag(S)))
    # some entries in, some out; kept off any |S_ij| so that no pair sits
    # exactly on the free-set boundary |G_ij| = lambda at the optimum
    lam = 0.97 * float(np.median(off[off > 0]))
    sols = _brute_force(S, lam)
    assert sols, "brute force found no optimum"
    A, _, info, _ = oracle.solve(S, lam, tol=1e-12)
    assert info["status"] == 0
    for M in sols:  # all surviving patterns describe the same (unique) optimum
        assert np.allclose(A, M, atol=1e-9), (A, M)


@pytest.mark.parametrize("cfg_seed", [31, 32])
def test_solve_kkt_and_duality_gap(cfg_seed):
    p = synth.random_problem(40, 60, 0.12, cfg_seed, gen="sparse")
    S = oracle.form_S(p.X)
    A, W, info, _ = oracle.solve(S, p.lam, tol=1e-11)
    assert info["status"] == 0 and info["rel_kkt"] <= 1e-11
    _kkt_ok(S, A, p.lam, 1e-8)
    # duality certificate: W~ = S + clip(A^{-1} - S, -lam, lam) is dual feasible
    Wi = np.linalg.inv(A)
    Wt = S + np.clip(Wi - S, -p.lam, p.lam)
    primal = -np.linalg.slogdet(A)[1] + np.sum(S * A) + p.lam * np.abs(A).sum()
    dual = np.linalg.slogdet(Wt)[1] + S.shape[0]
    assert primal - dual >= -1e-12
    assert primal - dual < 1e-8
    assert abs(primal - info["objective"]) < 1e-9


def test_solve_monotone_per_relaxation():
    p = synth.config_problem(1)
    S = oracle.form_S(p.X)
    A, W, info, tr = oracle.solve(S, p.lam, tol=1e-8, trace_cap=500)
    assert info["status"] == 0
    F = tr[:, 0]
    # monotone up to the line search's rounding allowance 1e-12 max(|F|, n)
    assert np.all(np.diff(F) <= 1e-12 * max(abs(F).max(), S.shape[0]))
    assert set(tr[:, 1].astype(int).tolist()) >= {0, 1}


def test_solve_scaling_and_permutation_equivariance():
    p = synth.random_problem(25, 40, 0.15, 41, gen="sparse")
    S = oracle.form_S(p.X)
    A, *_ = oracle.solve(S, p.lam, tol=1e-12)
    c = 3.0
    A2, *_ = oracle.solve(c * S, c * p.lam, tol=1e-12)
    assert np.allclose(A2, A / c, atol=1e-9)
    perm = np.random.default_rng(42).permutation(25)
    A3, *_ = oracle.solve(S[np.ix_(perm, perm)], p.lam, tol=1e-12)
    assert np.allclose(A3, A[np.ix_(perm, perm)], atol=1e-9)


def test_solve_block_separability():
    S1 = _S(6, 12, 51)
    S2 = _S(5, 10, 52)
    lam = 0.1
    S = np.zeros((11, 11))
    S[:6, :6] = S1
    S[6:, 6:] = S2
    S[0, 8] = S[8, 0] = 0.05  # below lambda: blocks stay separate
    A, *_ = oracle.solve(S, lam, tol=1e-12)
    A1, *_ = oracle.solve(S1, lam, tol=1e-12)
    A2, *_ = oracle.solve(S2, lam, tol=1e-12)
    assert np.count_nonzero(A[:6, 6:]) == 0
    assert np.allclose(A[:6, :6], A1, atol=1e-9) and np.allclose(A[6:, 6:], A2, atol=1e-9)


def test_warm_start_at_optimum_stops_immediately():
    """Algorithm 1 maps x^(k) to x^(k+1); at the optimum the finest-level check
    stops the solve without moving A (resume from a saved iterate)."""
    p = synth.random_problem(20, 30, 0.15, 61, gen="tridiag")
    S = oracle.form_S(p.X)
    A, *_ = oracle.solve(S, p.lam, tol=1e-12)
    A2, _, info, _ = oracle.solve(S, p.lam, tol=1e-9, A0=A)
    assert info["status"] == 0 and info["cycles"] == 1
    assert np.allclose(A2, A, atol=1e-12)


@pytest.mark.parametrize("gen,n,lam,seed", [("sparse", 60, 0.1, 41), ("tridiag", 90, 0.15, 42)])
def test_one_level_reaches_the_same_minimiser(gen, n, lam, seed):
    """The one-level method (the paper's Section 8 comparison: every cycle a
    single relaxation on the full free set) and the ML-cycle minimise the
    same strictly convex objective, whose minimiser is unique: the two
    oracle runs must agree, the one-level run must make exactly one
    relaxation per cycle, and max-supp bounds the final support."""
    p = synth.random_problem(n, 2 * n, lam, seed, gen=gen)
    S = oracle.form_S(p.X)
    A_ml, _, i_ml, _ = oracle.solve(S, lam, tol=1e-11)
    A_1, _, i_1, tr = oracle.solve(S, lam, tol=1e-11, one_level=True, trace_cap=200)
    assert i_ml["status"] == 0 and i_1["status"] == 0
    assert np.abs(A_1 - A_ml).max() <= 1e-7
    assert abs(i_1["objective"] - i_ml["objective"]) <= 1e-10 * abs(i_ml["objective"])
    assert i_1["relaxations"] in (i_1["cycles"], i_1["cycles"] - 1)
    assert np.all(tr[:, 1] == 0)  # every relaxation on the finest level
    for info in (i_ml, i_1):
        assert info["max_nnz"] >= info["nnz"] == np.count_nonzero(A_ml)



def test_continuation_lambdas_hand_derived():
    """Section 8's continuation values: lambda_4 halfway between lambda and the
    largest off-diagonal |S_ij| (the smallest lambda with a diagonal minimiser;
    1 on normalised data, where the paper's lambda_4 = (1 + lambda) / 2), then
    lambda_3, lambda_2 evenly spaced down to lambda.  Hand values: the largest
    off-diagonal entry is -0.7 (the diagonal, larger still, does not count),
    so lambda = 0.1 gives 0.4, 0.3, 0.2."""
    S = np.array([[3.0, 0.2, -0.7], [0.2, 2.0, 0.5], [-0.7, 0.5, 4.0]])
    np.testing.assert_allclose(oracle.continuation_lambdas(S, 0.1), [0.4, 0.3, 0.2], rtol=1e-15)
    # no stages once the solution at lambda is diagonal
    assert oracle.continuation_lambdas(S, 0.7).size == 0
    assert oracle.continuation_lambdas(np.diag([1.0, 2.0]), 0.05).size == 0
    # normalised data: never above the paper's (1 + lambda) / 2
    X = np.random.default_rng(3).standard_normal((40, 12))
    Sn = np.corrcoef(X, rowvar=False)
    lam = 0.05
    l4 = oracle.continuation_lambdas(Sn, lam)[0]
    assert lam < l4 <= 0.5 * (1.0 + lam)


def test_continuation_is_one_relaxation_per_stage():
    """The continuation stages are one level-0 relaxation at each lambda_s in
    decreasing order, each from the previous iterate: with no cycles at the
    target lambda the solve must return exactly what three single-relaxation
    one-level solves at lambda_4, lambda_3, lambda_2 chained from A0 return,
    and each stage's recorded objective is F(A_s) at its own lambda_s
    (library slogdet)."""
    p = synth.random_problem(50, 100, 0.1, 51, gen="sparse")
    S = oracle.form_S(p.X)
    lams = oracle.continuation_lambdas(S, p.lam)
    assert lams.size == 3 and np.all(np.diff(lams) < 0) and lams[-1] > p.lam
    A0 = np.diag(1.0 / (np.diag(S) + p.lam))
    A_c, _, info, tr = oracle.solve(S, p.lam, tol=0.0, max_cycles=0, A0=A0, continuation=True,
                                    trace_cap=10)
    assert info["cycles"] == 0 and info["relaxations"] == 3 and tr.shape[0] == 3
    A = A0
    for s, ls in enumerate(lams):
        A, _, inf1, _ = oracle.solve(S, ls, tol=0.0, max_cycles=1, A0=A, one_level=True)
        assert inf1["relaxations"] == 1
        sign, ld = np.linalg.slogdet(A)
        assert sign > 0
        F = -ld + np.sum(S * A) + ls * np.abs(A).sum()
        assert abs(tr[s, 0] - F) <= 1e-11 * abs(F) and tr[s, 1] == 0
    assert np.array_equal(A_c, A)


@pytest.mark.parametrize("one_level", [False, True])
def test_continuation_reaches_the_same_minimiser(one_level):
    """Continuation changes the path, not the minimiser (the objective at the
    target lambda is strictly convex): with the ML-cycle or the one-level
    method after the stages, the result is the ML-cycle's; the three stage
    relaxations come first, on the finest level."""
    p = synth.random_problem(60, 120, 0.1, 41, gen="sparse")
    S = oracle.form_S(p.X)
    A_ml, _, i_ml, _ = oracle.solve(S, p.lam, tol=1e-11)
    A_c, _, i_c, tr = oracle.solve(S, p.lam, tol=1e-11, one_level=one_level, continuation=True,
                                   trace_cap=200)
    assert i_c["status"] == 0
    assert np.abs(A_c - A_ml).max() <= 1e-7
    assert abs(i_c["objective"] - i_ml["objective"]) <= 1e-10 * abs(i_ml["objective"])
    assert np.all(tr[:3, 1] == 0)
    if one_level:
        assert i_c["relaxations"] in (3 + i_c["cycles"], 3 + i_c["cycles"] - 1)
    assert i_c["max_nnz"] >= i_c["nnz"] == np.count_nonzero(A_ml)


def _library_components(S, lam):
    """Component labels by scipy's graph routine, renamed to each component's
    smallest vertex."""
    from scipy.sparse import csr_matrix
    from scipy.sparse.csgraph import connected_components

    G = np.abs(np.triu(S, 1)) > lam
    k, lab = connected_components(csr_matrix(G | G.T), directed=False)
    first = {}
    for i, c in enumerate(lab):
        first.setdefault(c, i)
    return np.array([first[c] for c in lab], dtype=np.int32), k


def _screen_cases():
    rng = np.random.default_rng(61)
    out = []
    for gen, n, lam in (("sparse", 120, 0.2), ("sparse", 120, 0.1), ("sparse", 200, 0.3),
                        ("tridiag", 80, 0.2), ("tridiag", 80, 0.6)):
        p = synth.random_problem(n, 2 * n, lam, 71, gen=gen)
        out.append((oracle.form_S(p.X), lam))
    # hand-built blocks {0, 3, 5}, {1, 4}, {2}, {6} under a permutation-free layout
    S = np.eye(7) * 2.0
    for i, j, v in ((0, 3, 0.5), (3, 5, -0.4), (1, 4, 0.3), (2, 6, 0.05), (0, 6, -0.1)):
        S[i, j] = S[j, i] = v
    out.append((S, 0.2))
    out.append((np.array([[1.5]]), 0.1))
    X = rng.standard_normal((30, 25))
    out.append((X.T @ X / 30, 1e-6))  # every pair an edge: one component
    return out


def test_components_match_library():
    """Component labels (smallest vertex of each component) equal scipy's
    connected components of the thresholded graph; the hand-built case has
    components {0, 3, 5}, {1, 4}, {2}, {6} (0.05 and -0.1 are below lambda)."""
    for S, lam in _screen_cases():
        comp, k = oracle.components(S, lam)
        ref, kr = _library_components(S, lam)
        assert k == kr and np.array_equal(comp, ref)
    S, lam = _screen_cases()[5]
    comp, k = oracle.components(S, lam)
    assert k == 4 and comp.tolist() == [0, 1, 2, 0, 1, 0, 6]


def test_screening_theorem_blocks_solve_separately():
    """The minimiser is block diagonal over the components, each block the
    minimiser on its own sub-matrix, an isolated vertex 1/(S_ii + lambda); and
    solving all non-isolated vertices as one sub-problem (the GPU's screened
    solve) gives the same matrix."""
    p = synth.random_problem(90, 180, 0.2, 72, gen="sparse")
    S = oracle.form_S(p.X)
    lam = p.lam
    comp, k = oracle.components(S, lam)
    sizes = np.bincount(comp, minlength=S.shape[0])
    assert 3 <= k < S.shape[0] and (sizes >= 2).sum() >= 2  # several non-trivial blocks
    A_full, _, info, _ = oracle.solve(S, lam, tol=1e-12)
    assert info["status"] == 0
    A_blk = np.zeros_like(S)
    for r in np.unique(comp):
        idx = np.flatnonzero(comp == r)
        if idx.size == 1:
            A_blk[idx[0], idx[0]] = 1.0 / (S[idx[0], idx[0]] + lam)
        else:
            Ab, *_ = oracle.solve(S[np.ix_(idx, idx)], lam, tol=1e-12)
            A_blk[np.ix_(idx, idx)] = Ab
    assert np.abs(A_blk - A_full).max() <= 1e-8
    iso = sizes[comp] == 1
    idx = np.flatnonzero(~iso)
    A_uni = np.diag(np.where(iso, 1.0 / (np.diag(S) + lam), 0.0))
    Au, *_ = oracle.solve(S[np.ix_(idx, idx)], lam, tol=1e-12)
    A_uni[np.ix_(idx, idx)] = Au
    assert np.abs(A_uni - A_full).max() <= 1e-8


def _coupled_lasso(n=14, lam=0.06, seed=11):
    """A Newton LASSO whose Hessian couples the coordinates: the iterate after
    one ML-cycle (off-diagonal support), its inverse and its free set."""
    S = _S(n, 30, seed)
    A, *_ = oracle.solve(S, lam, tol=1e-2, max_cycles=1)
    assert np.count_nonzero(A - np.diag(np.diag(A))) > 0
    W = np.linalg.inv(A)
    fi, fj = oracle.free_set(S, W, A, lam)
    return S, A, W, fi, fj, lam


def test_pcd_direction_is_each_coordinates_1d_minimiser():
    """Section 2's PCD direction (eq. IST_direction with the Hessian's
    diagonal): each component is that coordinate's own exact minimiser of the
    dense Newton LASSO model (library matmul) with every other coordinate
    held, at a Delta that is not zero."""
    from scipy.optimize import minimize_scalar

    S, A, W, fi, fj, lam = _coupled_lasso()
    n = A.shape[0]
    D0, U0 = oracle.cd_sweeps(S, W, A, lam, fi, fj, 1)
    d, _ = oracle.pcd_direction(S, W, A, lam, fi, fj, D0, U0)
    G = S - W
    base = _dense(n, fi, fj, D0)
    for p in range(len(fi)):
        E = _dense(n, [fi[p]], [fj[p]], [1.0])
        f = lambda mu: _model(G, W, A, base + mu * E, lam)  # noqa: E731
        r = minimize_scalar(f, bounds=(d[p] - 1.0, d[p] + 1.0), method="bounded",
                            options={"xatol": 1e-12})
        assert f(d[p]) <= f(r.x) + 1e-13
        assert abs(r.x - d[p]) <= 1e-6


def test_pcd_step_is_the_exact_minimiser_along_the_direction():
    """One PCD iteration moves Delta by t d with t the exact minimiser of the
    dense model along d (library matmul, bounded scalar search and a grid)."""
    from scipy.optimize import minimize_scalar

    S, A, W, fi, fj, lam = _coupled_lasso()
    n = A.shape[0]
    D0, U0 = oracle.cd_sweeps(S, W, A, lam, fi, fj, 1)
    d, _ = oracle.pcd_direction(S, W, A, lam, fi, fj, D0, U0)
    D1, U1, k = oracle.pcd(S, W, A, lam, fi, fj, 1, cg=False, D=D0, U=U0)
    assert k == 1
    G = S - W
    step = D1 - D0
    t = step[np.argmax(np.abs(d))] / d[np.argmax(np.abs(d))]
    assert t > 0
    # every coordinate moved by the same multiple of d (or landed on an exact zero)
    T1 = A[fi, fj] + D1
    ok = np.isclose(step, t * d, rtol=1e-9, atol=1e-15) | (T1 == 0.0)
    assert ok.all()
    f = lambda s: _model(G, W, A, _dense(n, fi, fj, D0 + s * d), lam)  # noqa: E731
    r = minimize_scalar(f, bounds=(0.0, 4.0 * t), method="bounded", options={"xatol": 1e-13})
    assert f(t) <= f(r.x) + 1e-13
    assert all(f(t) <= f(s) + 1e-13 for s in np.linspace(0.0, 3.0 * t, 301))
    assert np.allclose(U1, _dense(n, fi, fj, D1) @ W, atol=1e-13)


@pytest.mark.parametrize("cg", [False, True])
def test_pcd_decreases_the_model_and_solves_the_lasso(cg):
    """PCD and PCD-CG decrease the model at every iteration and reach the
    restricted Newton LASSO's KKT point, the same minimiser the CD sweeps
    reach; U stays Delta W (library matmul)."""
    S, A, W, fi, fj, lam = _coupled_lasso()
    n = A.shape[0]
    G = S - W
    prev = _model(G, W, A, np.zeros((n, n)), lam)
    for k in range(1, 16):
        Dk, _, _ = oracle.pcd(S, W, A, lam, fi, fj, k, cg=cg)
        cur = _model(G, W, A, _dense(n, fi, fj, Dk), lam)
        assert cur <= prev + 1e-13
        prev = cur
    D, U, _ = oracle.pcd(S, W, A, lam, fi, fj, 2000, cg=cg)
    Dm = _dense(n, fi, fj, D)
    assert np.allclose(U, Dm @ W, atol=1e-12)
    R = G + W @ Dm @ W
    T = A + Dm
    for i, j in zip(fi, fj):
        if T[i, j] != 0:
            assert abs(R[i, j] + lam * np.sign(T[i, j])) < 1e-9
        else:
            assert abs(R[i, j]) <= lam + 1e-9
    Dc, _ = oracle.cd_sweeps(S, W, A, lam, fi, fj, 2000)
    assert np.abs(D - Dc).max() <= 1e-10
    # the minimiser's zeros are exact (kinks and the zero snap), as CD's are
    assert np.array_equal(A[fi, fj] + D == 0, A[fi, fj] + Dc == 0)


def test_pcd_cg_needs_fewer_iterations_than_pcd():
    """The conjugate-gradient acceleration (Section 6.3's PCD-CG) brings the
    PCD direction below 1e-10 in fewer iterations than plain PCD on a coupled
    problem."""
    S, A, W, fi, fj, lam = _coupled_lasso()

    def below(D, U, tol):
        d, _ = oracle.pcd_direction(S, W, A, lam, fi, fj, D, U)
        return np.abs(d).max() <= tol

    # plain PCD keeps no state between iterations: continue one at a time
    D, U, k_pcd = None, None, 0
    while k_pcd < 3000:
        D, U, _ = oracle.pcd(S, W, A, lam, fi, fj, 1, cg=False, D=D, U=U)
        k_pcd += 1
        if below(D, U, 1e-10):
            break
    # PCD-CG carries its previous direction: rerun from the start
    k_cg = next(k for k in range(1, 3001)
                if below(*oracle.pcd(S, W, A, lam, fi, fj, k, cg=True)[:2], 1e-10))
    assert k_cg < k_pcd < 3000


def test_pcd_final_shrinkage_at_the_precision_stop():
    """The stop at relative precision ends with the final shrinkage: the
    coordinates whose own 1-D minimiser is zero at the last direction take
    their exact zero.  Against the same iterations without it (the iteration
    cap instead of the precision stop): only such coordinates change, each to
    exactly -A_p, each by less than the stopping precision, U stays Delta W,
    and the model of eq. Quad_MLE_l1_prior does not increase (each change is
    that coordinate's own minimiser, and the changes are below the precision)."""
    S, A, W, fi, fj, lam = _coupled_lasso()
    n = A.shape[0]
    G = S - W
    rtol = 1e-2
    D1, U1, k = oracle.pcd(S, W, A, lam, fi, fj, 500, cg=True, rtol=rtol)
    D0, U0, k0 = oracle.pcd(S, W, A, lam, fi, fj, k, cg=True)
    assert k0 == k and 1 <= k < 500
    d, _ = oracle.pcd_direction(S, W, A, lam, fi, fj, D0, U0)
    c = A[fi, fj] + D0
    own_zero = (c != 0) & (c + d == 0)
    changed = D1 != D0
    assert changed.any()
    assert np.array_equal(changed, own_zero)
    assert np.all(D1[changed] == -A[fi, fj][changed])
    d_first, _ = oracle.pcd_direction(S, W, A, lam, fi, fj)
    assert np.all(np.abs(D1 - D0) <= rtol * np.abs(d_first).max())
    assert np.allclose(U1, _dense(n, fi, fj, D1) @ W, atol=1e-12)
    m1 = _model(G, W, A, _dense(n, fi, fj, D1), lam)
    m0 = _model(G, W, A, _dense(n, fi, fj, D0), lam)
    assert m1 <= m0 + 1e-13


@pytest.mark.parametrize("gen,n,lam,seed", [("sparse", 60, 0.1, 41), ("tridiag", 90, 0.15, 42)])
def test_pcd_cg_inner_solver_reaches_the_same_minimiser(gen, n, lam, seed):
    """The ML-cycle with PCD-CG (to Section 8's relative precision 1e-4) as
    the Newton-direction solver minimises the same strictly convex objective:
    it must reach the CD-based solve's minimiser, and the relative-precision
    stop must end the inner iteration well before its cap."""
    p = synth.random_problem(n, 2 * n, lam, seed, gen=gen)
    S = oracle.form_S(p.X)
    A_cd, _, i_cd, _ = oracle.solve(S, lam, tol=1e-11)
    A_pc, _, i_pc, _ = oracle.solve(S, lam, tol=1e-11, inner="pcd_cg")
    assert i_cd["status"] == 0 and i_pc["status"] == 0
    assert np.abs(A_pc - A_cd).max() <= 1e-9
    assert abs(i_pc["objective"] - i_cd["objective"]) <= 1e-12 * abs(i_cd["objective"])
    # the relative stop: from a fresh Newton LASSO, far fewer than 500 iterations
    A0 = np.diag(1.0 / (np.diag(S) + lam))
    W0 = np.linalg.inv(A0)
    fi, fj = oracle.free_set(S, W0, A0, lam)
    _, _, k = oracle.pcd(S, W0, A0, lam, fi, fj, 500, cg=True, rtol=1e-4)
    assert 1 <= k < 500
    with pytest.raises(ValueError):
        oracle.solve(S, lam, inner="newton")
