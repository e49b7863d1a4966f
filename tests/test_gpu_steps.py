"""GPU parity of each step of one relaxation against the FP64 oracle.

Every call goes through the C ABI (libglasso.so) on device buffers; the
expected values come from oracle/ on the same seeded inputs.  Sizes span
several 32-wide tiles with ragged tails; tolerances follow from FP64
rounding of the reassociated sums (documented per test).
"""
import numpy as np
import pytest

import oracle
from paper_1607_00315_gb300 import synth

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


def _dev(a):
    import torch

    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _spd(n, seed, cond=50.0):
    rng = np.random.default_rng(seed)
    q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    return (q * np.exp(rng.uniform(0, np.log(cond), n))) @ q.T


def _problem(n, seed, lam=0.1, gen="sparse"):
    p = synth.random_problem(n, max(2 * n, 8), lam, seed, gen=gen)
    S = oracle.form_S(p.X)
    return p, S


@pytest.mark.parametrize("m,n,center,f32", [(7, 1, False, False), (40, 33, False, False),
                                            (300, 97, True, False), (130, 65, False, True)])
def test_form_S(ctx, m, n, center, f32):
    rng = np.random.default_rng(n)
    X = rng.standard_normal((m, n))
    if f32:
        X = X.astype(np.float32)
    S_ref = oracle.form_S(X.astype(np.float64), center=center)
    import torch

    S = torch.empty((n, n), dtype=torch.float64, device="cuda")
    ctx.form_S(_dev(X), S, center=center)
    # FP64 sums of m products reassociated: |err| <= m eps max|S|
    assert np.abs(S.cpu().numpy() - S_ref).max() <= 4 * m * 2.2e-16 * np.abs(S_ref).max()


@pytest.mark.parametrize("n", [1, 2, 31, 32, 33, 100, 161, 257])
def test_potrf_and_inverse(ctx, n):
    A = _spd(n, n)
    info_ref, L_ref = oracle.cholesky(A)
    W_ref = oracle.inverse_from_chol(L_ref)
    Ad = _dev(A)
    info, logdet = ctx.potrf(Ad)
    assert info == 0 == info_ref
    L = np.tril(Ad.cpu().numpy())
    assert np.abs(L - L_ref).max() <= 1e-12 * np.abs(L_ref).max()
    assert abs(logdet - oracle.logdet_from_chol(L_ref)) <= 1e-12 * max(1.0, abs(logdet))
    # upper triangle untouched
    assert np.array_equal(np.triu(Ad.cpu().numpy(), 1), np.triu(A, 1))
    import torch

    W = torch.empty_like(Ad)
    ctx.inverse(Ad, W)
    W = W.cpu().numpy()
    assert np.array_equal(W, W.T)
    assert np.abs(W - W_ref).max() <= 1e-10 * np.abs(W_ref).max()


@pytest.mark.parametrize("n,k", [(5, 3), (64, 40), (100, 77), (130, 31)])
def test_potrf_reports_first_bad_pivot(ctx, n, k):
    A = _spd(n, 3 * n)
    A[k, k] -= 1e3
    info_ref, _ = oracle.cholesky(A)
    info, _ = ctx.potrf(_dev(A))
    assert info == info_ref > 0


def _state(n, seed, lam):
    """An iterate with some off-diagonal support, its inverse and S."""
    p, S = _problem(n, seed, lam)
    A = np.diag(1.0 / (np.diag(S) + lam))
    # take two oracle relaxations' worth of structure: solve loosely
    A, W, _, _ = oracle.solve(S, lam, tol=1e-2, max_cycles=2)
    info, L = oracle.cholesky(A)
    W = oracle.inverse_from_chol(L)
    return S, A, W


@pytest.mark.parametrize("n,lam", [(37, 0.1), (130, 0.08), (300, 0.12)])
def test_free_set_full_and_kkt(ctx, n, lam):
    S, A, W = _state(n, n + 1, lam)
    fi, fj = oracle.free_set(S, W, A, lam)
    rk_ref, mk_ref = oracle.rel_kkt(S, W, A, lam)
    import torch

    cap = n * (n + 1) // 2
    oi = torch.empty(cap, dtype=torch.int32, device="cuda")
    oj = torch.empty_like(oi)
    ab = torch.empty(cap, dtype=torch.float64, device="cuda")
    cnt, rk, mk = ctx.free_set(_dev(S), _dev(W), _dev(A), lam, oi, oj, ab)
    assert cnt == len(fi)
    assert np.array_equal(oi[:cnt].cpu().numpy(), fi) and np.array_equal(oj[:cnt].cpu().numpy(), fj)
    assert np.allclose(ab[:cnt].cpu().numpy(), np.abs(S - W)[fi, fj], rtol=0, atol=0)
    assert abs(rk - rk_ref) <= 1e-12 * rk_ref and abs(mk - mk_ref) <= 1e-15 * max(mk_ref, 1)


def test_free_set_candidates(ctx):
    n, lam = 90, 0.1
    S, A, W = _state(n, 5, lam)
    rng = np.random.default_rng(1)
    iu = np.triu_indices(n)
    sel = np.sort(rng.choice(len(iu[0]), 700, replace=False))
    ci, cj = iu[0][sel].astype(np.int32), iu[1][sel].astype(np.int32)
    ri, rj = oracle.free_set(S, W, A, lam, cand=(ci, cj))
    import torch

    oi = torch.empty(700, dtype=torch.int32, device="cuda")
    oj = torch.empty_like(oi)
    cnt, _, _ = ctx.free_set(_dev(S), _dev(W), _dev(A), lam, oi, oj, None,
                             cand=(_dev(ci), _dev(cj)))
    assert cnt == len(ri)
    assert np.array_equal(oi[:cnt].cpu().numpy(), ri) and np.array_equal(oj[:cnt].cpu().numpy(), rj)


@pytest.mark.parametrize("nf,ties,psupp", [(1, False, 1.0), (20, False, 0.15), (1000, False, 0.3),
                                           (5003, True, 0.1), (4000, True, 0.5), (300, False, 0.0)])
def test_hierarchy_bit_exact(ctx, nf, ties, psupp):
    rng = np.random.default_rng(nf)
    insupp = (rng.random(nf) < psupp).astype(np.uint8)
    if nf == 1:
        insupp[:] = 1
    absg = (rng.integers(0, 9, nf) / 3.0) if ties else rng.exponential(1.0, nf)
    tag_ref, L_ref = oracle.hierarchy(absg, insupp)
    import torch

    tag = torch.empty(nf, dtype=torch.uint8, device="cuda")
    L = ctx.hierarchy(_dev(absg), _dev(insupp), tag)
    assert L == L_ref
    assert np.array_equal(tag.cpu().numpy(), tag_ref)


@pytest.mark.parametrize("n,lam,sweeps", [(40, 0.1, 1), (129, 0.08, 2), (260, 0.1, 3)])
def test_cd_sweeps(ctx, n, lam, sweeps):
    S, A, W = _state(n, 2 * n, lam)
    fi, fj = oracle.free_set(S, W, A, lam)
    D_ref, U_ref = oracle.cd_sweeps(S, W, A, lam, fi, fj, sweeps)
    import torch

    D = torch.zeros(len(fi), dtype=torch.float64, device="cuda")
    U = torch.zeros((n, n), dtype=torch.float64, device="cuda")
    ctx.cd_sweeps(_dev(S), _dev(W), _dev(A), lam, _dev(fi), _dev(fj), sweeps, D, U)
    D = D.cpu().numpy()
    U = U.cpu().numpy()
    # the blocked sweep equals the sequential one up to reassociation of the
    # length-n dots; the chain amplifies that by the sweep's contraction only
    scale = np.abs(D_ref).max()
    assert np.abs(D - D_ref).max() <= 1e-9 * scale
    assert np.abs(U - U_ref).max() <= 1e-9 * np.abs(U_ref).max()
    # zeros of the shrinkage are exact on both sides for clearly inactive pairs
    assert np.array_equal(D == 0, D_ref == 0) or np.abs(D - D_ref).max() <= 1e-12


@pytest.fixture(scope="module")
def mctx():
    import torch

    from paper_1607_00315_gb300 import build, glasso

    build.build()
    torch.cuda.init()
    c = glasso.Context(0, precision=glasso.MIXED)
    yield c
    c.close()


# pair lists of one block (<= 128 coordinates), two blocks, and several with
# a ragged last block; one to three sweeps (the pipelined FP32 sweep keeps
# two copies of U and the matrices of the next two blocks, so these are the
# cases whose bookkeeping differs)
# The pipelined kernel runs when its interaction matrices (three 64 KB per
# block) fit in n^2 doubles, else the one-copy sweep does.  Pipelined: 241
# pairs (two blocks), 640, 1431 (five, twelve); one-copy: 95 (one block),
# 155 and 250 (two), 406, 811, 1123.
@pytest.mark.parametrize("n,lam,sweeps", [(240, 0.35, 1), (240, 0.35, 3), (500, 0.15, 2), (700, 0.1, 3),
                                          (30, 0.15, 1), (30, 0.15, 3), (45, 0.15, 2), (40, 0.1, 1),
                                          (70, 0.1, 2), (129, 0.08, 1), (260, 0.1, 3)])
def test_cd_sweeps_mixed(mctx, n, lam, sweeps):
    """The mixed solve's FP32 sweep against the FP64 sequential sweep of the
    oracle.  W and U are rounded to FP32 and the chain and the length-n dots
    run in FP32: each b_t = G_t + (W Delta W)_t carries an error of at most
    about n 2^-24 max|b| (FP32 dot of n terms), and the coordinate's
    increment that error divided by a_t; the Gauss-Seidel sweep (a
    contraction) does not amplify it beyond a small factor per sweep, so
    |Delta - Delta_ref| <= 8 sweeps n 2^-24 max|b| / min a.  U is checked
    against Delta W formed in FP64 from the GPU's own Delta, which pins the
    row-update bookkeeping independently of the chain's rounding: each entry
    is a sum of at most d_max sweeps updates rounded to FP32, d_max the
    largest number of pairs touching a row.  A wrong cross term or a skipped
    block gives errors of the order of Delta itself."""
    S, A, W = _state(n, 2 * n + 1, lam)
    fi, fj = oracle.free_set(S, W, A, lam)
    D_ref, U_ref = oracle.cd_sweeps(S, W, A, lam, fi, fj, sweeps)
    import torch

    D = torch.zeros(len(fi), dtype=torch.float64, device="cuda")
    U = torch.zeros((n, n), dtype=torch.float64, device="cuda")
    mctx.cd_sweeps(_dev(S), _dev(W), _dev(A), lam, _dev(fi), _dev(fj), sweeps, D, U)
    D = D.cpu().numpy()
    U = U.cpu().numpy()
    eps = 2.0 ** -24
    a = np.where(fi == fj, W[fi, fi] ** 2, W[fi, fj] ** 2 + W[fi, fi] * W[fj, fj])
    bmax = np.abs((S - W)[fi, fj]).max() + np.abs((W @ U_ref)[fi, fj]).max()
    tol_d = 8 * sweeps * n * eps * bmax / a.min()
    err_d = np.abs(D - D_ref).max()
    assert err_d <= tol_d, (len(fi), err_d, tol_d)
    # U against Delta W in FP64 from the returned Delta.  Each pair is updated
    # once per sweep, so sum_k |mu_k| = sum_s |Delta_s - Delta_{s-1}| (the
    # oracle's sweep-by-sweep Delta); the FP32 sum of those terms (W and mu
    # rounded) errs by at most about (2 + d_max sweeps) 2^-24 of |mu| |W|,
    # plus FP32 underflow
    Dm = np.zeros((n, n))
    Dm[fi, fj] = D
    Dm[fj, fi] = D
    prev, msum = np.zeros(len(fi)), np.zeros(len(fi))
    for s_ in range(1, sweeps + 1):
        Ds = D_ref if s_ == sweeps else oracle.cd_sweeps(S, W, A, lam, fi, fj, s_)[0]
        msum += np.abs(Ds - prev)
        prev = Ds
    msum = np.maximum(msum, np.abs(D))  # pairs the two sides zero differently
    Mm = np.zeros((n, n))
    Mm[fi, fj] = msum
    Mm[fj, fi] = msum
    E = np.abs(Mm) @ np.abs(W)
    dmax = np.bincount(np.concatenate([fi, fj[fi != fj]]), minlength=n).max()
    # (+ entries of W below FP32's smallest normal, 2^-126, flush to zero)
    bound = 2 * (2 + dmax * sweeps) * eps * E + (dmax * sweeps + 1) * 2.0 ** -126 * msum.max() + 1e-300
    ratio = (np.abs(U - Dm @ W) / bound).max()
    assert ratio <= 1.0, (ratio, dmax)
    # exact zeros: the patterns agree except where the oracle's increment is
    # itself within the FP32 error of zero
    differ = (D == 0) != (D_ref == 0)
    assert np.all(np.abs(D_ref[differ]) <= tol_d)


def test_line_search(ctx):
    n, lam = 120, 0.1
    S, A, W = _state(n, 11, lam)
    fi, fj = oracle.free_set(S, W, A, lam)
    D, _ = oracle.cd_sweeps(S, W, A, lam, fi, fj, 3)
    for scale in (1.0, 30.0):
        d = D * scale
        _, F0 = oracle.objective(S, A, lam)
        rc, A1_ref, F1_ref, al_ref, tr_ref = oracle.line_search(S, W, A, lam, fi, fj, d, F0)
        Ad = _dev(A)
        s, F1, al, tr = ctx.line_search(_dev(S), _dev(W), Ad, lam, _dev(fi), _dev(fj), _dev(d), F0)
        assert s == rc == 0
        assert (al, tr) == (al_ref, tr_ref)
        assert np.abs(Ad.cpu().numpy() - A1_ref).max() <= 1e-15 * np.abs(A1_ref).max()
        assert abs(F1 - F1_ref) <= 1e-11 * abs(F1_ref)


def test_objective(ctx):
    n, lam = 77, 0.2
    S, A, W = _state(n, 3, lam)
    _, F_ref = oracle.objective(S, A, lam)
    info, F = ctx.objective(_dev(S), _dev(A), lam)
    assert info == 0 and abs(F - F_ref) <= 1e-12 * abs(F_ref)
