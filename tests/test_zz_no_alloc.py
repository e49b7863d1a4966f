"""The allocation-free free-set scan (glasso_free_set_noalloc) against the
regular context-based entry point (glasso_free_set).

glasso_free_set_noalloc serves callers that must not allocate device memory
(code under another framework's memory manager, or loops that cannot take
cudaMalloc's device-wide synchronisation); its scratch is a fixed array
inside the library.  This file is named so that pytest collects it last.
"""
import numpy as np
import pytest

import oracle
from paper_1607_00315_gb300 import synth

pytestmark = pytest.mark.gpu


def _state(n, seed, lam):
    p = synth.random_problem(n, 2 * n, lam, seed, gen="sparse")
    S = oracle.form_S(p.X)
    A, _, _, _ = oracle.solve(S, lam, tol=1e-2, max_cycles=2)
    _, L = oracle.cholesky(A)
    return S, A, oracle.inverse_from_chol(L)


def test_noalloc_matches_context_entry_point_on_consecutive_calls():
    import torch

    from paper_1607_00315_gb300 import build, glasso

    build.build()
    torch.cuda.init()
    ctx = glasso.Context(0)
    try:
        # two calls in a row with different sizes: a stale scratch value from
        # the first (larger) call would show up in the second
        for n, seed, lam in ((300, 71, 0.1), (130, 72, 0.08)):
            S, A, W = (torch.from_numpy(np.ascontiguousarray(x)).cuda() for x in _state(n, seed, lam))
            cap = n * (n + 1) // 2
            ri = torch.empty(cap, dtype=torch.int32, device="cuda")
            rj, ni, nj = torch.empty_like(ri), torch.empty_like(ri), torch.empty_like(ri)
            ra = torch.empty(cap, dtype=torch.float64, device="cuda")
            na = torch.empty_like(ra)
            cnt_ref, rk_ref, mk_ref = ctx.free_set(S, W, A, lam, ri, rj, ra)
            s, cnt, rk, mk = glasso.free_set_noalloc(S, W, A, lam, ni, nj, na)
            assert s == glasso.OK
            assert cnt == cnt_ref > n
            assert torch.equal(ni[:cnt], ri[:cnt]) and torch.equal(nj[:cnt], rj[:cnt])
            assert torch.equal(na[:cnt], ra[:cnt])
            assert abs(rk - rk_ref) <= 1e-12 * rk_ref and abs(mk - mk_ref) <= 1e-15 * max(mk_ref, 1)
    finally:
        ctx.close()


def test_noalloc_rejects_sizes_beyond_its_scratch():
    import torch

    from paper_1607_00315_gb300 import glasso

    torch.cuda.init()
    n = glasso.NOALLOC_MAX_N + 1
    t = torch.empty(1, dtype=torch.float64, device="cuda")
    i = torch.empty(1, dtype=torch.int32, device="cuda")

    class Shape:  # only .shape[0] is read before the size check rejects the call
        shape = (n, n)

        def data_ptr(self):
            return t.data_ptr()

    s, cnt, _, _ = glasso.free_set_noalloc(t, t, Shape(), 0.1, i, i)
    assert s == glasso.EINVAL and cnt == 0


def test_noalloc_at_its_largest_size_matches_the_oracle():
    """n = GLASSO_NOALLOC_MAX_N, where the fixed scratch (bit masks, row counts,
    partial sums) is used to its end: the free pairs are bit-exact against
    the oracle's eq. active_set scan, |S - W| on them is exact, and the KKT
    residual agrees with the oracle's to rounding.  A is the generator's
    sparse precision matrix, W its inverse, S the covariance of 512 samples,
    so both halves of the free-set rule (A_ij != 0, |G_ij| > lambda) occur."""
    import torch

    from paper_1607_00315_gb300 import build, glasso

    build.build()
    torch.cuda.init()
    n, lam = glasso.NOALLOC_MAX_N, 0.05
    rng = np.random.default_rng(4096)
    theta = synth.sparse_theta(n, rng)
    X = synth.gaussian_samples(theta, 512, rng)
    S = X.T @ X / X.shape[0]
    W = np.linalg.inv(theta)
    S, W = (S + S.T) / 2, (W + W.T) / 2  # exactly symmetric, as the solver's matrices are
    fi, fj = oracle.free_set(S, W, theta, lam)
    rk_ref, mk_ref = oracle.rel_kkt(S, W, theta, lam)
    offd = int(np.count_nonzero(fi != fj))
    supp = int(np.count_nonzero(np.triu(theta, 1)))
    assert offd > supp > 0  # pairs from both halves of the rule
    Sd, Wd, Ad = (torch.from_numpy(np.ascontiguousarray(x)).cuda() for x in (S, W, theta))
    cap = n * (n + 1) // 2
    oi = torch.full((cap,), -1, dtype=torch.int32, device="cuda")
    oj = torch.full_like(oi, -1)
    ab = torch.empty(cap, dtype=torch.float64, device="cuda")
    for _ in range(2):  # the second call runs on the first one's leftover scratch
        s, cnt, rk, mk = glasso.free_set_noalloc(Sd, Wd, Ad, lam, oi, oj, ab)
        assert s == glasso.OK and cnt == len(fi)
        assert np.array_equal(oi[:cnt].cpu().numpy(), fi)
        assert np.array_equal(oj[:cnt].cpu().numpy(), fj)
        assert np.array_equal(ab[:cnt].cpu().numpy(), np.abs(S - W)[fi, fj])
        assert abs(rk - rk_ref) <= 1e-12 * rk_ref
        assert abs(mk - mk_ref) <= 1e-15 * max(mk_ref, 1.0)
