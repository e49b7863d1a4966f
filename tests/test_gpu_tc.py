"""The tcgen05 tensor-core GEMM, through the C ABI: S = X^T X / m from FP32
samples in a mixed-precision context (the n = 10000, X FP32 workload's step
a1), against the FP64 oracle's S.

Each product is formed as split TF32 (x = hi + lo, hi hi + hi lo + lo hi): at
most about 2^-20 relative error per product; the partial sums of every 8-wide
k step are added in FP32 with round-to-nearest outside the tensor core, so the
summation adds at most (m / 8 + 2) 2^-24 (no truncation bias).  The bound per
entry is (2^-20 + (m / 8 + 2) 2^-24) (|X|^T |X|)_ij / m.
"""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mctx():
    import torch

    from paper_1607_00315_gb300 import build, glasso

    build.build()
    torch.cuda.init()
    c = glasso.Context(0, precision=glasso.MIXED)
    yield c
    c.close()


@pytest.mark.parametrize("m,n,center", [(64, 128, False), (200, 300, False), (1000, 513, True),
                                        (37, 1, False), (130, 260, True)])
def test_form_S_tensor_cores(mctx, m, n, center):
    import torch

    rng = np.random.default_rng(m + n)
    X = (rng.standard_normal((m, n)) * rng.uniform(0.5, 2.0, n)).astype(np.float32)
    S_ref = oracle.form_S(X.astype(np.float64), center=center)
    S = torch.empty((n, n), dtype=torch.float64, device="cuda")
    mctx.form_S(torch.from_numpy(X).cuda(), S, center=center)
    S = S.cpu().numpy()
    Xc = X.astype(np.float64) - (X.astype(np.float64).mean(0) if center else 0.0)
    bound = (2.0 ** -20 + (m / 8 + 2) * 2.0 ** -24) * (np.abs(Xc).T @ np.abs(Xc)) / m + 1e-30
    err = np.abs(S - S_ref)
    assert np.all(err <= bound), (err / bound).max()
    assert np.array_equal(S, S.T)
    # FP32-level, not FP64: the error is far above FP64 rounding somewhere
    assert err.max() > 1e-12 * np.abs(S_ref).max()
