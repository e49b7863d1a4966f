"""Seeded synthetic inputs for the l1-regularised log-det problem.

These generators are the only code shared between the CUDA solver's callers
(tests, bench) and the FP64 oracle's callers.  They hold none of the solver's
arithmetic: they draw a sparse SPD precision matrix Theta, Gaussian samples
x ~ N(0, Theta^{-1}) and the problem parameters, and stop there.  Forming the
empirical covariance S from the samples is step a1 of the method and is done
separately by each side.

Workload shapes follow the paper's synthetic experiments (Section 8.1): a
sparse precision matrix with a handful of nonzeros per row, Gaussian samples
drawn through its Cholesky factor (y = L^{-T} v with Theta = L L^T, v ~ N(0, I)).

Generator readings:
* tridiagonal Theta: Theta_ii = 1.25, Theta_{i,i+1} = Theta_{i+1,i} = -0.5.
* sparse Theta: floor(per_row * n / 2) distinct unordered off-diagonal pairs
  drawn uniformly, each with value +-U[lo, hi] (fair sign), mirrored, so a row
  has about `per_row` off-diagonals after symmetrisation; the diagonal is the
  row sum of absolute off-diagonals plus `margin` (strict diagonal dominance,
  hence SPD).
* seeds: numpy PCG64 with seed = 1000 * config + instance.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

__all__ = [
    "tridiag_theta",
    "sparse_theta",
    "gaussian_samples",
    "Problem",
    "config_problem",
    "random_problem",
    "batch_problems",
    "serving_trace",
    "CONFIGS",
]


def tridiag_theta(n: int, diag: float = 1.25, off: float = -0.5) -> np.ndarray:
    """Dense tridiagonal precision matrix (configuration 1)."""
    t = np.zeros((n, n), dtype=np.float64)
    idx = np.arange(n)
    t[idx, idx] = diag
    t[idx[:-1], idx[:-1] + 1] = off
    t[idx[:-1] + 1, idx[:-1]] = off
    return t


def sparse_theta(n: int, rng: np.random.Generator, per_row: float = 5.0,
                 lo: float = 0.1, hi: float = 0.3, margin: float = 0.5) -> np.ndarray:
    """Dense storage of a sparse, strictly diagonally dominant SPD matrix."""
    t = np.zeros((n, n), dtype=np.float64)
    npairs_total = n * (n - 1) // 2
    k = min(int(per_row * n // 2), npairs_total)
    if k > 0:
        lin = np.sort(rng.choice(npairs_total, size=k, replace=False))
        # map a linear index over the strict upper triangle (row-major) to (i, j)
        # row i starts at offset i*(n-1) - i*(i-1)/2
        i = (n - 0.5 - np.sqrt((n - 0.5) ** 2 - 2.0 * lin)).astype(np.int64)
        start = i * (n - 1) - i * (i - 1) // 2
        # guard the float root against off-by-one at row boundaries
        over = lin < start
        i[over] -= 1
        start = i * (n - 1) - i * (i - 1) // 2
        nxt = (i + 1) * (n - 1) - (i + 1) * i // 2
        under = lin >= nxt
        i[under] += 1
        start = i * (n - 1) - i * (i - 1) // 2
        j = lin - start + i + 1
        val = rng.uniform(lo, hi, size=k) * np.where(rng.random(k) < 0.5, -1.0, 1.0)
        t[i, j] = val
        t[j, i] = val
    t[np.arange(n), np.arange(n)] = np.abs(t).sum(axis=1) + margin
    return t


def gaussian_samples(theta: np.ndarray, m: int, rng: np.random.Generator) -> np.ndarray:
    """m samples (rows) of N(0, Theta^{-1}): x = L^{-T} v with Theta = L L^T."""
    import scipy.linalg as sla

    n = theta.shape[0]
    lower = np.linalg.cholesky(theta)
    v = rng.standard_normal((n, m))
    x = sla.solve_triangular(lower, v, lower=True, trans="T")
    return np.ascontiguousarray(x.T)


@dataclasses.dataclass
class Problem:
    """One seeded instance: samples X (m x n, row-major) and parameters."""

    name: str
    n: int
    m: int
    lam: float
    tol: float
    X: np.ndarray
    theta: np.ndarray | None = None
    seed: int = 0


# name, n, m, lambda, tol, generator
CONFIGS = {
    1: dict(name="tridiag n=100 m=200 lambda=0.2", n=100, m=200, lam=0.2, tol=1e-8, gen="tridiag"),
    2: dict(name="sparse n=2000 m=1000 lambda=0.1", n=2000, m=1000, lam=0.1, tol=1e-5, gen="sparse"),
    3: dict(name="sparse n=10000 m=5000 lambda=0.08", n=10000, m=5000, lam=0.08, tol=1e-5, gen="sparse"),
}


def _theta(gen: str, n: int, rng: np.random.Generator) -> np.ndarray:
    if gen == "tridiag":
        return tridiag_theta(n)
    if gen == "sparse":
        return sparse_theta(n, rng)
    raise ValueError(gen)


def config_problem(cfg: int, instance: int = 0, keep_theta: bool = False) -> Problem:
    """Configurations 1-3 (single solves)."""
    c = CONFIGS[cfg]
    seed = 1000 * cfg + instance
    rng = np.random.Generator(np.random.PCG64(seed))
    theta = _theta(c["gen"], c["n"], rng)
    x = gaussian_samples(theta, c["m"], rng)
    return Problem(c["name"], c["n"], c["m"], c["lam"], c["tol"], x,
                   theta if keep_theta else None, seed)


def random_problem(n: int, m: int, lam: float, seed: int, gen: str = "sparse",
                   tol: float = 1e-8) -> Problem:
    """A seeded instance of either generator at any size (test cases)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    theta = _theta(gen, n, rng)
    x = gaussian_samples(theta, m, rng)
    return Problem(f"{gen} n={n} m={m} lambda={lam}", n, m, lam, tol, x, theta, seed)


def batch_problems(count: int = 512, seed_base: int = 4000, n_lo: int = 32, n_hi: int = 512):
    """Configuration 4: independent instances, n ~ U[n_lo, n_hi], m = 2n,
    alternating tridiagonal / sparse generators; each is solved along the
    lambda path (0.4, 0.2, 0.1, 0.05)."""
    out = []
    for k in range(count):
        rng = np.random.Generator(np.random.PCG64(seed_base + k))
        n = int(rng.integers(n_lo, n_hi + 1))
        gen = "tridiag" if k % 2 == 0 else "sparse"
        theta = _theta(gen, n, rng)
        x = gaussian_samples(theta, 2 * n, rng)
        out.append(Problem(f"batch#{k} {gen} n={n}", n, 2 * n, 0.05, 1e-5, x, None, seed_base + k))
    return out


LAMBDA_PATH = (0.4, 0.2, 0.1, 0.05)


def serving_trace(count: int = 2000, seed: int = 5000, n_lo: int = 64, n_hi: int = 4096,
                  rate_per_s: float = 200.0):
    """Configuration 5: Poisson arrivals; n log-uniform in [n_lo, n_hi], m = n,
    lambda ~ U[0.05, 0.3].  Returns (arrival_s, n, lambda, instance_seed) rows;
    samples are drawn lazily with `serving_problem`."""
    rng = np.random.Generator(np.random.PCG64(seed))
    gaps = rng.exponential(1.0 / rate_per_s, size=count)
    t = np.cumsum(gaps)
    ns = np.exp(rng.uniform(math.log(n_lo), math.log(n_hi), size=count)).astype(np.int64)
    lams = rng.uniform(0.05, 0.3, size=count)
    return [(float(t[k]), int(ns[k]), float(lams[k]), seed * 10 + k) for k in range(count)]


def serving_problem(n: int, lam: float, seed: int) -> Problem:
    rng = np.random.Generator(np.random.PCG64(seed))
    theta = sparse_theta(n, rng)
    x = gaussian_samples(theta, n, rng)
    return Problem(f"serve n={n}", n, n, lam, 1e-5, x, None, seed)
