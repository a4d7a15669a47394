"""Seeded synthetic inputs shared by the tests, the bench and the CPU baseline.

This module holds no arithmetic of the SMC method: it only draws problem
instances, particle clouds, log-weights and copy-count vectors with numpy's own
generator, in the shapes and distributions of the workloads:

* Gaussian target (the plain FP64 sampler and the batched samplers):
  mu ~ U[-2, 2]^D, A_ij ~ N(0, 1), Sigma = A A^T / 4 + I.
* Logistic-regression data: X_mj ~ N(0, 1) (FP32), beta* ~ N(0, I),
  y_m ~ Bernoulli(sigmoid(x_m . beta*)).
* Resample / redistribute inputs: particles x ~ N(0, 1) in D-wide rows,
  log-weights i.i.d. N(0, s^2), or the adversarial one-hot case (one entry 0,
  the rest -inf).

It imports nothing from the rest of the package, so importing it loads no
native code.
"""
from __future__ import annotations

import numpy as np


def rng(seed: int, stream: int = 0) -> np.random.Generator:
    return np.random.default_rng(np.random.SeedSequence([int(seed), int(stream), 0x534D43]))


def gaussian_target(D: int, seed: int = 0):
    """(mu, Sigma) with mu ~ U[-2,2]^D and Sigma = A A^T / 4 + I, A_ij ~ N(0,1)."""
    g = rng(seed, 1)
    mu = g.uniform(-2.0, 2.0, size=D)
    A = g.standard_normal((D, D))
    Sigma = A @ A.T / 4.0 + np.eye(D)
    Sigma = 0.5 * (Sigma + Sigma.T)
    return mu, Sigma


def logistic_data(M: int, D: int, seed: int = 0):
    """(X float32 [M, D], y float32 [M] in {0, 1}, beta_star [D])."""
    g = rng(seed, 2)
    X = g.standard_normal((M, D)).astype(np.float32)
    beta = g.standard_normal(D)
    logits = X.astype(np.float64) @ beta
    p = 1.0 / (1.0 + np.exp(-logits))
    y = (g.uniform(size=M) < p).astype(np.float32)
    return X, y, beta


def particles(N: int, D: int, seed: int = 0, dtype=np.float32) -> np.ndarray:
    """x ~ N(0, 1), shape [N, D]."""
    return rng(seed, 3).standard_normal((N, D)).astype(dtype)


def log_weights(N: int, s: float, seed: int = 0) -> np.ndarray:
    """logw_i ~ N(0, s^2), float64."""
    return rng(seed, 4).normal(0.0, s, size=N)


def one_hot_log_weights(N: int, seed: int = 0) -> np.ndarray:
    """All -inf except one entry (index drawn from the seed) equal to 0."""
    lw = np.full(N, -np.inf)
    lw[int(rng(seed, 5).integers(0, N))] = 0.0
    return lw


def log_pi(N: int, seed: int = 0, dtype=np.float32) -> np.ndarray:
    """A cached log-target payload carried next to each particle row."""
    return (-0.5 * rng(seed, 6).chisquare(4, size=N)).astype(dtype)


def composition(N: int, seed: int = 0, kind: str = "multinomial") -> np.ndarray:
    """A copy-count vector with sum N (int32).

    multinomial : N draws over N equally likely particles
    skewed      : multinomial over weights exp(N(0, 2^2))
    one_hot     : all N copies on one index
    ones        : every particle kept once
    """
    g = rng(seed, 7)
    if kind == "ones":
        return np.ones(N, dtype=np.int32)
    if kind == "one_hot":
        c = np.zeros(N, dtype=np.int32)
        c[int(g.integers(0, N))] = N
        return c
    if kind == "skewed":
        p = np.exp(g.normal(0.0, 2.0, size=N))
    else:
        p = np.ones(N)
    p = p / p.sum()
    return g.multinomial(N, p).astype(np.int32)


def batch_shapes(count: int, seed: int = 0, n_min: int = 1 << 10, n_max: int = 1 << 18,
                 dims=(2, 8, 32)) -> list[tuple[int, int]]:
    """(N, D) of `count` independent samplers: N log-uniform integers in
    [n_min, n_max], D drawn uniformly from `dims` (the batched workload)."""
    g = rng(seed, 3)
    ln = g.uniform(np.log(n_min), np.log(n_max), size=count)
    ns = np.clip(np.floor(np.exp(ln)).astype(np.int64), n_min, n_max)
    ds = g.choice(np.asarray(dims, dtype=np.int64), size=count)
    return [(int(n), int(d)) for n, d in zip(ns, ds)]
