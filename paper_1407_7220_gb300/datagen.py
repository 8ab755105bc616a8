"""Seeded synthetic instances shaped like the paper's experiments.

This module holds the input recipes only (no part of the solver's
arithmetic); the tests feed the same arrays to the CUDA path and to the CPU
oracle.  The data model is the paper's Eq. (data): ybar_l = f0(x_l) + eps_l
with f0 convex and x_l i.i.d. from a continuous distribution (Sec. II).

Recipes (NumPy ``default_rng``; default seed = 1000 + recipe index):
  ``sq2``      (1) x ~ U[-1,1]^n, f0 = ||x||^2, eps ~ N(0, 0.1^2)            N=500,  n=2
  ``maxaff``   (2) x ~ N(0, I), f0 = max_{k<=8} a_k^T x + b_k,
                   a_k ~ N(0, I), b_k ~ N(0, 1), eps ~ N(0, (0.1 std f0)^2)   N=20000, n=10
  ``lse``      (3) x ~ U[-1,1]^n, f0 = log sum_{k<=16} exp(a_k^T x),
                   a_k ~ N(0, I/n), eps ~ N(0, 0.05^2)                       N=100000, n=20
  ``batch``    (4) per fit: N_i log-uniform in [64, 4096], n_i in {1, 2, 5},
                   x ~ N(0, I), f0 = ||x||^2 + |x_1|, eps ~ N(0, 0.1^2)      1024 fits
  ``sumexp``   (5) x ~ U[-1,1]^n, f0 = sum_j exp(x_j / 2), eps ~ N(0, 0.1^2) N=5000, n=5
  ``xqx``      (6) the small experiment of Sec. III: Lambda (n x n), x and eps with i.i.d.
                   N(0, 1) entries, f0 = 1/2 x^T Q x with Q = Lambda^T Lambda  N=100, n=5
"""
from __future__ import annotations

import numpy as np

RECIPES = {
    "sq2": dict(index=1, N=500, n=2),
    "maxaff": dict(index=2, N=20000, n=10),
    "lse": dict(index=3, N=100000, n=20),
    "batch": dict(index=4, B=1024),
    "sumexp": dict(index=5, N=5000, n=5),
    "xqx": dict(index=6, N=100, n=5),
}


def default_seed(recipe: str) -> int:
    return 1000 + RECIPES[recipe]["index"]


def make(recipe: str, N: int | None = None, n: int | None = None, seed: int | None = None):
    """Return (X (N x n float64), ybar (N,), f0(X) (N,)) for a recipe."""
    r = RECIPES[recipe]
    N = int(r["N"] if N is None else N)
    n = int(r["n"] if n is None else n)
    rng = np.random.default_rng(default_seed(recipe) if seed is None else seed)
    if recipe == "sq2":
        X = rng.uniform(-1.0, 1.0, size=(N, n))
        f0 = (X * X).sum(axis=1)
        eps = rng.normal(0.0, 0.1, size=N)
    elif recipe == "maxaff":
        A = rng.normal(0.0, 1.0, size=(8, n))
        b = rng.normal(0.0, 1.0, size=8)
        X = rng.normal(0.0, 1.0, size=(N, n))
        f0 = (X @ A.T + b).max(axis=1)
        eps = rng.normal(0.0, 0.1 * float(f0.std()), size=N)
    elif recipe == "lse":
        A = rng.normal(0.0, np.sqrt(1.0 / n), size=(16, n))
        X = rng.uniform(-1.0, 1.0, size=(N, n))
        Z = X @ A.T
        zmax = Z.max(axis=1, keepdims=True)
        f0 = (zmax[:, 0] + np.log(np.exp(Z - zmax).sum(axis=1)))
        eps = rng.normal(0.0, 0.05, size=N)
    elif recipe == "sumexp":
        X = rng.uniform(-1.0, 1.0, size=(N, n))
        f0 = np.exp(0.5 * X).sum(axis=1)
        eps = rng.normal(0.0, 0.1, size=N)
    elif recipe == "xqx":
        Lam = rng.normal(0.0, 1.0, size=(n, n))
        X = rng.normal(0.0, 1.0, size=(N, n))
        f0 = 0.5 * np.einsum("lj,jk,lk->l", X, Lam.T @ Lam, X)
        eps = rng.normal(0.0, 1.0, size=N)
    else:
        raise ValueError(f"recipe {recipe!r} has no single instance; use make_batch")
    return np.ascontiguousarray(X), f0 + eps, f0


def make_batch(B: int = 1024, seed: int | None = None, Nmin: int = 64, Nmax: int = 4096,
               dims=(1, 2, 5)):
    """Recipe (4): B independent fits of uneven size.  Returns a list of (X, ybar, f0)."""
    rng = np.random.default_rng(default_seed("batch") if seed is None else seed)
    out = []
    Ns = np.rint(np.exp(rng.uniform(np.log(Nmin), np.log(Nmax), size=B))).astype(np.int64)
    ns = rng.choice(np.asarray(dims), size=B)
    for i in range(B):
        N, n = int(Ns[i]), int(ns[i])
        X = rng.normal(0.0, 1.0, size=(N, n))
        f0 = (X * X).sum(axis=1) + np.abs(X[:, 0])
        eps = rng.normal(0.0, 0.1, size=N)
        out.append((np.ascontiguousarray(X), f0 + eps, f0))
    return out
