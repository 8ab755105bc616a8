"""Writes the oracle's derivatives for the differentiation configuration (recipe (5)).

Calls only ``oracle/`` (and the seeded input recipes).  Usage:

    python tests/golden/make_c5.py [N] [K] [directions] [fd_directions]

Defaults: N = 5000, n = 5, gamma = 0.1, K = 500 unrolled plain P-APG iterations from
Iteration 0 (Fig. 2), 32 random directions, 2 of them also by central finite differences.
The loss is ||yhat - t||^2 with the target t = f0(X) held fixed; its gradient seed at the
oracle's fitted values is u = 2 (yhat - t).  Stored (tests/golden/sumexp_N<N>_K<K>_jvp.npz):
the oracle's fitted values, u . (d yhat / d(ybar, X)) [d_k] for every direction d_k (forward
mode, ``oracle.papg_jvp_multi``), and for the first fd_directions directions the central
differences (L(+h d) - L(-h d)) / (2 h) of the oracle's loss for h = 1e-7, 1e-8, 1e-9.  The
unrolled map is piecewise linear in theta (the projection max(0, .) of every pair), so a
central difference agrees with the derivative only when no pair changes sides within +-h: at
N = 1000, K = 100 that needed h <= 1e-7 (larger steps cross kinks and differ by 1e-3).  Directions: rng =
default_rng(seed); for each k, dybar ~ N(0, I_N) then dX ~ N(0, I_{N x n}).
"""
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import oracle as O  # noqa: E402
from paper_1407_7220_gb300 import datagen  # noqa: E402

SEED = 2024


def directions(N: int, n: int, D: int, seed: int = SEED):
    rng = np.random.default_rng(seed)
    dY = np.empty((D, N))
    dX = np.empty((D, N, n))
    for k in range(D):
        dY[k] = rng.normal(size=N)
        dX[k] = rng.normal(size=(N, n))
    return dY, dX


def main():
    N = int(sys.argv[1]) if len(sys.argv) > 1 else 5000
    K = int(sys.argv[2]) if len(sys.argv) > 2 else 500
    D = int(sys.argv[3]) if len(sys.argv) > 3 else 32
    F = int(sys.argv[4]) if len(sys.argv) > 4 else 2
    n, gamma = 5, 0.1
    hs = (1e-7, 1e-8, 1e-9)
    X, yb, f0 = datagen.make("sumexp", N=N, n=n)
    L, s = O.lipschitz(X, gamma), O.shift(yb)
    t0 = time.time()
    dY, dX = directions(N, n, D)
    yhat, J = O.papg_jvp_multi(X, yb, gamma, L, s, K, dY, dX)
    u = 2.0 * (yhat - f0)
    jvp = J @ u
    print(f"JVP of {D} directions: {time.time() - t0:.0f} s", flush=True)

    def loss(yb_, X_):
        o = O.Solver(X_, yb_, gamma=gamma, L=L, s=s, restart=False)
        o.iterate(K)
        return float(((o.y_hat - f0) ** 2).sum())

    fd = np.empty((F, len(hs)))
    for k in range(F):
        for i, h in enumerate(hs):
            fd[k, i] = (loss(yb + h * dY[k], X + h * dX[k]) - loss(yb - h * dY[k], X - h * dX[k])) / (2 * h)
            print(f"direction {k} h {h:g}: jvp {jvp[k]:.12e} fd {fd[k, i]:.12e} "
                  f"rel {abs(fd[k, i] - jvp[k]) / abs(jvp[k]):.2e}", flush=True)
    out = os.path.join(HERE, f"sumexp_N{N}_K{K}_jvp.npz")
    np.savez(out, y_hat=yhat, jvp=jvp, fd=fd, fd_h=np.array(hs), seed=SEED, N=N, n=n, K=K, gamma=gamma, L=L, shift=s,
             X_sum=X.sum(), ybar_sum=yb.sum())
    print(f"wrote {out} in {time.time() - t0:.0f} s")


if __name__ == "__main__":
    main()
