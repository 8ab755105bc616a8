"""Writes the exact solution of (regularize) used by the converged GPU parity tests.

Calls only ``oracle/`` (and the seeded input recipes).  Usage:

    python tests/golden/make_exact.py sq2 500 0.1

runs the FP64 oracle's P-APG (Fig. 2, with momentum restart) to KKT 1e-5 to pick the
candidate pairs (theta > 0 or a constraint value below 1e-3 of the data scale), then
``oracle.exact.solve`` (dual NNLS with constraint generation, exact up to rounding), and
stores the fitted values and subgradients in tests/golden/<recipe>_N<N>_g<gamma>_exact.npz.
"""
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import exact as E  # noqa: E402
from oracle import oracle as O  # noqa: E402
from paper_1407_7220_gb300 import datagen  # noqa: E402


def main():
    recipe, N, gamma = sys.argv[1], int(sys.argv[2]), float(sys.argv[3])
    X, yb, _ = datagen.make(recipe, N=N)
    t0 = time.time()
    o = O.Solver(X, yb, gamma=gamma, restart=True, restart_tol=1e-12)
    o.solve(1e-5, 2_000_000, check_every=100)
    G = O.residual(o.y_shifted, o.xi, X)
    off = ~np.eye(N, dtype=bool)
    cand = np.argwhere(((o.theta1 > 0) | (G < 1e-3 * O.data_scale(yb))) & off)
    y, xi, T, info = E.solve(X, yb, gamma, candidates=cand)
    print(f"oracle iterations {o.iters}, kkt {o.metrics['kkt']:.2e}; exact: {info}; {time.time() - t0:.0f} s")
    out = os.path.join(HERE, f"{recipe}_N{N}_g{gamma:g}_exact.npz")
    np.savez(out, y_hat=y, xi=xi, recipe=recipe, N=N, gamma=gamma, X_sum=X.sum(), ybar_sum=yb.sum(),
             shift=O.shift(yb), min_constraint=info["min_constraint"], complementarity=info["complementarity"],
             active=info["active"], pairs=info["pairs"], rounds=info["rounds"])


if __name__ == "__main__":
    main()
