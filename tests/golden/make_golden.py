"""Writes the converged FP64 oracle references used by the GPU parity tests.

Calls only ``oracle/`` (and the seeded input recipes).  Usage:

    python tests/golden/make_golden.py sq2 500 0.1 1e-8 [max_minutes] [restart_tol]

runs P-APG (with momentum restart; a restart needs the dual value to fall by more
than restart_tol relative, default 1e-12, so that rounding noise does not trigger
it) to KKT <= tol and stores fitted values, subgradients and run metadata in
tests/golden/<recipe>_N<N>_g<gamma>.npz.
"""
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import oracle as O  # noqa: E402
from paper_1407_7220_gb300 import datagen  # noqa: E402


def main():
    recipe, N, gamma, tol = sys.argv[1], int(sys.argv[2]), float(sys.argv[3]), float(sys.argv[4])
    max_minutes = float(sys.argv[5]) if len(sys.argv) > 5 else 120.0
    rtol = float(sys.argv[6]) if len(sys.argv) > 6 else 1e-12
    X, yb, _ = datagen.make(recipe, N=N)
    s = O.Solver(X, yb, gamma=gamma, restart=True, restart_tol=rtol)
    out = os.path.join(HERE, f"{recipe}_N{N}_g{gamma:g}.npz")
    t0 = time.time()
    while True:
        s.solve(tol, 50_000, check_every=10)
        m = s.metrics
        el = (time.time() - t0) / 60
        print(f"iters {s.iters} kkt {m['kkt']:.3e} fit {m['fit']:.9e} {el:.1f} min", flush=True)
        np.savez(out, y_hat=s.y_hat, xi=s.xi, kkt=m["kkt"], iters=s.iters, gamma=gamma, L=s.L, shift=s.s,
                 recipe=recipe, N=N, X_sum=X.sum(), ybar_sum=yb.sum(), restarts=s.restarts, restart_tol=rtol)
        if m["kkt"] <= tol or el > max_minutes:
            break


if __name__ == "__main__":
    main()
