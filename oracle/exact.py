"""Exact solution of problem (regularize) by its dual NNLS on a growing set of pairs.

TEST INFRASTRUCTURE ONLY (like the rest of ``oracle/``): the reference the converged
GPU fits are compared with.  It shares no code with the CUDA path.

Problem (regularize) of Sec. II-C with the pairwise constraints of problem (original),

    min 1/2 ||y - h||^2 + gamma/2 ||xi||^2   s.t.  y_l1 - y_l2 - xi_l2^T (x_l1 - x_l2) >= 0,

has the Lagrangian dual (dual of Eq. (lambda_dual) at K = N, without the y >= 0 rows, which
the shift h = ybar + s makes inactive)

    min_{theta >= 0}  1/2 || A_1^T theta + h ||^2 + 1/(2 gamma) || A_2^T theta ||^2,

a nonnegative least-squares problem, with y = h + A_1^T theta and xi = A_2^T theta / gamma
(Step 1's closed form).  At the solution most pairs are inactive (theta = 0), so the NNLS is
solved on a candidate set W of pairs only (scipy's Lawson-Hanson active-set NNLS, which
terminates with an exact solution of the restricted problem), and every pair outside W is
then checked for feasibility at the resulting (y, xi).  Violated pairs join W and the NNLS is
solved again.  When no pair is violated, (y, xi, theta) satisfies the KKT conditions of the
full problem: stationarity by construction, theta >= 0, primal feasibility of every pair, and
complementary slackness on W (theta = 0 outside W).  This is the textbook constraint-generation
(cutting-plane) method for a QP; its answer does not depend on any iteration count.
"""
from __future__ import annotations

import numpy as np

from . import oracle as O


def _restricted_matrix(X: np.ndarray, pairs: np.ndarray, gamma: float) -> np.ndarray:
    """[A_1^T; A_2^T / sqrt(gamma)] restricted to the columns of the given pairs (rows of (l1, l2))."""
    N, n = X.shape
    P = pairs.shape[0]
    A = np.zeros((N + N * n, P))
    cols = np.arange(P)
    l1, l2 = pairs[:, 0], pairs[:, 1]
    A[l1, cols] += 1.0        # row p of A_1 is e_l1 - e_l2
    A[l2, cols] -= 1.0
    d = -(X[l1] - X[l2]) / np.sqrt(gamma)   # row p of A_2: -(x_l1 - x_l2)^T in block l2
    for k in range(n):
        A[N + l2 * n + k, cols] = d[:, k]
    return A


def solve(X, ybar, gamma: float, candidates=None, s: float | None = None, feas_tol: float = 1e-13,
          max_rounds: int = 50, add_per_round: int = 20000):
    """Exact (y_hat, xi, theta, info) of (regularize) for data (X, ybar).

    candidates: optional (k, 2) integer array of pairs to start from (for instance the pairs
    where a P-APG iterate has theta > 0 or a small constraint value).  s: the shift (default:
    the oracle's reading, ``oracle.shift``).  feas_tol: a pair with constraint value below
    -feas_tol * max(1, range ybar) counts as violated."""
    from scipy.optimize import nnls

    X = np.ascontiguousarray(np.asarray(X, dtype=np.float64))
    ybar = np.asarray(ybar, dtype=np.float64)
    N, n = X.shape
    s = O.shift(ybar) if s is None else float(s)
    h = ybar + s
    sigma = O.data_scale(ybar)
    if candidates is None:
        # every pair between near neighbours in x (a start; the rounds add what is missing)
        d2 = ((X[:, None, :] - X[None, :, :]) ** 2).sum(-1)
        np.fill_diagonal(d2, np.inf)
        nb = np.argsort(d2, axis=1)[:, :min(8, N - 1)]
        candidates = np.array([(a, b) for a in range(N) for b in nb[a]] + [(b, a) for a in range(N) for b in nb[a]])
    W = {tuple(map(int, p)) for p in np.asarray(candidates).reshape(-1, 2) if p[0] != p[1]}
    info = {"rounds": 0}
    for rnd in range(max_rounds):
        pairs = np.array(sorted(W), dtype=np.int64)
        A = _restricted_matrix(X, pairs, gamma)
        b = np.concatenate([-h, np.zeros(N * n)])
        th, _ = nnls(A, b, maxiter=50 * A.shape[1])
        y = h + A[:N] @ th
        xi = (A[N:] @ th).reshape(N, n) / np.sqrt(gamma)
        G = O.residual(y, xi, X)            # constraint values of every pair
        np.fill_diagonal(G, np.inf)
        viol = np.argwhere(G < -feas_tol * sigma)
        new = [tuple(map(int, v)) for v in viol if (int(v[0]), int(v[1])) not in W]
        info = {"rounds": rnd + 1, "pairs": len(W), "active": int((th > 0).sum()), "min_constraint": float(G.min()),
                "y_min": float(y.min())}
        if not new:
            break
        order = np.argsort([G[a, c] for a, c in new])[:add_per_round]
        W |= {new[i] for i in order}
    else:
        raise RuntimeError("constraint generation did not terminate")
    T = np.zeros((N, N))
    T[pairs[:, 0], pairs[:, 1]] = th
    info["complementarity"] = float(np.abs(T * np.where(np.isfinite(G), G, 0.0)).max())
    return y - s, xi, T, info
