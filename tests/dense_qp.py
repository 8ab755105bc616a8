"""Dense, explicit-matrix reference constructions for tiny instances.

Used to pin the oracle to something other than itself.  The constraint
matrices are built row by row from problem (original) of the paper:
for every ordered pair (l1, l2), l1 != l2,

    y_{l1} - y_{l2} - xi_{l2}^T (x_{l1} - x_{l2}) >= 0,

i.e. row p of A_1 is e_{l1} - e_{l2} and row p of A_2 holds
-(x_{l1} - x_{l2})^T in the n columns of block l2 (compact form
(original_compact)).  C of Eq. (eq:C) at K = N appends the identity rows
(y >= 0).  The regularized problem (regularize) is then solved exactly by
its dual, a nonnegative least-squares problem, with scipy's Lawson-Hanson
NNLS -- an active-set method that terminates in finitely many steps, so its
answer does not depend on any iteration count.
"""
from __future__ import annotations

import numpy as np


def pair_list(N: int):
    return [(l1, l2) for l1 in range(N) for l2 in range(N) if l1 != l2]


def constraint_matrices(X: np.ndarray):
    """A_1 (P x N), A_2 (P x N n) in the row order of ``pair_list``."""
    N, n = X.shape
    pairs = pair_list(N)
    P = len(pairs)
    A1 = np.zeros((P, N))
    A2 = np.zeros((P, N * n))
    for p, (l1, l2) in enumerate(pairs):
        A1[p, l1] = 1.0
        A1[p, l2] = -1.0
        A2[p, l2 * n:(l2 + 1) * n] = -(X[l1] - X[l2])
    return A1, A2, pairs


def big_C(X: np.ndarray):
    """C = [A_1 A_2; I 0] of Eq. (eq:C) with every pair dualized (K = N)."""
    N, n = X.shape
    A1, A2, pairs = constraint_matrices(X)
    top = np.hstack([A1, A2])
    bot = np.hstack([np.eye(N), np.zeros((N, N * n))])
    return np.vstack([top, bot]), pairs


def theta_vec(theta_mat: np.ndarray, pairs):
    return np.array([theta_mat[l1, l2] for (l1, l2) in pairs])


def theta_mat(theta: np.ndarray, pairs, N: int):
    T = np.zeros((N, N))
    for v, (l1, l2) in zip(theta, pairs):
        T[l1, l2] = v
    return T


def solve_regularized_nnls(X: np.ndarray, h: np.ndarray, gamma: float):
    """Exact solution of (regularize) without the y >= 0 rows, via its dual.

    Lagrangian 1/2||y-h||^2 + gamma/2||xi||^2 - theta^T (A_1 y + A_2 xi) gives
    y = h + A_1^T theta, xi = A_2^T theta / gamma, and the dual is
        min_{theta >= 0} 1/2 || [A_1^T; A_2^T/sqrt(gamma)] theta + [h; 0] ||^2 .
    Returns (y, xi (N x n), theta_matrix (N x N), dual value)."""
    from scipy.optimize import nnls

    N, n = X.shape
    A1, A2, pairs = constraint_matrices(X)
    A = np.vstack([A1.T, A2.T / np.sqrt(gamma)])
    b = np.concatenate([-h, np.zeros(N * n)])
    theta, _ = nnls(A, b, maxiter=50 * A.shape[1])
    y = h + A1.T @ theta
    xi = (A2.T @ theta) / gamma
    dual = -0.5 * np.sum((A1.T @ theta) ** 2) - theta @ (A1 @ h) - 0.5 / gamma * np.sum((A2.T @ theta) ** 2)
    return y, xi.reshape(N, n), theta_mat(theta, pairs, N), dual


def dense_dual(X, h, gamma, T, mu):
    """g_gamma(theta) of Eq. (eq:g_gamma) evaluated through the explicit matrices."""
    N, n = X.shape
    C, pairs = big_C(X)
    th = np.concatenate([theta_vec(T, pairs), mu])
    Hinv = np.concatenate([np.ones(N), np.full(N * n, 1.0 / gamma)])
    htil = np.concatenate([h, np.zeros(N * n)])
    eta = Hinv * (htil + C.T @ th)
    y, xi = eta[:N], eta[N:]
    return 0.5 * np.sum((y - h) ** 2) + 0.5 * gamma * np.sum(xi ** 2) - th @ (C @ eta), eta
