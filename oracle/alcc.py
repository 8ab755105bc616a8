"""FP64 oracle of ALCC with the MAPG inner solver (Sec. II-D, Fig. `fig:alcc` and the MAPG
figure) on problem (regularize), every pairwise constraint kept in one block (the full problem).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` import this module; the CUDA path never does.

Plain dense numpy, one step of the paper per line group, no blocking or fusion:

* constraint values ``(A_1 y + A_2 xi)_p = y_l1 - y_l2 - xi_l2^T (x_l1 - x_l2)`` for every ordered
  pair p = (l1, l2), l1 != l2, held as an N x N matrix (row l1, column l2, diagonal unused);
* ``h_k(y, xi) = 1/2 ||(A_1 y + A_2 xi - theta_k)_-||^2`` and its gradients
  ``-A_1^T (.)_-``, ``-A_2^T (.)_-`` (Sec. II-D), with ``(z)_- = max(-z, 0)``;
* the block Lipschitz constants ``L^y_k = 1/mu_k + sigma_max^2(A_1)``,
  ``L^xi_k = gamma/mu_k + sigma_max^2(A_2)`` (Fig. `fig:alcc` step 1);
* MAPG (steps 1-10 of its figure) with projections on the balls Q_y, Q_xi;
* the ALCC outer update of theta, mu, tau and the alphas (Fig. `fig:alcc` steps 2-6).

Readings where the paper is silent (each also stated where it is used):

* Iteration 0 takes theta = 0; the first subproblem therefore uses theta_1 = 0.
* The feasible point behind the radii is (mean(ybar) 1, 0): every constant vector with zero
  subgradients satisfies all pairwise constraints, so Bbar = ||ybar - mean(ybar)||_2,
  Bbar_y = Bbar and Bbar_xi = Bbar / sqrt(gamma) (Sec. II-D).
* The start point is (y_0, xi_0) = (ybar, 0).
* mu_1, tau_1, alpha^y_1, alpha^xi_1, c and kappa have the defaults of ``AlccParams``.
* ALCC stops when the KKT residual of (regularize) at (y_k, xi_k) with the multiplier estimate
  lambda_k = mu_{k+1} theta_{k+1} = mu_k (A_1 y_k + A_2 xi_k - theta_k)_- is at most tol (see
  ``kkt``); the paper gives the complexity of ALCC but no stopping rule for it.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

__all__ = ["constraint_values", "adjoint", "sigma2_A1", "sigma2_A2", "radii", "proj_ball",
           "subproblem_value", "subproblem_grad", "mapg", "kkt", "AlccParams", "Alcc"]


def constraint_values(y, xi, X):
    """N x N matrix G, G[l1, l2] = y_l1 - y_l2 - xi_l2^T (x_l1 - x_l2) (problem (original));
    the diagonal is set to 0 and never used."""
    N = X.shape[0]
    G = np.empty((N, N))
    for l2 in range(N):
        G[:, l2] = y - y[l2] - (X - X[l2]) @ xi[l2]
    np.fill_diagonal(G, 0.0)
    return G


def adjoint(M, X):
    """(A_1^T m, A_2^T m) for multipliers m held as an N x N matrix (diagonal ignored).

    Row p = (l1, l2) of A_1 is e_l1 - e_l2, so (A_1^T m)_l = sum_l2 m[l, l2] - sum_l1 m[l1, l].
    Row p of A_2 holds -(x_l1 - x_l2)^T in block l2, so (A_2^T m)_l = -sum_l1 m[l1, l](x_l1 - x_l)."""
    M = M.copy()
    np.fill_diagonal(M, 0.0)
    a1 = M.sum(axis=1) - M.sum(axis=0)
    N, n = X.shape
    a2 = np.empty((N, n))
    for l in range(N):
        a2[l] = -(M[:, l] @ (X - X[l]))
    return a1, a2


def sigma2_A1(N: int) -> float:
    """sigma_max^2(A_1): A_1^T A_1 = 2 (N I - 1 1^T) over the ordered pairs, eigenvalues 2N and 0."""
    return 2.0 * N


def sigma2_A2(X) -> float:
    """sigma_max^2(A_2): A_2^T A_2 is block diagonal with blocks
    sum_l1 (x_l1 - x_l)(x_l1 - x_l)^T; the largest eigenvalue over the blocks."""
    best = 0.0
    for l in range(X.shape[0]):
        D = X - X[l]
        best = max(best, float(np.linalg.eigvalsh(D.T @ D)[-1]))
    return best


def radii(ybar, gamma: float):
    """(Bbar_y, Bbar_xi) from the feasible point (mean(ybar) 1, 0) (Sec. II-D)."""
    B = float(np.linalg.norm(ybar - ybar.mean()))
    return B, B / np.sqrt(gamma)


def proj_ball(z, center, r: float):
    """Euclidean projection on {z : ||z - center||_2 <= r}."""
    d = z - center
    nd = float(np.linalg.norm(d))
    return z.copy() if nd <= r else center + d * (r / nd)


def subproblem_value(y, xi, theta, ybar, gamma, mu, X):
    """P_k(y, xi) of Eq. (eq:subproblem)."""
    G = constraint_values(y, xi, X)
    m = np.maximum(theta - G, 0.0)
    np.fill_diagonal(m, 0.0)
    return (0.5 / mu) * np.sum((y - ybar) ** 2) + (0.5 * gamma / mu) * np.sum(xi ** 2) + 0.5 * np.sum(m ** 2)


def subproblem_grad(y, xi, theta, ybar, gamma, mu, X):
    """(grad_y P_k, grad_xi P_k): f/mu part plus -A^T (A_1 y + A_2 xi - theta)_- (Sec. II-D)."""
    G = constraint_values(y, xi, X)
    m = np.maximum(theta - G, 0.0)           # (G - theta)_-
    np.fill_diagonal(m, 0.0)
    a1, a2 = adjoint(m, X)
    return (y - ybar) / mu - a1, gamma * xi / mu - a2


def mapg(theta, ybar, gamma, mu, X, Ly, Lxi, y0, xi0, alpha_y, alpha_xi, lmax, By, Bxi):
    """MAPG (its figure) on P_k from (y0, xi0); returns (y, xi, iterations)."""
    y1p, xi1p = y0.copy(), xi0.copy()          # (y, xi)^(1)_{l-1}, Iteration 0: = (y0, xi0)
    y2, xi2 = y0.copy(), xi0.copy()            # (y, xi)^(2)_1
    t = 1.0
    zero = np.zeros_like(xi0)
    ell = 0
    while True:
        ell += 1
        gy, gxi = subproblem_grad(y2, xi2, theta, ybar, gamma, mu, X)
        y1 = proj_ball(y2 - gy / Ly, ybar, By)                       # step 1
        xi1 = proj_ball(xi2 - gxi / Lxi, zero, Bxi)                  # step 2
        tn = 0.5 * (1.0 + np.sqrt(1.0 + 4.0 * t * t))               # step 3
        w = (t - 1.0) / tn
        y2n = y1 + w * (y1 - y1p)                                    # step 4
        xi2n = xi1 + w * (xi1 - xi1p)                                # step 5
        dy = float(np.linalg.norm(y1 - y2))
        dxi = float(np.linalg.norm(xi1 - xi2))
        if (dy <= alpha_y and dxi <= alpha_xi) or ell >= lmax:       # steps 6-9
            return y1, xi1, ell
        y1p, xi1p, y2, xi2, t = y1, xi1, y2n, xi2n, tn


def kkt(y, xi, lam, ybar, gamma, X, sigma):
    """KKT residual of (regularize) at (y, xi) with multipliers lam (N x N, >= 0):
    stationarity y - ybar - A_1^T lam = 0 and gamma xi - A_2^T lam = 0, feasibility
    (A_1 y + A_2 xi)_- = 0 and complementarity lam_p (A_1 y + A_2 xi)_p = 0; each measured in the
    max norm and divided by the data scale sigma (sigma^2 for complementarity)."""
    G = constraint_values(y, xi, X)
    off = ~np.eye(X.shape[0], dtype=bool)
    a1, a2 = adjoint(lam, X)
    stat = max(float(np.abs(y - ybar - a1).max()), float(np.abs(gamma * xi - a2).max())) / sigma
    pri = float(np.maximum(-G[off], 0.0).max()) / sigma
    comp = float(np.abs(lam[off] * G[off]).max()) / (sigma * sigma)
    return {"kkt": max(stat, pri, comp), "stat": stat, "pri": pri, "comp": comp}


@dataclass
class AlccParams:
    """Inputs of ALCC the paper leaves to the user (Fig. `fig:alcc`): mu_1 = mu1_scale / sigma_max^2(A_1),
    tau_1 = tau1_rel * Bbar^2 / mu_1, alpha^y_1 = alpha1_rel * Bbar_y, alpha^xi_1 = alpha1_rel * Bbar_xi,
    c > 1, kappa > 0."""
    mu1_scale: float = 1e3
    tau1_rel: float = 1e-2
    alpha1_rel: float = 1e-2
    c: float = 2.0
    kappa: float = 0.1
    lmax_cap: int = 1 << 62          # optional bound on MAPG iterations per call (none in the paper)
    fixed_inner: int = 0             # > 0: every MAPG call runs exactly this many iterations
    mu_max_scale: float = 0.0        # NOT IN THE PAPER: > 0 caps mu_k at mu_max_scale / sigma_max^2(A_1)


@dataclass
class Alcc:
    """ALCC (Fig. `fig:alcc`) with MAPG; state after k outer iterations."""
    X: np.ndarray
    ybar: np.ndarray
    gamma: float
    prm: AlccParams = field(default_factory=AlccParams)

    def __post_init__(self):
        X = np.ascontiguousarray(self.X, dtype=np.float64)
        self.X = X.reshape(X.shape[0], -1)
        self.ybar = np.asarray(self.ybar, dtype=np.float64)
        N, n = self.X.shape
        self.s2a1 = sigma2_A1(N)
        self.s2a2 = sigma2_A2(self.X)
        self.By, self.Bxi = radii(self.ybar, self.gamma)
        self.sigma = max(1.0, float(np.ptp(self.ybar)))
        self.y = self.ybar.copy()                   # (y_0, xi_0)
        self.xi = np.zeros((N, n))
        self.theta = np.zeros((N, N))               # theta_1 (Iteration 0 takes theta = 0)
        self.mu = self.prm.mu1_scale / self.s2a1    # mu_1
        self.tau = self.prm.tau1_rel * self.By ** 2 / self.mu
        self.alpha_y = self.prm.alpha1_rel * self.By
        self.alpha_xi = self.prm.alpha1_rel * self.Bxi
        self.k = 1
        self.inner = []                             # MAPG iterations of every outer iteration
        self.metrics = None

    def lmax(self) -> int:
        """Fig. `fig:alcc` steps 1-2 at the current k."""
        Ly = 1.0 / self.mu + self.s2a1
        Lxi = self.gamma / self.mu + self.s2a2
        v = 4.0 * np.sqrt((Ly * self.By ** 2 + Lxi * self.Bxi ** 2) / self.tau)
        return int(min(max(1.0, np.ceil(v)), float(self.prm.lmax_cap)))

    def outer(self):
        """One ALCC iteration k (steps 1-6); returns the KKT metrics at (y_k, xi_k)."""
        p = self.prm
        Ly = 1.0 / self.mu + self.s2a1                                  # step 1
        Lxi = self.gamma / self.mu + self.s2a2
        lmax = p.fixed_inner if p.fixed_inner > 0 else self.lmax()      # step 2
        ay, axi = (0.0, 0.0) if p.fixed_inner > 0 else (self.alpha_y, self.alpha_xi)
        y, xi, it = mapg(self.theta, self.ybar, self.gamma, self.mu, self.X, Ly, Lxi, self.y, self.xi,
                         ay, axi, lmax, self.By, self.Bxi)             # step 3
        self.inner.append(it)
        G = constraint_values(y, xi, self.X)
        m = np.maximum(self.theta - G, 0.0)                             # (A_1 y + A_2 xi - theta_k)_-
        np.fill_diagonal(m, 0.0)
        mu_next = p.c * self.mu                                         # step 5
        if p.mu_max_scale > 0.0:                                        # optional cap (not in the paper)
            mu_next = min(mu_next, max(self.mu, p.mu_max_scale / self.s2a1))
        self.theta = (self.mu / mu_next) * m                            # step 4
        lam = mu_next * self.theta                                      # multiplier estimate
        shrink = (p.c * float(self.k) ** (1.0 + p.kappa)) ** 2
        self.tau /= shrink
        self.alpha_y /= shrink                                          # step 6
        self.alpha_xi /= shrink
        self.mu = mu_next
        self.y, self.xi = y, xi
        self.k += 1
        self.metrics = kkt(y, xi, lam, self.ybar, self.gamma, self.X, self.sigma)
        return self.metrics

    def solve(self, tol: float, max_outer: int) -> bool:
        for _ in range(max_outer):
            if self.outer()["kkt"] <= tol:
                return True
        return False
