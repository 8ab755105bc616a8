"""FP64 oracle of P-APG (Fig. 2) with the data partitioned into K blocks (Sec. II-A).

TEST INFRASTRUCTURE ONLY.  Only ``tests/`` imports this module; the CUDA path never does.

The points are split into blocks C_1..C_K.  The pairwise constraints of problem (original)
inside a block stay in that block's Step-1 problem; the constraints between blocks and the
y >= 0 rows of C (Eq. (eq:C)) are dualized with multipliers theta >= 0, mu >= 0, and P-APG runs on
that dual.  With v = A_1^T theta + mu and w = A_2^T theta (sums over the dualized rows only),
Step 1 separates into one problem per block,

    min  1/2 ||y_i - (h_i + v_i)||^2 + gamma/2 ||xi_i - w_i / gamma||^2
    s.t. y_l1 - y_l2 - xi_l2^T (x_l1 - x_l2) >= 0 for l1 != l2 in block i,

the projection of the closed-form point (h + v, w/gamma) onto the block's constraint set in the
norm weighted by diag(1, gamma).  The oracle solves it exactly through its dual, a nonnegative
least-squares problem (scipy's active-set Lawson-Hanson NNLS), or -- with ``inner_iters`` set --
inexactly, as the paper's block solvers do: ``inner_iters`` iterations of P-APG (Fig. 2) on each
block problem's dual (every pair inside the block dualized: the closed form y = a + A_1b^T lam,
xi = b + A_2b^T lam / gamma, the clamp of lam - (constraint values) / L_in, the t-sequence from
t = 1), started at the previous call's multipliers lam.  Step 2 is the projected step on
the dualized rows, Steps 3-4 the momentum of Fig. 2.  With singleton blocks (K = N) this is the
P-APG of ``oracle.py``; with one block (K = 1) Step 1 is the whole problem.

Dense matrices, small N only.
"""
from __future__ import annotations

import numpy as np
from scipy.optimize import nnls

__all__ = ["pair_rows", "BlockPapg"]


def pair_rows(X, pairs):
    """Rows of A_1 (len(pairs) x N) and A_2 (len(pairs) x N n) for the given ordered pairs:
    e_l1 - e_l2 and -(x_l1 - x_l2)^T in the columns of block l2 (problem (original))."""
    N, n = X.shape
    A1 = np.zeros((len(pairs), N))
    A2 = np.zeros((len(pairs), N * n))
    for p, (l1, l2) in enumerate(pairs):
        A1[p, l1] = 1.0
        A1[p, l2] = -1.0
        A2[p, l2 * n:(l2 + 1) * n] = -(X[l1] - X[l2])
    return A1, A2


class BlockPapg:
    """P-APG (Fig. 2) on the dual of the constraints between blocks and of the y >= 0 rows."""

    def __init__(self, X, ybar, blocks, gamma: float, L: float, s: float, inner_iters=None, L_inner=None):
        self.X = np.ascontiguousarray(X, dtype=np.float64)
        N, n = self.X.shape
        self.N, self.n, self.gamma, self.L = N, n, float(gamma), float(L)
        self.h = np.asarray(ybar, dtype=np.float64) + s
        self.s = float(s)
        self.blocks = [np.asarray(b, dtype=np.int64) for b in blocks]
        owner = np.empty(N, dtype=np.int64)
        for i, b in enumerate(self.blocks):
            owner[b] = i
        assert sorted(np.concatenate(self.blocks).tolist()) == list(range(N)), "blocks must partition the points"
        self.cross = [(l1, l2) for l1 in range(N) for l2 in range(N) if l1 != l2 and owner[l1] != owner[l2]]
        self.A1c, self.A2c = pair_rows(self.X, self.cross)
        # intra-block constraint rows, per block, in the block's local coordinates
        self.intra = []
        for b in self.blocks:
            loc = [(i, j) for i in range(len(b)) for j in range(len(b)) if i != j]
            A1b, A2b = pair_rows(self.X[b], loc)
            self.intra.append((A1b, A2b))
        self.inner_iters = None if inner_iters is None else int(inner_iters)
        self.L_inner = float(L if L_inner is None else L_inner)
        self.lam = [np.zeros(A1b.shape[0]) for A1b, _ in self.intra]   # inner multipliers (warm start)
        m = len(self.cross)
        # Iteration 0 of Fig. 2: theta^(1)_0 = theta^(2)_1 = 0, t_1 = 1
        self.th1p = np.zeros(m)         # theta^(1)_{l-1}
        self.th2 = np.zeros(m)          # theta^(2)_l
        self.mu1p = np.zeros(N)
        self.mu2 = np.zeros(N)
        self.t = 1.0
        self.iters = 0
        if self.inner_iters is None:
            self.y, self.xi = self.step1(self.th2, self.mu2)
        else:   # the inexact Step 1 moves its warm start: it runs only inside iterate()
            self.y, self.xi = self.h.copy(), np.zeros((N, n))

    def step1(self, theta, mu):
        """Step 1: eta(theta, mu), block by block (exact NNLS on each block's dual)."""
        N, n, g = self.N, self.n, self.gamma
        v = self.A1c.T @ theta + mu
        w = (self.A2c.T @ theta).reshape(N, n)
        y0 = self.h + v                  # unconstrained minimizer
        xi0 = w / g
        y = np.empty(N)
        xi = np.empty((N, n))
        for i, (b, (A1b, A2b)) in enumerate(zip(self.blocks, self.intra)):
            yb0, xb0 = y0[b], xi0[b].ravel()
            if A1b.shape[0] == 0:        # a single point: no constraint inside
                y[b], xi[b] = yb0, xb0.reshape(-1, n)
                continue
            if self.inner_iters is not None:
                y[b], xi[b] = self._inner_papg(i, A1b, A2b, yb0, xb0)
                continue
            # min_{lambda >= 0} 1/2 || [A1b^T ; A2b^T / sqrt(g)] lambda + [yb0 ; sqrt(g) xb0] ||^2
            M = np.vstack([A1b.T, A2b.T / np.sqrt(g)])
            rhs = -np.concatenate([yb0, np.sqrt(g) * xb0])
            lam, _ = nnls(M, rhs, maxiter=50 * M.shape[1])
            y[b] = yb0 + A1b.T @ lam
            xi[b] = (xb0 + (A2b.T @ lam) / g).reshape(-1, n)
        return y, xi

    def _inner_papg(self, i, A1b, A2b, a, b):
        """inner_iters iterations of P-APG (Fig. 2) on block i's dual from its last multipliers."""
        g, Lin = self.gamma, self.L_inner
        lam1 = self.lam[i]            # lambda^(1) of the last call
        lam2 = lam1.copy()            # Iteration 0 at lam1: lambda^(2)_1 = lambda^(1)_0
        lamp = lam1
        t = 1.0
        for _ in range(self.inner_iters):
            y = a + A1b.T @ lam2                                   # Step 1 (closed form)
            xi = b + (A2b.T @ lam2) / g
            gc = A1b @ y + A2b @ xi                                # the constraint values
            l1 = np.maximum(0.0, lam2 - gc / Lin)                  # Step 2
            tn = 0.5 * (1.0 + np.sqrt(1.0 + 4.0 * t * t))         # Step 3
            beta = (t - 1.0) / tn
            lam2 = l1 + beta * (l1 - lamp)                         # Step 4
            lamp, t = l1, tn
        self.lam[i] = lamp
        return a + A1b.T @ lamp, (b + (A2b.T @ lamp) / g).reshape(-1, self.n)

    def iterate(self, k: int):
        N, n = self.N, self.n
        for _ in range(k):
            y, xi = self.step1(self.th2, self.mu2)                        # Step 1 at theta^(2)_l
            gc = self.A1c @ y + self.A2c @ xi.ravel()                      # (C eta)_p on the cross rows
            th1 = np.maximum(0.0, self.th2 - gc / self.L)                  # Step 2
            mu1 = np.maximum(0.0, self.mu2 - y / self.L)                   # Step 2 on the y >= 0 rows
            tn = 0.5 * (1.0 + np.sqrt(1.0 + 4.0 * self.t * self.t))       # Step 3
            beta = (self.t - 1.0) / tn
            self.th2 = th1 + beta * (th1 - self.th1p)                      # Step 4
            self.mu2 = mu1 + beta * (mu1 - self.mu1p)
            self.th1p, self.mu1p, self.t = th1, mu1, tn
            self.iters += 1
        # the primal point at the dual iterate theta^(1)_l
        self.y, self.xi = self.step1(self.th1p, self.mu1p)

    @property
    def y_hat(self):
        return self.y - self.s

    def theta_matrix(self):
        """theta^(1)_l as an N x N matrix (zero on the intra-block pairs and the diagonal)."""
        T = np.zeros((self.N, self.N))
        for v, (l1, l2) in zip(self.th1p, self.cross):
            T[l1, l2] = v
        return T
