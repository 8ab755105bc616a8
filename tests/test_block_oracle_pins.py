"""Pins of the K-block P-APG oracle (Sec. II-A, Fig. 2; ``oracle/papg_blocks.py``).

References: the K = N P-APG of the C oracle (an independent implementation: closed-form Step 1,
C loops), its converged fit, and the explicit constraint rows of problem (original).  CPU only.
"""
import numpy as np
import pytest

from oracle import oracle as O
from oracle.papg_blocks import BlockPapg, pair_rows
from paper_1407_7220_gb300 import datagen


def _inst(N, n=2, seed=5):
    X, yb, _ = datagen.make("sq2", N=N, n=n, seed=seed)
    return X, yb


def _blocks(N, K):
    return [np.arange(i, N, K) for i in range(K)]   # interleaved, as equal as possible


def test_singleton_blocks_reproduce_the_K_equals_N_trajectory():
    X, yb = _inst(14)
    g, L, s = 0.1, O.lipschitz(X, 0.1), O.shift(yb)
    b = BlockPapg(X, yb, [[l] for l in range(14)], g, L, s)
    o = O.Solver(X, yb, gamma=g, L=L, s=s, momentum=True, restart=False)
    for k in (1, 4, 30):
        b.iterate(k - b.iters)
        o.iterate(k - o.iters)
        np.testing.assert_allclose(b.y_hat, o.y_hat, rtol=0, atol=1e-11 * np.abs(o.y_hat).max())
        np.testing.assert_allclose(b.theta_matrix(), o.theta1, rtol=0, atol=1e-11 * max(1.0, np.abs(o.theta1).max()))


@pytest.fixture(scope="module")
def converged():
    X, yb = _inst(16)
    o = O.Solver(X, yb, gamma=0.1, restart=True)
    o.solve(1e-11, 3_000_000, check_every=100)
    assert o.metrics["kkt"] <= 1e-11
    return X, yb, o.y_hat, o.xi


def test_one_block_is_the_whole_problem(converged):
    X, yb, y_ref, xi_ref = converged
    b = BlockPapg(X, yb, [np.arange(16)], 0.1, O.lipschitz(X, 0.1), O.shift(yb))
    assert len(b.cross) == 0
    # Step 1 at Iteration 0 already solves (regularize); the y >= 0 rows stay inactive
    np.testing.assert_allclose(b.y_hat, y_ref, rtol=0, atol=1e-8 * np.abs(y_ref).max())
    b.iterate(5)
    assert b.mu1p.max() == 0.0
    np.testing.assert_allclose(b.y_hat, y_ref, rtol=0, atol=1e-8 * np.abs(y_ref).max())
    np.testing.assert_allclose(b.xi, xi_ref, rtol=0, atol=1e-6 * max(1.0, np.abs(xi_ref).max()))


@pytest.mark.parametrize("K", [2, 4])
def test_block_papg_converges_to_the_solution(converged, K):
    X, yb, y_ref, _ = converged
    b = BlockPapg(X, yb, _blocks(16, K), 0.1, O.lipschitz(X, 0.1), O.shift(yb))
    b.iterate(3000)
    assert np.abs(b.y_hat - y_ref).max() <= 1e-4 * np.abs(y_ref).max()


def test_step1_blocks_are_feasible_and_multipliers_live_on_cross_pairs():
    X, yb = _inst(12)
    blocks = _blocks(12, 3)
    b = BlockPapg(X, yb, blocks, 0.1, O.lipschitz(X, 0.1), O.shift(yb))
    b.iterate(40)
    for blk in blocks:
        loc = [(int(i), int(j)) for i in blk for j in blk if i != j]
        A1, A2 = pair_rows(X, loc)
        gval = A1 @ b.y + A2 @ b.xi.ravel()
        assert gval.min() >= -1e-9 * max(1.0, np.abs(b.y).max())   # intra-block constraints hold exactly
    T = b.theta_matrix()
    assert T.min() >= 0.0
    for blk in blocks:
        assert np.all(T[np.ix_(blk, blk)] == 0.0)


def test_fewer_blocks_start_closer():
    # Step 1 with intra-block constraints kept is exact on more of the problem: after one
    # iteration the fit of K = 2 is closer to the solution than that of K = N
    X, yb = _inst(16)
    o = O.Solver(X, yb, gamma=0.1, restart=True)
    o.solve(1e-10, 3_000_000, check_every=100)
    L, s = O.lipschitz(X, 0.1), O.shift(yb)
    e = {}
    for K in (2, 16):
        b = BlockPapg(X, yb, _blocks(16, K), 0.1, L, s)
        b.iterate(1)
        e[K] = np.abs(b.y_hat - o.y_hat).max()
    assert e[2] < e[16]


def test_inexact_step1_tends_to_the_exact_one():
    # the inner P-APG on the block problems' duals (the inexact Step 1) approaches the exact NNLS
    # Step 1 as its iteration count grows; singleton blocks have no inner constraints at all
    X, yb = _inst(30)
    g, L, s = 0.1, O.lipschitz(X, 0.1), O.shift(yb)
    bl = _blocks(30, 2)
    ex = BlockPapg(X, yb, bl, g, L, s)
    ex.iterate(4)
    errs = []
    for M in (50, 500, 6000):
        inx = BlockPapg(X, yb, bl, g, L, s, inner_iters=M)
        inx.iterate(4)
        errs.append(np.abs(inx.y_hat - ex.y_hat).max() / np.abs(ex.y_hat).max())
    assert errs[2] <= 1e-6 and errs[2] < errs[1] < errs[0]
    one = BlockPapg(X, yb, [[l] for l in range(30)], g, L, s, inner_iters=4)
    o = O.Solver(X, yb, gamma=g, L=L, s=s, momentum=True, restart=False)
    one.iterate(10)
    o.iterate(10)
    np.testing.assert_allclose(one.y_hat, o.y_hat, rtol=0, atol=1e-11 * np.abs(o.y_hat).max())
