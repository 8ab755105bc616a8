"""P-APG with the points partitioned into K blocks (Sec. II-A, Fig. 2) on the GPU (cr_blocks_*)
against the FP64 block oracle (oracle/papg_blocks.py) taking the same inexact Step 1: the same
number of inner P-APG iterations on the block problems' duals, warm-started, momentum restarted.
FP64 on both sides: the bars are FP64 summation-order bars."""
import numpy as np
import pytest

from oracle import oracle as O
from oracle.papg_blocks import BlockPapg
from paper_1407_7220_gb300 import datagen

pytestmark = pytest.mark.gpu


def _rel(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def _blocks(N, K):
    return [np.arange(i, N, K) for i in range(K)]   # interleaved partition, as equal as possible


# K = 2, 4, and N / 100 (N = 200: K = 2; N = 900: K = 9, several stripes, so that the inner pass
# visits only the rows of each stripe's blocks), ragged blocks (96 / 3 with n = 5)
@pytest.mark.parametrize("N,n,K,M,outer", [(120, 2, 2, 40, 15), (200, 2, 4, 20, 12), (200, 3, 2, 30, 10),
                                           (96, 5, 3, 16, 8), (900, 2, 9, 10, 5)])
def test_block_papg_trajectory_matches_oracle(N, n, K, M, outer):
    import paper_1407_7220_gb300 as crg
    X, yb, _ = datagen.make("sq2" if n < 5 else "sumexp", N=N, n=n)
    bl = _blocks(N, K)
    g = crg.BlockSolver(X, yb, bl, inner_iters=M, gamma=0.1)
    o = BlockPapg(X, yb, bl, 0.1, O.lipschitz(X, 0.1), O.shift(yb), inner_iters=M)
    for k in (1, outer):
        g.iterate(k - g.info()["iters"])
        o.iterate(k - o.iters)
        y, xi = g.solution()
        assert g.info()["iters"] == k
        assert _rel(y, o.y_hat) <= 1e-11, _rel(y, o.y_hat)
        np.testing.assert_allclose(xi, o.xi, rtol=0, atol=1e-9 * max(1.0, np.abs(o.xi).max()))


def test_singleton_blocks_are_the_every_pair_papg():
    # K = N: no constraint inside any block, Step 1 is the closed form of cr_create's P-APG
    import paper_1407_7220_gb300 as crg
    X, yb, _ = datagen.make("sq2", N=150)
    g = crg.BlockSolver(X, yb, np.arange(150), inner_iters=2, gamma=0.1)
    s = crg.Solver(X, yb, gamma=0.1, theta_dtype="f64", restart=0)
    g.iterate(25)
    s.iterate(25)
    assert _rel(g.solution()[0], s.solution()[0]) <= 1e-12


def test_block_papg_converges_to_the_exact_solution():
    from oracle import exact as E
    import paper_1407_7220_gb300 as crg
    X, yb, _ = datagen.make("sq2", N=100, seed=31)
    y_ex, _, _, _ = E.solve(X, yb, 0.1)
    g = crg.BlockSolver(X, yb, _blocks(100, 2), inner_iters=60, gamma=0.1)
    g.iterate(3000)
    err = _rel(g.solution()[0], y_ex)
    print(f"K = 2, 3000 outer x 60 inner iterations: fit {err:.2e} from the exact solution")
    assert err <= 1e-3


def test_block_solver_rejects_bad_arguments():
    import paper_1407_7220_gb300 as crg
    X, yb, _ = datagen.make("sq2", N=40)
    for bad in (dict(inner_iters=3), dict(inner_iters=0)):
        with pytest.raises(crg.CrError):
            crg.BlockSolver(X, yb, _blocks(40, 2), gamma=0.1, **bad)
    g = crg.BlockSolver(X, yb, _blocks(40, 2), inner_iters=4, gamma=0.1)
    assert crg.lib().cr_iterate(g.handle, 1) == crg.CR_ESTATE
    assert crg.lib().cr_reset(g.handle) == crg.CR_ESTATE
    # the handles hold the points sorted by block: the fit comes from cr_blocks_solution only
    assert crg.lib().cr_get_solution(g.handle, None, None) == crg.CR_ESTATE
    assert crg.lib().cr_get_solution_device(g.handle, None, None) == crg.CR_ESTATE
