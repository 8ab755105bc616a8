"""Batched persistent solve (many independent fits in one launch) against single
instances and the FP64 oracle, through the C ABI."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1407_7220_gb300 import datagen

pytestmark = pytest.mark.gpu


def _rel(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def _instances(sizes, seed=5):
    rng = np.random.default_rng(seed)
    out = []
    for N, n in sizes:
        X = rng.normal(size=(N, n))
        yb = (X ** 2).sum(1) + np.abs(X[:, 0]) + rng.normal(0, 0.1, size=N)   # recipe (4) shape
        out.append((X, yb))
    return out


SIZES = [(20, 1), (97, 2), (300, 5), (513, 2), (64, 1), (1000, 5), (257, 5)]


@pytest.mark.parametrize("grid", [0, 1, 4])
def test_batch_trajectories_match_single_instances_and_oracle(grid):
    import paper_1407_7220_gb300 as crg
    inst = _instances(SIZES)
    bs = crg.BatchSolver(inst, gamma=0.1, stochastic_round=0, restart=0, grid=grid)
    bs.iterate(30)
    for i, (X, yb) in enumerate(inst):
        m = bs.member(i)
        y, xi = m.solution()
        assert m.info()["iters"] == 30
        s = crg.Solver(X, yb, gamma=0.1, stochastic_round=0, restart=0)
        s.iterate(30)
        ys, xs = s.solution()
        assert _rel(y, ys) <= 1e-6          # same algorithm, other partition (summation order)
        o = O.Solver(X, yb, gamma=0.1, restart=False)   # the oracle's own L_g and shift
        o.iterate(30)
        assert _rel(y, o.y_hat) <= 1e-6
        assert np.abs(xi - o.xi).max() <= 2e-4 * max(1.0, np.abs(o.xi).max())


def test_batch_solve_reaches_tolerance_per_instance():
    import paper_1407_7220_gb300 as crg
    inst = _instances([(40, 1), (80, 2), (120, 2), (60, 5), (150, 1)], seed=9)
    bs = crg.BatchSolver(inst, gamma=0.1, kkt_every=10)   # plain P-APG (no restart)
    conv = bs.solve(1e-4, 200000)
    assert conv == len(inst)
    iters = []
    for i in range(len(inst)):
        m = bs.member(i)
        k = m.kkt_residual()
        assert k["kkt"] <= 1e-4
        iters.append(m.info()["iters"])
    # members stop at their own iteration counts
    assert len(set(iters)) > 1
    # and each converged fit is the oracle's fit to the KKT-driven accuracy
    X, yb = inst[0]
    o = O.Solver(X, yb, gamma=0.1, restart=True)
    o.solve(1e-10, 2_000_000, check_every=50)
    assert _rel(bs.member(0).solution()[0], o.y_hat) <= 5e-4


def test_batch_runs_from_its_cuda_graph_and_autotunes():
    # the persistent launch is captured once in a CUDA graph and replayed chunk after chunk;
    # the autotuner timed every granularity candidate
    import paper_1407_7220_gb300 as crg
    inst = _instances(SIZES, seed=3)
    bs = crg.BatchSolver(inst, gamma=0.1, stochastic_round=0, restart=0)
    bs.iterate(40)
    bs.iterate(40)
    st = bs.stats()
    print(st)
    assert st["graph_live"] and st["graph_launches"] >= 2 and st["direct_launches"] == 0
    assert st["tuned"] == 10 and len(st["tune_ms"]) == 8 and min(st["tune_ms"]) > 0.0


def test_batch_tile_shapes_give_the_same_trajectories():
    # 8-row and 16-row stages visit the same pairs and add every row and column partial in the
    # same order, so the batched trajectories agree bit for bit
    import paper_1407_7220_gb300 as crg
    inst = _instances(SIZES, seed=11)
    fits = {}
    for rows in (16, 8):
        bs = crg.BatchSolver(inst, gamma=0.1, stochastic_round=1, restart=0, grid=2, batch_stage_rows=rows)
        assert bs.tuning()["stage_rows"] == rows
        bs.iterate(25)
        fits[rows] = [bs.member(i).solution()[0] for i in range(len(inst))]
        bs.close()
    for a, b in zip(fits[16], fits[8]):
        assert np.array_equal(a, b)


def test_batch_autotuner_times_tile_shapes_and_granularities():
    import paper_1407_7220_gb300 as crg
    inst = _instances(SIZES, seed=3)
    bs = crg.BatchSolver(inst, gamma=0.1, stochastic_round=0, restart=0)
    t = bs.tuning()
    print(t)
    cands = t["candidates"]
    assert len(cands) == 10
    assert {c["stage_rows"] for c in cands} == {8, 16}
    assert {c["factor"] for c in cands} == {1, 2, 4, 8, 16}
    best = min(cands, key=lambda c: c["ms"])
    assert (t["stage_rows"], t["factor"]) == (best["stage_rows"], best["factor"])
    with pytest.raises(crg.CrError):
        crg.BatchSolver(inst, gamma=0.1, batch_stage_rows=12)
