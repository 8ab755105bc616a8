"""ALCC with the MAPG inner solver on the full problem (Sec. II-D) through the C ABI.

Reference: the FP64 oracle ``oracle/alcc.py`` (pinned in ``tests/test_alcc_oracle_pins.py``) on
the same seeded inputs.  With a fixed number of MAPG iterations per outer iteration both sides
take the same steps, so the iterates are compared element by element: the GPU's pair pass is
FP32 (one rounding per residual and compensated FP32 partial sums), its folds FP64, which keeps
the fitted values within 1e-6 relative and the multiplier array within 1e-6 of the data scale
(the FP32 rounding of the residuals it is formed from); the KKT terms agree within 1e-3
relative.  With the paper's stopping rule the inner counts of the first outer iterations match
the oracle's; converged runs are compared with the exact solution of (regularize).
"""
import numpy as np
import pytest

from oracle import alcc as A
from paper_1407_7220_gb300 import datagen
from tests import dense_qp as D

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def crg():
    import paper_1407_7220_gb300 as m
    return m


def _rel(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


class _DevArray:
    """A device buffer described by __cuda_array_interface__ (read through torch without a copy)."""

    def __init__(self, ptr, shape, typestr):
        self.__cuda_array_interface__ = {"shape": shape, "typestr": typestr, "data": (ptr, False), "version": 2,
                                         "strides": None}


def _theta(s):
    import torch
    ds = s.device_state()
    t = torch.as_tensor(_DevArray(ds["theta"], (s.N, ds["ld"]), "<f4"), device="cuda")
    torch.cuda.synchronize()
    return t[:, :s.N].double().cpu().numpy()


@pytest.mark.parametrize("N,n,recipe", [(97, 2, "sq2"), (300, 5, "sumexp"), (517, 1, "sq2"), (260, 10, "maxaff"),
                                        (33, 32, "lse")])
def test_trajectory_matches_oracle(crg, N, n, recipe):
    X, yb, _ = datagen.make(recipe, N=N, n=n)
    g = crg.AlccSolver(X, yb, gamma=0.1, fixed_inner=15)
    o = A.Alcc(X, yb, 0.1, A.AlccParams(fixed_inner=15))
    for _ in range(3):
        assert g.iterate(1) == [15]
        o.outer()
        y, xi = g.solution()
        assert _rel(y, o.y) <= 1e-6, _rel(y, o.y)
        assert np.abs(xi - o.xi).max() <= 1e-6 * max(1.0, np.abs(o.xi).max())
        th = _theta(g)
        # theta_{k+1} = a (g - theta_k)_-: the FP32 rounding of g (of the size of y) sets the bar
        assert np.abs(th - o.theta).max() <= 1e-6 * max(1.0, np.abs(yb).max())
        assert np.all(np.diag(th) == 0.0) and th.min() >= 0.0
        m = g.metrics()
        # stationarity subtracts mu_{k+1} A^T theta_{k+1} (FP32 partial sums) from the FP64 point
        for key in ("kkt", "stat", "pri", "comp"):
            assert m[key] == pytest.approx(o.metrics[key], rel=1e-3, abs=1e-9), key
    info = g.info()
    assert info["outer"] == 3 and info["inner_total"] == 45
    assert info["mu"] == pytest.approx(o.mu, rel=1e-14)


def test_stopping_rule_gives_the_oracle_inner_counts(crg):
    # MAPG steps 6-9 with the schedule of Fig. `fig:alcc` steps 2, 5-6: the first outer
    # iterations stop on the alpha test long before the FP32 floor matters
    X, yb, _ = datagen.make("sq2", N=97, n=2)
    g = crg.AlccSolver(X, yb, gamma=0.1)
    o = A.Alcc(X, yb, 0.1)
    gi = g.iterate(4)
    for _ in range(4):
        o.outer()
    assert gi == o.inner, (gi, o.inner)
    assert g.info()["lmax_next"] == o.lmax()
    assert _rel(g.solution()[0], o.y) <= 1e-5


def test_launch_boundaries_do_not_change_the_iterates(crg):
    X, yb, _ = datagen.make("sq2", N=300, n=2)
    r = []
    for li in (1, 7, 0):
        s = crg.AlccSolver(X, yb, gamma=0.1, launch_iters=li)
        inner = s.iterate(3)
        r.append((inner, *s.solution()))
    for inner, y, xi in r[1:]:
        assert inner == r[0][0]
        assert np.array_equal(y, r[0][1]) and np.array_equal(xi, r[0][2])


@pytest.mark.parametrize("grid", [1, 3, 40])
def test_grid_partitions_give_the_same_iterates(crg, grid):
    X, yb, _ = datagen.make("sumexp", N=530, n=5)
    ref = crg.AlccSolver(X, yb, gamma=0.1, fixed_inner=10)
    s = crg.AlccSolver(X, yb, gamma=0.1, fixed_inner=10, grid=grid)
    ref.iterate(2)
    s.iterate(2)
    assert _rel(s.solution()[0], ref.solution()[0]) <= 1e-6


def test_converges_to_the_exact_solution(crg):
    # the pairs whose theta - g is near 0 (all active pairs near the solution) are evaluated in
    # FP64, so mu_k (A_1 y + A_2 xi - theta_k)_- stays resolved as mu_k grows
    X, yb, _ = datagen.make("sq2", N=40, n=2)
    y_ref, xi_ref, _, _ = D.solve_regularized_nnls(X, yb, 0.1)
    s = crg.AlccSolver(X, yb, gamma=0.1)
    conv, outer = s.solve(1e-5, 14)
    m = s.metrics()
    y, xi = s.solution()
    err = _rel(y, y_ref)
    print(f"conv={conv} outer={outer} inner={s.info()['inner_total']} metrics={m} yrel={err:.2e}")
    assert conv and m["kkt"] <= 1e-5
    assert err <= 5e-4


def test_mu_cap_trajectory_matches_oracle(crg):
    X, yb, _ = datagen.make("sumexp", N=300, n=5)
    g = crg.AlccSolver(X, yb, gamma=0.1, fixed_inner=12, mu_max_scale=4e3)
    o = A.Alcc(X, yb, 0.1, A.AlccParams(fixed_inner=12, mu_max_scale=4e3))
    for _ in range(5):
        g.iterate(1)
        o.outer()
    assert g.info()["mu"] == pytest.approx(o.mu, rel=1e-14)
    assert _rel(g.solution()[0], o.y) <= 1e-6
    assert np.abs(_theta(g) - o.theta).max() <= 1e-6 * max(1.0, np.abs(yb).max())


def test_papg_calls_refuse_an_alcc_handle_and_reset_restores_iteration_zero(crg):
    X, yb, _ = datagen.make("sq2", N=64, n=2)
    s = crg.AlccSolver(X, yb, gamma=0.1, fixed_inner=5)
    with pytest.raises(crg.CrError) as e:
        s.metrics()
    assert e.value.status == crg.CR_ESTATE
    for call in (lambda: crg.Solver.iterate(s, 1), lambda: crg.Solver.solve(s, 1e-3, 10), s.kkt_residual,
                 s.objective):
        with pytest.raises(crg.CrError) as e:
            call()
        assert e.value.status == crg.CR_ESTATE
    s.iterate(2)
    assert np.abs(s.solution()[0] - yb).max() > 0
    s.reset()
    y, xi = s.solution()
    np.testing.assert_array_equal(y, yb)
    assert np.all(xi == 0.0) and np.all(_theta(s) == 0.0)
    assert s.info()["outer"] == 0


@pytest.mark.parametrize("bad", [dict(c=1.0), dict(kappa=0.0), dict(mu1_scale=-1.0), dict(theta_dtype="bf16"),
                                 dict(pair_engine=2)])
def test_bad_options_are_rejected(crg, bad):
    X, yb, _ = datagen.make("sq2", N=64, n=2)
    with pytest.raises(crg.CrError) as e:
        crg.AlccSolver(X, yb, **bad)
    assert e.value.status == crg.CR_EINVAL

