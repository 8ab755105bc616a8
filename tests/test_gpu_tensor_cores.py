"""The tensor-core pair pass (tcgen05 MMA for the residual and adjoint products) through the C ABI.

The two dense products of Step 2 and of the fused adjoint run as three TF32 products per
FP32 product, so the iterates differ from the CUDA-core engine only at FP32 rounding level.
The same trajectory bars as the CUDA-core parity tests apply against the FP64 oracle:
fitted values within 1e-6 relative, subgradients within 2e-4 of max(1, max|xi|), dual
value within 1e-5 relative.  Sizes cover several 256-column stripes, a ragged last stripe,
N not a multiple of 8 or 16, segments that change stripe inside a CTA, and every compiled
padded width from 8 up.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1407_7220_gb300 import datagen

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def crg():
    import paper_1407_7220_gb300 as m
    return m


def _rel(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def _recipe(n):
    return "maxaff" if n <= 10 else "lse"


def test_engine_selection(crg):
    X, yb, _ = datagen.make("maxaff", N=300, n=10)
    assert crg.Solver(X, yb, theta_dtype="bf16").info()["engine"] == "tensor_cores"
    assert crg.Solver(X, yb).info()["engine"] == "cuda_cores"          # FP32, n = 10
    X16, y16, _ = datagen.make("lse", N=300, n=16)
    assert crg.Solver(X16, y16).info()["engine"] == "tensor_cores"     # FP32, n = 16
    assert crg.Solver(X, yb, pair_engine=crg.PAIR_TENSOR_CORES).info()["engine"] == "tensor_cores"
    assert crg.Solver(X, yb, pair_engine=crg.PAIR_CUDA_CORES).info()["engine"] == "cuda_cores"
    assert crg.Solver(X, yb, theta_dtype="bf16", driver=crg.DRIVER_PERSISTENT).info()["engine"] == "cuda_cores"
    assert crg.Solver(X, yb, record_every=10).info()["engine"] == "cuda_cores"
    for bad in (dict(driver=crg.DRIVER_PERSISTENT), dict(record_every=10)):
        with pytest.raises(crg.CrError):
            crg.Solver(X, yb, pair_engine=crg.PAIR_TENSOR_CORES, **bad)
    X5, y5, _ = datagen.make("sumexp", N=300, n=5)
    assert crg.Solver(X5, y5).info()["engine"] == "cuda_cores"
    assert crg.Solver(X5, y5, pair_engine=crg.PAIR_TENSOR_CORES).info()["engine"] == "tensor_cores"


@pytest.mark.parametrize("N,n", [(300, 8), (1031, 10), (517, 16), (777, 20), (300, 32), (301, 5)])
@pytest.mark.parametrize("k", [1, 3, 40])
def test_trajectory_matches_oracle(crg, N, n, k):
    X, yb, _ = datagen.make(_recipe(n), N=N, n=n)
    g = crg.Solver(X, yb, gamma=0.1, stochastic_round=0, restart=0, pair_engine=crg.PAIR_TENSOR_CORES)
    assert g.info()["engine"] == "tensor_cores"
    o = O.Solver(X, yb, gamma=0.1, momentum=True, restart=False)   # the oracle's own L_g and shift
    g.iterate(k)
    o.iterate(k)
    y, xi = g.solution()
    assert _rel(y, o.y_hat) <= 1e-6, _rel(y, o.y_hat)
    assert np.abs(xi - o.xi).max() <= 2e-4 * max(1.0, np.abs(o.xi).max())
    assert g.objective()["dual"] == pytest.approx(o.metrics["dual"], rel=1e-5, abs=1e-9)


@pytest.mark.parametrize("N,n", [(1031, 10), (777, 20)])
def test_engines_agree(crg, N, n):
    X, yb, _ = datagen.make(_recipe(n), N=N, n=n)
    r = {}
    for eng in (crg.PAIR_TENSOR_CORES, crg.PAIR_CUDA_CORES):
        s = crg.Solver(X, yb, gamma=0.1, stochastic_round=0, restart=0, pair_engine=eng)
        s.iterate(60)
        r[eng] = s.solution()
    assert _rel(r[crg.PAIR_TENSOR_CORES][0], r[crg.PAIR_CUDA_CORES][0]) <= 1e-6


# the precision configuration's bound: fitted values within 1e-3 relative of the FP64 oracle
@pytest.mark.parametrize("dtype,tol", [("bf16", 1e-3), ("f16", 1e-3)])
def test_16bit_storage_matches_oracle(crg, dtype, tol):
    # theta rounded to 8 (BF16) or 11 (FP16) significant bits per store
    X, yb, _ = datagen.make("lse", N=640, n=20)
    g = crg.Solver(X, yb, gamma=0.1, theta_dtype=dtype, stochastic_round=0, restart=0)
    assert g.info()["engine"] == "tensor_cores"
    o = O.Solver(X, yb, gamma=0.1, momentum=True, restart=False)
    g.iterate(20)
    o.iterate(20)
    assert _rel(g.solution()[0], o.y_hat) <= tol


@pytest.mark.parametrize("grid", [1, 2, 7, 40])
def test_partitions_give_same_iterates(crg, grid):
    # one CTA walks every stripe (Xi reloaded at each segment); more CTAs split stripes
    X, yb, _ = datagen.make("maxaff", N=1201, n=10)
    tc = crg.PAIR_TENSOR_CORES
    ref = crg.Solver(X, yb, stochastic_round=0, restart=0, grid=64, pair_engine=tc)
    s = crg.Solver(X, yb, stochastic_round=0, restart=0, grid=grid, pair_engine=tc)
    assert s.info()["engine"] == "tensor_cores"
    ref.iterate(15)
    s.iterate(15)
    assert _rel(s.solution()[0], ref.solution()[0]) <= 1e-6


def test_deterministic_with_stochastic_rounding(crg):
    X, yb, _ = datagen.make("lse", N=900, n=20)
    r = []
    for _ in range(2):
        s = crg.Solver(X, yb, theta_dtype="bf16", stochastic_round=1, seed=7)
        s.iterate(12)
        r.append(s.solution())
    assert np.array_equal(r[0][0], r[1][0]) and np.array_equal(r[0][1], r[1][1])


def test_solve_reaches_fp64_confirmed_kkt(crg):
    X, yb, _ = datagen.make("maxaff", N=800, n=10)
    tc = crg.Solver(X, yb, gamma=0.1, stochastic_round=1, restart=0, kkt_every=50, pair_engine=crg.PAIR_TENSOR_CORES)
    cc = crg.Solver(X, yb, gamma=0.1, stochastic_round=1, restart=0, kkt_every=50, pair_engine=crg.PAIR_CUDA_CORES)
    conv, _ = tc.solve(1e-3, 200_000)
    assert conv and tc.kkt_residual()["kkt"] <= 1e-3
    conv2, _ = cc.solve(1e-3, 200_000)
    assert conv2
    # both at KKT 1e-3 of the same problem: fitted values within a few KKT units
    assert _rel(tc.solution()[0], cc.solution()[0]) <= 1e-2


# -------------------------------------------------------------------------
# the precision configuration at its stated sizes: recipe (3), n = 20, gamma = 1e-2
# -------------------------------------------------------------------------
@pytest.fixture(scope="module")
def lse_5000_oracle():
    X, yb, _ = datagen.make("lse", N=5000, n=20)
    o = O.Solver(X, yb, gamma=1e-2, momentum=True, restart=False)
    o.iterate(20)
    return X, yb, o.y_hat.copy()


@pytest.mark.parametrize("dtype", ["bf16", "f16"])
def test_16bit_subsample_instance_matches_oracle(crg, lse_5000_oracle, dtype):
    # the N = 5,000 instance of recipe (3): 16-bit multipliers against the FP64 oracle, bound 1e-3
    X, yb, y_o = lse_5000_oracle
    g = crg.Solver(X, yb, gamma=1e-2, theta_dtype=dtype, stochastic_round=0, restart=0)
    assert g.info()["engine"] == "tensor_cores"
    g.iterate(20)
    err = _rel(g.solution()[0], y_o)
    print(f"{dtype} N=5000 20 iterations: rel err vs oracle {err:.2e}")
    assert err <= 1e-3
    g.close()


def test_16bit_full_size_matches_fp32_path():
    # recipe (3) at N = 100,000 (2 x 20 GB of BF16 or FP16 multipliers, 2 x 40 GB in FP32): the
    # fitted values after the same iterations against the FP32 path, bound 1e-3 relative
    import torch
    import paper_1407_7220_gb300 as crg
    X, yb, _ = datagen.make("lse", N=100_000, n=20)
    K = 10
    res = {}
    for dt in ("bf16", "f16", "f32"):
        s = crg.Solver(X, yb, gamma=1e-2, theta_dtype=dt, stochastic_round=1, restart=0, driver=crg.DRIVER_PHASES)
        s.iterate(K)
        res[dt] = s.solution()[0]
        s.close()
        torch.cuda.synchronize()
    for dt in ("bf16", "f16"):
        err = _rel(res[dt], res["f32"])
        print(f"{dt} N=100000 {K} iterations: rel err vs FP32 {err:.2e}")
        assert err <= 1e-3


# -------------------------------------------------------------------------
# precision schedule: 16-bit multipliers first, then FP32 (cr_promote)
# -------------------------------------------------------------------------
@pytest.mark.parametrize("dtype,n", [("bf16", 10), ("f16", 10), ("bf16", 20)])
def test_promotion_widens_exactly_and_keeps_iterating(crg, dtype, n):
    from tests import devarray
    X, yb, _ = datagen.make("maxaff" if n == 10 else "lse", N=700, n=n)
    g = crg.Solver(X, yb, gamma=0.1, theta_dtype=dtype, stochastic_round=1, restart=0)
    g.iterate(15)
    before = devarray.theta_f64(g.device_state(), 700, dtype, fp16_exponent=g.options.fp16_exponent)
    y0, _ = g.solution()
    g.promote("f32")
    after = devarray.theta_f64(g.device_state(), 700, "f32")
    assert np.array_equal(before, after)                    # the widening is exact
    assert np.array_equal(g.solution()[0], y0)              # the iterate itself is unchanged
    assert g.info()["engine"] == ("tensor_cores" if n >= 16 else "cuda_cores")
    g.iterate(15)
    assert g.info()["iters"] == 30 and np.isfinite(g.solution()[0]).all()
    with pytest.raises(crg.CrError):
        g.promote("f32")                                    # already FP32


def test_promoted_schedule_converges_to_the_exact_fit(crg):
    import os
    X, yb, _ = datagen.make("sq2", N=500)
    ref = np.load(os.path.join(os.path.dirname(__file__), "golden", "sq2_N500_g0.1_exact.npz"))
    g = crg.Solver(X, yb, gamma=0.1, theta_dtype="bf16", stochastic_round=1, restart=0, kkt_every=50)
    g.solve(5e-2, 200_000)                                  # above the BF16 rounding floor
    g.promote("f32")
    conv, _ = g.solve(1e-4, 400_000)
    assert conv and g.kkt_residual()["kkt"] <= 1e-4
    assert _rel(g.solution()[0], ref["y_hat"]) <= 3e-4


def test_solve_runs_the_precision_schedule_of_promote_at(crg):
    # cr_options.promote_at: cr_solve solves in FP16 down to promote_at, widens to FP32 and goes
    # on to its tol; the same as doing the three steps by hand, bit for bit
    X, yb, _ = datagen.make("sq2", N=400)
    opts = dict(gamma=0.1, theta_dtype="f16", stochastic_round=1, restart=0, kkt_every=50)
    a = crg.Solver(X, yb, promote_at=0.1, **opts)
    conv_a, it_a = a.solve(1e-3, 200_000)
    b = crg.Solver(X, yb, **opts)
    c1, i1 = b.solve(0.1, 200_000)
    b.promote("f32")
    c2, i2 = b.solve(1e-3, 200_000 - i1)
    assert conv_a and c1 and c2 and it_a == i1 + i2
    assert np.array_equal(a.solution()[0], b.solution()[0])
    assert a.kkt_residual()["kkt"] <= 1e-3
    with pytest.raises(crg.CrError):
        a.promote("f32")                                    # the handle is FP32 now
