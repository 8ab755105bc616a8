"""Reverse mode through unrolled P-APG iterations (cr_backward) against the FP64
oracle's forward-mode derivative (itself pinned to central finite differences)."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1407_7220_gb300 import datagen

pytestmark = pytest.mark.gpu


def _rel(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def _vjp(crg, X, yb, K, k, ubar, gamma=0.1, **opts):
    import torch
    s = crg.Solver(X, yb, gamma=gamma, restart=0, stochastic_round=0, record_every=k, **opts)
    s.iterate(K)
    y_before, _ = s.solution()
    u = torch.tensor(ubar, dtype=torch.float32, device="cuda")
    dyb = torch.empty_like(u)
    dX = torch.empty((X.shape[0], X.shape[1]), dtype=torch.float32, device="cuda")
    s.backward(u, dyb, dX)
    y_after, _ = s.solution()
    assert np.array_equal(y_before, y_after)          # forward state restored
    assert s.info()["iters"] == K
    return s, dyb.cpu().numpy().astype(np.float64), dX.cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("N,n,K,k", [(60, 2, 23, 5), (130, 3, 40, 10), (300, 5, 30, 30)])
def test_backward_matches_oracle_directional_derivatives(N, n, K, k):
    import paper_1407_7220_gb300 as crg
    X, yb, f0 = datagen.make("sumexp", N=N, n=n, seed=N)
    rng = np.random.default_rng(1)
    ubar = rng.normal(size=N)
    s, gyb, gX = _vjp(crg, X, yb, K, k, ubar)
    L, sh = O.lipschitz(X, 0.1), O.shift(yb)   # the oracle's own constants
    errs = []
    for _ in range(6):
        dy = rng.normal(size=N)
        dX = rng.normal(size=X.shape)
        _, jv = O.papg_jvp(X, yb, 0.1, L, sh, K, dy, dX)
        want = float(ubar @ jv)
        got = float(gyb @ dy + (gX * dX).sum())
        errs.append(abs(got - want) / max(abs(want), 1e-12))
    print("rel errors", ["%.2e" % e for e in errs])
    assert max(errs) < 1e-3


def test_backward_independent_of_checkpoint_spacing_and_linear():
    import paper_1407_7220_gb300 as crg
    X, yb, _ = datagen.make("sumexp", N=200, n=5, seed=2)
    rng = np.random.default_rng(0)
    u1, u2 = rng.normal(size=200), rng.normal(size=200)
    _, a_y, a_X = _vjp(crg, X, yb, 36, 36, u1)
    _, b_y, b_X = _vjp(crg, X, yb, 36, 5, u1)
    np.testing.assert_allclose(b_y, a_y, rtol=0, atol=1e-5 * np.abs(a_y).max())
    np.testing.assert_allclose(b_X, a_X, rtol=0, atol=1e-5 * np.abs(a_X).max())
    _, c_y, c_X = _vjp(crg, X, yb, 36, 5, u2)
    _, d_y, d_X = _vjp(crg, X, yb, 36, 5, 2.0 * u1 - 3.0 * u2)
    np.testing.assert_allclose(d_y, 2.0 * b_y - 3.0 * c_y, rtol=0, atol=1e-4 * np.abs(d_y).max())
    np.testing.assert_allclose(d_X, 2.0 * b_X - 3.0 * c_X, rtol=0, atol=1e-4 * np.abs(d_X).max())


def test_autograd_function_gradient_matches_oracle():
    import torch
    import paper_1407_7220_gb300 as crg
    X, yb, f0 = datagen.make("sumexp", N=150, n=5, seed=7)
    Xt = torch.tensor(X, dtype=torch.float32, device="cuda", requires_grad=True)
    yt = torch.tensor(yb, dtype=torch.float32, device="cuda", requires_grad=True)
    K = 30
    yhat = crg.convex_fit(Xt, yt, iters=K, record_every=10, gamma=0.1, stochastic_round=0)
    target = torch.tensor(f0, dtype=torch.float32, device="cuda")
    loss = ((yhat - target) ** 2).sum()          # the differentiation workload's loss
    loss.backward()
    # the solver works on the FP32-rounded inputs; compare with the oracle on the same data
    Xr = Xt.detach().double().cpu().numpy()
    yr = yt.detach().double().cpu().numpy()
    L, sh = O.lipschitz(Xr, 0.1), O.shift(yr)
    rng = np.random.default_rng(11)
    for _ in range(4):
        dy = rng.normal(size=yb.shape)
        dX = rng.normal(size=X.shape)
        yo, jv = O.papg_jvp(Xr, yr, 0.1, L, sh, K, dy, dX)
        want = float(2.0 * (yo - f0) @ jv)
        got = float((yt.grad.double().cpu().numpy() * dy).sum() + (Xt.grad.double().cpu().numpy() * dX).sum())
        assert abs(got - want) <= 2e-3 * abs(want) + 1e-6, (got, want)


# -------------------------------------------------------------------------
# the differentiation configuration at its stated size: recipe (5), N = 5,000, n = 5,
# 500 unrolled iterations, checkpoints every 50, 32 random directions
# -------------------------------------------------------------------------
def _c5_reference():
    import importlib.util
    import os
    here = os.path.join(os.path.dirname(__file__), "golden")
    spec = importlib.util.spec_from_file_location("make_c5", os.path.join(here, "make_c5.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod, np.load(os.path.join(here, "sumexp_N5000_K500_jvp.npz"))


def _c5_check(dtype):
    import torch
    import paper_1407_7220_gb300 as crg
    mod, ref = _c5_reference()
    N, n, K = int(ref["N"]), int(ref["n"]), int(ref["K"])
    X, yb, f0 = datagen.make("sumexp", N=N, n=n)
    assert float(ref["X_sum"]) == pytest.approx(X.sum(), rel=0, abs=1e-9)
    # the stored central differences pin the stored forward-mode values at this size
    fd, jvp = ref["fd"], ref["jvp"]
    assert abs(fd[0, -1] - jvp[0]) <= 1e-4 * abs(jvp[0])
    s = crg.Solver(X, yb, gamma=float(ref["gamma"]), theta_dtype=dtype, restart=0, stochastic_round=0, record_every=50)
    s.iterate(K)
    y, _ = s.solution()
    err_y = _rel(y, ref["y_hat"])
    u = torch.tensor(2.0 * (ref["y_hat"] - f0), dtype=torch.float32, device="cuda")
    gy = torch.empty_like(u)
    gX = torch.empty((N, n), dtype=torch.float32, device="cuda")
    s.backward(u, gy, gX)
    s.close()
    # (the seed enters as FP32: its rounding, below 1e-7 relative, is far inside the bars)
    jvp_u = jvp
    gy = gy.double().cpu().numpy()
    gX = gX.double().cpu().numpy()
    dY, dX = mod.directions(N, n, len(jvp), int(ref["seed"]))
    got = np.array([gy @ dY[k] + (gX * dX[k]).sum() for k in range(len(jvp))])
    rel = np.abs(got - jvp_u) / np.abs(jvp_u)
    agg = np.linalg.norm(got - jvp_u) / np.linalg.norm(jvp_u)
    vs_fd = np.abs(got[:fd.shape[0]] - fd[:, -1]) / np.abs(fd[:, -1])
    print(f"{dtype}: fit vs oracle {err_y:.2e}; directional derivatives: max rel {rel.max():.2e}, "
          f"median {np.median(rel):.2e}, aggregate {agg:.2e}; vs central differences {vs_fd}")
    return err_y, rel, agg, vs_fd


def test_differentiation_configuration_fp64_matches_oracle_derivatives():
    # tests/golden/make_c5.py stored, from the FP64 oracle only: its fitted values after 500
    # iterations, u . J d_k for 32 directions d_k (forward mode; u = 2 (yhat - f0), the gradient
    # of the loss ||yhat - f0||^2 with the target held fixed), and central differences of the
    # oracle's loss on 2 of them.  With FP64 multipliers the GPU runs the oracle's map (fit to
    # 1e-12): its reverse mode (cr_backward, checkpoint every 50) seeded with the same u must give
    # <grad, d_k> within the configuration's 1e-4 of the oracle and of the central differences.
    err_y, rel, agg, vs_fd = _c5_check("f64")
    assert err_y <= 1e-12
    assert rel.max() <= 1e-4 and agg <= 1e-4
    assert vs_fd.max() <= 1e-4


def test_differentiation_configuration_fp32_forward():
    # With FP32 multipliers (the configuration's FP32 forward) the fit stays within 1e-6, but the
    # unrolled map is piecewise linear with N(N-1) K kinks and its derivative jumps where a pair
    # changes sides: the FP64 oracle's own derivative moves by 2e-3 (N = 2000, K = 200) to 1e-2
    # when its inputs move by 1e-7 relative, which is the size of the FP32 trajectory's drift.
    # The FP32 reverse mode is the exact derivative of the FP32 map (masks recomputed bit for
    # bit); against the FP64 map's derivative it measured 1.3e-2 aggregate at this size.
    err_y, rel, agg, vs_fd = _c5_check("f32")
    assert err_y <= 1e-6
    assert agg <= 5e-2


@pytest.mark.parametrize("N,n,K,k", [(60, 2, 23, 5), (300, 5, 30, 10), (517, 4, 40, 40)])
def test_fp64_backward_matches_oracle_directional_derivatives(N, n, K, k):
    # FP64 multipliers: forward and reverse mode in FP64, the oracle's masks exactly
    import paper_1407_7220_gb300 as crg
    X, yb, f0 = datagen.make("sumexp", N=N, n=n, seed=N + 1)
    rng = np.random.default_rng(5)
    ubar = rng.normal(size=N)
    s, gyb, gX = _vjp(crg, X, yb, K, k, ubar, theta_dtype="f64")
    L, sh = O.lipschitz(X, 0.1), O.shift(yb)
    errs = []
    for _ in range(6):
        dy = rng.normal(size=N)
        dX = rng.normal(size=X.shape)
        _, jv = O.papg_jvp(X, yb, 0.1, L, sh, K, dy, dX)
        want = float(ubar.astype(np.float32).astype(np.float64) @ jv)
        got = float(gyb @ dy + (gX * dX).sum())
        errs.append(abs(got - want) / max(abs(want), 1e-12))
    print("rel errors", ["%.2e" % e for e in errs])
    assert max(errs) < 1e-6
