"""Reverse mode through unrolled P-APG iterations (cr_backward) against the FP64
oracle's forward-mode derivative (itself pinned to central finite differences)."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1407_7220_gb300 import datagen

pytestmark = pytest.mark.gpu


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
