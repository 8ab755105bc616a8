"""Pins of the ALCC/MAPG oracle (Sec. II-D) to facts other than itself.

References: the explicit constraint matrices A_1, A_2 built row by row from problem (original)
(``tests/dense_qp.py``), singular values from LAPACK's SVD of those matrices, central finite
differences of the subproblem value, scipy's L-BFGS minimizer of the subproblem written with the
explicit matrices, and the exact solution of (regularize) from the active-set NNLS solve of its
dual.  CPU only.
"""
import numpy as np
import pytest
from scipy.optimize import minimize

from oracle import alcc as A
from paper_1407_7220_gb300 import datagen
from tests import dense_qp as D


def _rand(N, n, seed):
    rng = np.random.default_rng(seed)
    X = rng.normal(size=(N, n))
    y = rng.normal(size=N)
    xi = rng.normal(size=(N, n))
    T = rng.exponential(size=(N, N))
    np.fill_diagonal(T, 0.0)
    return X, y, xi, T


@pytest.mark.parametrize("N,n", [(5, 1), (7, 3), (9, 2)])
def test_sigma_max_squares_match_svd_of_explicit_matrices(N, n):
    X, *_ = _rand(N, n, N + n)
    A1, A2, _ = D.constraint_matrices(X)
    assert A.sigma2_A1(N) == pytest.approx(np.linalg.svd(A1, compute_uv=False)[0] ** 2, rel=1e-12)
    assert A.sigma2_A2(X) == pytest.approx(np.linalg.svd(A2, compute_uv=False)[0] ** 2, rel=1e-12)


@pytest.mark.parametrize("N,n", [(6, 2), (8, 3)])
def test_constraint_values_and_adjoint_match_explicit_rows(N, n):
    X, y, xi, T = _rand(N, n, 3 * N + n)
    A1, A2, pairs = D.constraint_matrices(X)
    g = A1 @ y + A2 @ xi.ravel()
    np.testing.assert_allclose(D.theta_vec(A.constraint_values(y, xi, X), pairs), g, rtol=0, atol=1e-12)
    a1, a2 = A.adjoint(T, X)
    m = D.theta_vec(T, pairs)
    np.testing.assert_allclose(a1, A1.T @ m, rtol=0, atol=1e-12)
    np.testing.assert_allclose(a2.ravel(), A2.T @ m, rtol=0, atol=1e-12)


def _explicit_value(y, xi, theta_vec, ybar, gamma, mu, A1, A2):
    r = A1 @ y + A2 @ xi.ravel() - theta_vec
    return (0.5 / mu) * np.sum((y - ybar) ** 2) + (0.5 * gamma / mu) * np.sum(xi ** 2) \
        + 0.5 * np.sum(np.minimum(r, 0.0) ** 2)


def test_subproblem_value_and_gradient():
    N, n, gamma, mu = 7, 2, 0.3, 0.05
    X, y, xi, T = _rand(N, n, 11)
    ybar = y + 0.3
    A1, A2, pairs = D.constraint_matrices(X)
    tv = D.theta_vec(T, pairs)
    v = A.subproblem_value(y, xi, T, ybar, gamma, mu, X)
    assert v == pytest.approx(_explicit_value(y, xi, tv, ybar, gamma, mu, A1, A2), rel=1e-13)
    gy, gxi = A.subproblem_grad(y, xi, T, ybar, gamma, mu, X)
    eps = 1e-6
    for i in range(N):
        e = np.zeros(N)
        e[i] = eps
        fd = (_explicit_value(y + e, xi, tv, ybar, gamma, mu, A1, A2)
              - _explicit_value(y - e, xi, tv, ybar, gamma, mu, A1, A2)) / (2 * eps)
        assert gy[i] == pytest.approx(fd, rel=1e-6, abs=1e-6)
    for i in range(N):
        for k in range(n):
            e = np.zeros((N, n))
            e[i, k] = eps
            fd = (_explicit_value(y, xi + e, tv, ybar, gamma, mu, A1, A2)
                  - _explicit_value(y, xi - e, tv, ybar, gamma, mu, A1, A2)) / (2 * eps)
            assert gxi[i, k] == pytest.approx(fd, rel=1e-6, abs=1e-6)


def test_ball_projection():
    c = np.array([1.0, -2.0, 0.5])
    z_in = c + np.array([0.1, 0.2, -0.1])
    np.testing.assert_array_equal(A.proj_ball(z_in, c, 1.0), z_in)
    z = c + np.array([3.0, -4.0, 0.0])
    p = A.proj_ball(z, c, 2.0)
    np.testing.assert_allclose(p, c + np.array([1.2, -1.6, 0.0]), rtol=0, atol=1e-15)


def test_mapg_reaches_the_subproblem_minimizer():
    # balls large enough to be inactive: MAPG's limit is the unconstrained minimizer of P_k,
    # found independently by L-BFGS on the explicit-matrix form
    X, yb, _ = datagen.make("sq2", N=12, n=2, seed=5)
    N, n = X.shape
    gamma, mu = 0.1, 0.2
    rng = np.random.default_rng(2)
    T = rng.exponential(0.05, size=(N, N))
    np.fill_diagonal(T, 0.0)
    A1, A2, pairs = D.constraint_matrices(X)
    tv = D.theta_vec(T, pairs)

    def f(z):
        return _explicit_value(z[:N], z[N:].reshape(N, n), tv, yb, gamma, mu, A1, A2)

    res = minimize(f, np.concatenate([yb, np.zeros(N * n)]), method="L-BFGS-B",
                   options=dict(ftol=1e-15, gtol=1e-11, maxiter=20000, maxcor=30))
    Ly = 1.0 / mu + A.sigma2_A1(N)
    Lxi = gamma / mu + A.sigma2_A2(X)
    y, xi, it = A.mapg(T, yb, gamma, mu, X, Ly, Lxi, yb.copy(), np.zeros((N, n)), 1e-13, 1e-13, 200000,
                       1e6, 1e6)
    assert it < 200000
    np.testing.assert_allclose(y, res.x[:N], rtol=0, atol=2e-6)
    np.testing.assert_allclose(xi.ravel(), res.x[N:], rtol=0, atol=2e-5)


def test_mapg_respects_the_balls():
    X, yb, _ = datagen.make("sq2", N=10, n=2, seed=6)
    N, n = X.shape
    T = np.zeros((N, N))
    # theta = 0, ybar given: the subproblem pulls y toward ybar; a small y-ball around ybar
    # and a small xi-ball keep every iterate inside
    y0 = yb + 1.0
    Ly = 1.0 / 0.1 + A.sigma2_A1(N)
    Lxi = 0.1 / 0.1 + A.sigma2_A2(X)
    y, xi, _ = A.mapg(T, yb, 0.1, 0.1, X, Ly, Lxi, y0, np.ones((N, n)), 0.0, 0.0, 50, 0.3, 0.2)
    assert np.linalg.norm(y - yb) <= 0.3 * (1 + 1e-12)
    assert np.linalg.norm(xi) <= 0.2 * (1 + 1e-12)


def test_radii_contain_the_solution():
    X, yb, _ = datagen.make("sq2", N=15, n=2, seed=8)
    gamma = 0.1
    y, xi, _, _ = D.solve_regularized_nnls(X, yb, gamma)
    By, Bxi = A.radii(yb, gamma)
    assert np.linalg.norm(y - yb) <= By
    assert np.linalg.norm(xi) <= Bxi


def test_kkt_is_zero_at_the_exact_solution_and_sees_a_perturbation():
    X, yb, _ = datagen.make("sq2", N=14, n=2, seed=9)
    gamma = 0.1
    y, xi, T, _ = D.solve_regularized_nnls(X, yb, gamma)
    sigma = max(1.0, float(np.ptp(yb)))
    assert A.kkt(y, xi, T, yb, gamma, X, sigma)["kkt"] <= 1e-9
    assert A.kkt(y + 1e-3, xi, T, yb, gamma, X, sigma)["stat"] >= 0.9e-3 / sigma
    assert A.kkt(y, xi, T * 1.01, yb, gamma, X, sigma)["kkt"] >= 1e-6


@pytest.mark.parametrize("gamma,n", [(0.1, 2), (0.05, 1)])
def test_alcc_converges_to_the_exact_solution(gamma, n):
    X, yb, _ = datagen.make("sq2", N=20, n=n, seed=12)
    y_ref, xi_ref, _, _ = D.solve_regularized_nnls(X, yb, gamma)
    s = A.Alcc(X, yb, gamma)
    assert s.solve(1e-6, 12)
    # multiplier estimates stay nonnegative; tau, the alphas and mu follow steps 5-6
    assert s.theta.min() >= 0.0
    assert s.mu == pytest.approx(A.AlccParams().mu1_scale / (2.0 * 20) * 2.0 ** len(s.inner), rel=1e-12)
    rel = np.abs(s.y - y_ref).max() / np.abs(y_ref).max()
    assert rel <= 2e-5, rel
    np.testing.assert_allclose(s.xi, xi_ref, rtol=0, atol=1e-3 * max(1.0, np.abs(xi_ref).max()))


def test_alcc_schedule_of_fig_alcc():
    X, yb, _ = datagen.make("sq2", N=10, n=2, seed=3)
    prm = A.AlccParams(fixed_inner=5)
    s = A.Alcc(X, yb, 0.1, prm)
    tau1, ay1, mu1 = s.tau, s.alpha_y, s.mu
    s.outer()
    s.outer()
    # (c k^(1+kappa))^2 for k = 1, 2
    f = (prm.c * 1.0) ** 2 * (prm.c * 2.0 ** (1 + prm.kappa)) ** 2
    assert s.tau == pytest.approx(tau1 / f, rel=1e-14)
    assert s.alpha_y == pytest.approx(ay1 / f, rel=1e-14)
    assert s.mu == pytest.approx(mu1 * prm.c ** 2, rel=1e-14)
    assert s.inner == [5, 5]


def test_planted_adjoint_sign_error_is_caught(monkeypatch):
    # a sign slip in the A_2 adjoint breaks the gradient pin
    X, y, xi, T = _rand(6, 2, 4)
    A1, A2, pairs = D.constraint_matrices(X)
    good = A.adjoint

    def bad(M, X):
        a1, a2 = good(M, X)
        return a1, -a2

    monkeypatch.setattr(A, "adjoint", bad)
    _, gxi = A.subproblem_grad(y, xi, T, y + 0.3, 0.3, 0.05, X)
    eps = 1e-6
    e = np.zeros_like(xi)
    e[2, 1] = eps
    tv = D.theta_vec(T, pairs)
    fd = (_explicit_value(y, xi + e, tv, y + 0.3, 0.3, 0.05, A1, A2)
          - _explicit_value(y, xi - e, tv, y + 0.3, 0.3, 0.05, A1, A2)) / (2 * eps)
    assert abs(gxi[2, 1] - fd) > 1e-3


def test_optional_mu_cap_schedule():
    # not in the paper: mu_{k+1} = min(c mu_k, mu_max), mu_max = mu_max_scale / sigma_max^2(A_1)
    X, yb, _ = datagen.make("sq2", N=10, n=2, seed=3)
    prm = A.AlccParams(fixed_inner=3, mu_max_scale=3e3)
    s = A.Alcc(X, yb, 0.1, prm)
    mus = [s.mu]
    for _ in range(4):
        s.outer()
        mus.append(s.mu)
    mu_max = 3e3 / A.sigma2_A1(10)
    assert mus == pytest.approx([1e3 / 20, 2e3 / 20, mu_max, mu_max, mu_max], rel=1e-14)
    # with mu fixed, theta_{k+1} = (A_1 y_k + A_2 xi_k - theta_k)_- (step 4 with mu_k / mu_{k+1} = 1)
    y, xi, th = s.y.copy(), s.xi.copy(), s.theta.copy()
    s.outer()
    m = np.maximum(th - A.constraint_values(s.y, s.xi, X), 0.0)
    np.fill_diagonal(m, 0.0)
    np.testing.assert_allclose(s.theta, m, rtol=0, atol=1e-15)
