"""Pins of the FP64 oracle to facts fixed by the paper and by mathematics.

None of these re-types the oracle's formulas: the references are explicit
constraint matrices built from problem (original), an exact active-set NNLS
solve of the dual of (regularize), closed forms, and the inequalities of the
paper's theorems.  CPU only.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1407_7220_gb300 import datagen
from tests import dense_qp as D

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


def _inst(N=20, n=2, seed=7, recipe="sq2"):
    X, yb, _ = datagen.make(recipe, N=N, n=n, seed=seed)
    return X, yb


# --------------------------------------------------------------------------
# Step 1 closed form (Fig. 2 step 1, K = N) against the explicit Lagrangian
# --------------------------------------------------------------------------
@pytest.mark.parametrize("N,n", [(7, 3), (9, 1), (6, 5)])
def test_step1_matches_explicit_lagrangian_minimizer(N, n):
    rng = np.random.default_rng(N * 10 + n)
    X = rng.normal(size=(N, n))
    h = rng.normal(size=N) + 3.0
    gamma = 0.37
    T = rng.exponential(size=(N, N))
    np.fill_diagonal(T, 0.0)
    mu = rng.exponential(size=N)
    y, xi = O.eta(T, mu, X, h, gamma)
    # minimizer of 1/2||y-h||^2 + gamma/2||xi||^2 - theta^T C eta: H eta = htil + C^T theta
    _, eta = D.dense_dual(X, h, gamma, T, mu)
    np.testing.assert_allclose(y, eta[:N], rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(xi.ravel(), eta[N:], rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("N,n", [(7, 3), (8, 2)])
def test_residual_matches_explicit_constraint_rows(N, n):
    rng = np.random.default_rng(5)
    X = rng.normal(size=(N, n))
    y = rng.normal(size=N)
    xi = rng.normal(size=(N, n))
    G = O.residual(y, xi, X)
    A1, A2, pairs = D.constraint_matrices(X)
    Gd = A1 @ y + A2 @ xi.ravel()
    for v, (l1, l2) in zip(Gd, pairs):
        assert abs(G[l1, l2] - v) < 1e-12
    assert np.all(np.diag(G) == 0.0)


# --------------------------------------------------------------------------
# Lipschitz constant, Eq. (eq:lischitz)
# --------------------------------------------------------------------------
@pytest.mark.parametrize("N,n,gamma", [(8, 2, 0.5), (10, 3, 1.0), (6, 1, 0.05)])
def test_lipschitz_bound_dominates_true_constant(N, n, gamma):
    rng = np.random.default_rng(N + n)
    X = rng.uniform(-1, 1, size=(N, n))
    L = O.lipschitz(X, gamma)
    C, _ = D.big_C(X)
    smax2 = np.linalg.norm(C, 2) ** 2
    Hinv = np.concatenate([np.ones(N), np.full(N * n, 1.0 / gamma)])
    lam = np.linalg.eigvalsh((C * Hinv) @ C.T)[-1]  # Lipschitz constant of grad g_gamma
    assert L >= lam * (1 - 1e-12)
    if gamma <= 1.0:
        assert L * gamma >= smax2 * (1 - 1e-12)  # L_g = sigma_max(C)^2 / gamma is dominated
    # the bound is the sum 1 + ||A_1||^2 + ||A_2||^2: each term exact
    A1, A2, _ = D.constraint_matrices(X)
    a1 = np.linalg.norm(A1, 2) ** 2
    a2 = np.linalg.norm(A2, 2) ** 2
    assert abs(a1 - 2 * N) < 1e-9 * N
    np.testing.assert_allclose(L * gamma, 1 + a1 + a2, rtol=1e-10)


# --------------------------------------------------------------------------
# N = 2, n = 1: closed form of (regularize)
# --------------------------------------------------------------------------
def test_two_points_closed_form():
    # For x_1 < x_2, gap D = x_2 - x_1, the optimal slopes are xi_1 = min(0, d/D),
    # xi_2 = max(0, d/D) with d = y_2 - y_1, so (regularize) reduces to
    # min 1/2(y1-yb1)^2 + 1/2(y2-yb2)^2 + gamma/2 d^2/D^2, solved by
    # d = (yb2 - yb1) / (1 + 2 gamma / D^2) and y1 + y2 = yb1 + yb2.
    for yb, gamma in (([0.3, 1.1], 0.2), ([1.0, -0.5], 0.05)):
        X = np.array([[-0.4], [0.6]])
        yb = np.array(yb)
        Dx = 1.0
        d = (yb[1] - yb[0]) / (1 + 2 * gamma / Dx ** 2)
        m = yb.mean()
        y_ref = np.array([m - d / 2, m + d / 2])
        xi_ref = np.array([min(0.0, d / Dx), max(0.0, d / Dx)])
        s = O.Solver(X, yb, gamma=gamma, restart=True)
        s.solve(1e-13, 200000, check_every=10)
        np.testing.assert_allclose(s.y_hat, y_ref, rtol=0, atol=1e-10)
        np.testing.assert_allclose(s.xi[:, 0], xi_ref, rtol=0, atol=1e-9)


# --------------------------------------------------------------------------
# Brute force: exact dual NNLS at N = 20 (recipe (1))
# --------------------------------------------------------------------------
def _nnls_reference(X, yb, gamma):
    s = O.shift(yb)
    y, xi, T, dual = D.solve_regularized_nnls(X, yb + s, gamma)
    # the NNLS point is itself checked through the explicit matrices:
    A1, A2, pairs = D.constraint_matrices(X)
    g = A1 @ y + A2 @ xi.ravel()
    th = D.theta_vec(T, pairs)
    scale = max(1.0, np.ptp(yb))
    assert g.min() >= -1e-9 * scale            # primal feasibility
    assert th.min() >= 0.0                      # dual feasibility
    assert np.abs(th * g).max() <= 1e-9 * scale ** 2  # complementary slackness
    assert y.min() > 0.0                        # the shifted y >= 0 rows are inactive
    return y - s, xi, T, dual, s


@pytest.mark.parametrize("gamma,restart,n", [(0.1, True, 2), (0.01, True, 2), (0.1, False, 2), (0.05, True, 1),
                                             (0.1, True, 3)])
def test_oracle_converges_to_nnls_bruteforce(gamma, restart, n):
    X, yb = _inst(N=20, n=n, seed=11)
    y_ref, xi_ref, _, _, _ = _nnls_reference(X, yb, gamma)
    s = O.Solver(X, yb, gamma=gamma, restart=restart)
    k = s.solve(1e-11, 3_000_000, check_every=100)
    assert s.metrics["kkt"] <= 1e-11, (k, s.metrics)
    assert s.mu1.max() == 0.0                   # y >= 0 rows inactive after the shift
    rel = np.abs(s.y_hat - y_ref).max() / np.abs(y_ref).max()
    assert rel <= 1e-8, rel
    np.testing.assert_allclose(s.xi, xi_ref, rtol=0, atol=1e-6 * max(1.0, np.abs(xi_ref).max()))


# --------------------------------------------------------------------------
# Invariants at every iteration
# --------------------------------------------------------------------------
def test_invariants_every_iteration():
    X, yb = _inst(N=15, n=2, seed=3)
    s = O.Solver(X, yb, gamma=0.1)
    for _ in range(60):
        s.iterate(1)
        m = s.metrics
        T = s.theta1
        # sum_l (A_1^T theta)_l = 0 because every row of A_1 sums to zero
        assert abs(m["sum_check"]) <= 1e-12 * max(1.0, T.sum())
        assert T.min() >= 0.0 and s.mu1.min() >= 0.0
        assert np.all(np.diag(T) == 0.0) and np.all(np.diag(s.theta2) == 0.0)
        # metrics agree with the explicit-matrix definitions
        A1, A2, pairs = D.constraint_matrices(X)
        g = A1 @ s.y_shifted + A2 @ s.xi.ravel()
        npairs = len(pairs)
        viol = np.concatenate([np.minimum(g, 0.0), np.minimum(s.y_shifted, 0.0)])
        assert abs(m["infeas"] - np.linalg.norm(viol) / np.sqrt(npairs)) <= 1e-12
        th = np.concatenate([D.theta_vec(T, pairs), s.mu1])
        gap = th @ np.concatenate([g, s.y_shifted])
        assert abs(m["gap"] - gap / npairs) <= 1e-12 * max(1.0, abs(gap))
        dd, _ = D.dense_dual(X, s.h, s.gamma, T, s.mu1)
        assert abs(m["dual"] - dd) <= 1e-10 * max(1.0, abs(dd))


# --------------------------------------------------------------------------
# Convergence behaviour the paper states
# --------------------------------------------------------------------------
def test_dual_gradient_ascent_is_monotone():
    # momentum = 0 is the paper's comparator (dual gradient ascent, Sec. III);
    # with step 1/L on an L-smooth concave function the dual value never decreases.
    X, yb = _inst(N=15, n=2, seed=4)
    s = O.Solver(X, yb, gamma=0.05, momentum=False)
    prev = -np.inf
    for _ in range(300):
        s.iterate(1)
        d = s.metrics["dual"]
        assert d >= prev - 1e-12 * abs(d)
        prev = d


@pytest.mark.parametrize("gamma", [0.1, 0.02])
def test_apg_rate_and_theorem1_bounds(gamma):
    # Sec. II-D: rho* - rho(eta_l) <= 2 L ||eta_0 - eta*||^2 / (l + 1)^2 (eta_0 = 0 here);
    # Theorem 1: ||(A_1 y_d + A_2 xi_d)_-||_2 <= sqrt(2 delta / gamma) sigma_max(C).
    X, yb = _inst(N=12, n=2, seed=9)
    s = O.Solver(X, yb, gamma=gamma)
    _, _, Tstar, _, _ = _nnls_reference(X, yb, gamma)
    dstar, _ = D.dense_dual(X, s.h, gamma, Tstar, np.zeros(12))
    C, pairs = D.big_C(X)
    smax = np.linalg.norm(C, 2)
    A1, A2, _ = D.constraint_matrices(X)
    nrm2 = np.sum(Tstar ** 2)
    for ell in range(1, 400):
        s.iterate(1)
        m = s.metrics
        delta = dstar - m["dual"]
        assert delta >= -1e-10 * abs(dstar)
        assert delta <= 2 * s.L * nrm2 / (ell + 1) ** 2 * (1 + 1e-9) + 1e-12
        g = A1 @ s.y_shifted + A2 @ s.xi.ravel()
        infeas = np.linalg.norm(np.minimum(g, 0.0))
        assert infeas <= np.sqrt(2 * max(delta, 0.0) / gamma) * smax * (1 + 1e-9) + 1e-12


def test_unique_fitted_values_from_any_start():
    # y* is unique for N >= n + 1 (after problem (original)); at gamma > 0 the
    # strongly convex (regularize) has a unique (y, xi) even though theta* is not unique.
    X, yb = _inst(N=14, n=2, seed=12)
    a = O.Solver(X, yb, gamma=0.1, restart=True)
    a.solve(1e-11, 3_000_000, check_every=100)
    rng = np.random.default_rng(0)
    th0 = rng.exponential(0.3, size=(14, 14))
    b = O.Solver(X, yb, gamma=0.1, restart=True, theta0=th0)
    b.solve(1e-11, 3_000_000, check_every=100)
    assert not np.allclose(a.theta1, b.theta1, atol=1e-6)  # different dual points ...
    np.testing.assert_allclose(a.y_hat, b.y_hat, rtol=0, atol=1e-8)  # ... same fit


def test_shift_is_exact():
    # A_1 1 = 0, so shifting ybar by any constant changes y by the same constant
    # and leaves the fitted values unchanged.
    X, yb = _inst(N=12, n=2, seed=2)
    a = O.Solver(X, yb, gamma=0.1, restart=True)
    a.solve(1e-11, 2_000_000, check_every=100)
    b = O.Solver(X, yb, gamma=0.1, restart=True, s=O.shift(yb) + 3.25)
    b.solve(1e-11, 2_000_000, check_every=100)
    np.testing.assert_allclose(a.y_hat, b.y_hat, rtol=0, atol=1e-8)


def test_restart_and_plain_papg_same_limit():
    X, yb = _inst(N=16, n=2, seed=21)
    a = O.Solver(X, yb, gamma=0.1, restart=False)
    a.solve(1e-11, 3_000_000, check_every=100)
    b = O.Solver(X, yb, gamma=0.1, restart=True)
    b.solve(1e-11, 3_000_000, check_every=100)
    np.testing.assert_allclose(a.y_hat, b.y_hat, rtol=0, atol=1e-8)


def test_planted_sign_error_is_caught():
    # A mistake planted in an explicit-matrix copy (the sign of the xi term)
    # must disagree with the oracle's Step 1 -- this shows the explicit-matrix
    # pin can see such a mistake.
    rng = np.random.default_rng(1)
    N, n = 6, 2
    X = rng.normal(size=(N, n))
    h = rng.normal(size=N)
    T = rng.exponential(size=(N, N))
    np.fill_diagonal(T, 0)
    mu = np.zeros(N)
    y, xi = O.eta(T, mu, X, h, 0.5)
    A1, A2, pairs = D.constraint_matrices(X)
    th = D.theta_vec(T, pairs)
    bad_xi = (-A2.T @ th) / 0.5
    assert np.abs(bad_xi - xi.ravel()).max() > 1e-3


# --------------------------------------------------------------------------
# Forward-mode derivative of K unrolled iterations (differentiation reference)
# --------------------------------------------------------------------------
def test_oracle_jvp_matches_central_differences():
    X, yb, _ = datagen.make("sumexp", N=30, n=3, seed=4)
    g = 0.1
    L = O.lipschitz(X, g)
    s = O.shift(yb)
    K = 20
    rng = np.random.default_rng(3)
    for _ in range(3):
        dy = rng.normal(size=yb.shape)
        dX = rng.normal(size=X.shape)
        yh, dyh = O.papg_jvp(X, yb, g, L, s, K, dy, dX)
        eps = 1e-6
        yp, _ = O.papg_jvp(X + eps * dX, yb + eps * dy, g, L, s, K, dy, dX)
        ym, _ = O.papg_jvp(X - eps * dX, yb - eps * dy, g, L, s, K, dy, dX)
        fd = (yp - ym) / (2 * eps)
        assert np.abs(fd - dyh).max() <= 1e-7 * np.abs(fd).max()
    # the primal of the JVP routine is the P-APG iterate of the Solver
    o = O.Solver(X, yb, gamma=g, L=L, s=s, restart=False)
    o.iterate(K)
    np.testing.assert_allclose(yh, o.y_hat, rtol=0, atol=1e-12)
    # linearity in the direction
    _, d1 = O.papg_jvp(X, yb, g, L, s, K, dy, dX)
    _, d2 = O.papg_jvp(X, yb, g, L, s, K, 2.5 * dy, 2.5 * dX)
    np.testing.assert_allclose(d2, 2.5 * d1, rtol=1e-12, atol=1e-12)


# --------------------------------------------------------------------------
# Q_2 with a finite ball (Eq. (lambda_dual)): {lambda >= 0, ||lambda||_2 <= B_theta}
# --------------------------------------------------------------------------
def test_large_ball_leaves_the_iterates_unchanged():
    X, yb = _inst(N=25, n=2, seed=6)
    a = O.Solver(X, yb, gamma=0.1)
    a.iterate(40)
    big = 10.0 * max(1.0, np.sqrt((a.theta1 ** 2).sum() + (a.mu1 ** 2).sum()))
    b = O.Solver(X, yb, gamma=0.1, B_theta=big)
    b.iterate(40)
    assert np.array_equal(a.theta1, b.theta1) and np.array_equal(a.y_hat, b.y_hat)


@pytest.mark.parametrize("B", [0.05, 0.3])
def test_ball_step_is_the_euclidean_projection(B):
    # one step of Fig. 2 from theta0 (beta = 0 at the first iteration): theta^(1) = Pi_{Q_2}(v),
    # v = theta0 - (1/L) C eta(theta0), built here from the explicit matrices; the projection
    # is computed independently by SLSQP on min ||q - v||^2 s.t. q >= 0, ||q||^2 <= B^2
    from scipy.optimize import minimize
    X, yb = _inst(N=5, n=2, seed=8)
    N = 5
    rng = np.random.default_rng(2)
    th0 = rng.uniform(0.0, 0.2, size=(N, N))
    np.fill_diagonal(th0, 0.0)
    mu0 = rng.uniform(0.0, 0.05, size=N)
    s = O.Solver(X, yb, gamma=0.1, theta0=th0, mu0=mu0, B_theta=B)
    C, pairs = D.big_C(X)
    lam0 = np.concatenate([D.theta_vec(th0, pairs), mu0])
    Hinv = np.concatenate([np.ones(N), np.full(N * 2, 1.0 / 0.1)])
    htil = np.concatenate([s.h, np.zeros(N * 2)])
    eta0 = Hinv * (htil + C.T @ lam0)
    v = lam0 - (C @ eta0) / s.L
    res = minimize(lambda q: 0.5 * np.sum((q - v) ** 2), np.maximum(v, 0.0) * 0.5, jac=lambda q: q - v,
                   method="SLSQP", bounds=[(0.0, None)] * v.size,
                   constraints=[{"type": "ineq", "fun": lambda q: B * B - q @ q, "jac": lambda q: -2.0 * q}],
                   options={"ftol": 1e-15, "maxiter": 500})
    s.iterate(1)
    got = np.concatenate([D.theta_vec(s.theta1, pairs), s.mu1])
    assert np.sqrt(got @ got) <= B * (1 + 1e-12) and got.min() >= 0.0
    np.testing.assert_allclose(got, res.x, rtol=0, atol=1e-7)


def test_dual_gradient_ascent_with_ball_is_monotone():
    # projected gradient ascent with step 1/L on an L-smooth concave function over the convex
    # set Q_2 never decreases the dual value, with the ball active or not
    X, yb = _inst(N=15, n=2, seed=4)
    s = O.Solver(X, yb, gamma=0.05, momentum=False, B_theta=0.02)
    prev, active = -np.inf, 0
    for _ in range(200):
        s.iterate(1)
        d = s.metrics["dual"]
        assert d >= prev - 1e-12 * abs(d)
        prev = d
        nrm = np.sqrt((s.theta1 ** 2).sum() + (s.mu1 ** 2).sum())
        assert nrm <= 0.02 * (1 + 1e-12)
        active += nrm >= 0.02 * (1 - 1e-9)
    assert active > 100   # the ball constraint binds along the run


# --------------------------------------------------------------------------
# Lemma 1 (Sec. II-C): ||y(gamma) - y*||_2 <= B_xi sqrt(gamma), and special cases
# --------------------------------------------------------------------------
def _convex_ls_1d(x, yb):
    """Least-squares convex fit in one dimension (the textbook problem problem (original)
    reduces to for n = 1): with the points sorted by x, the slopes between neighbours must not
    decrease, D y >= 0; the projection of ybar onto that cone by the dual NNLS
    min_{lam >= 0} ||D^T lam + ybar||, y* = ybar + D^T lam."""
    from scipy.optimize import nnls
    order = np.argsort(x)
    xs, ys = x[order], yb[order]
    N = len(xs)
    D_ = np.zeros((N - 2, N))
    for i in range(1, N - 1):
        dl, dr = xs[i] - xs[i - 1], xs[i + 1] - xs[i]
        D_[i - 1, i - 1] = 1.0 / dl
        D_[i - 1, i] = -1.0 / dl - 1.0 / dr
        D_[i - 1, i + 1] = 1.0 / dr
    lam, _ = nnls(D_.T, -ys, maxiter=100 * N)
    y_sorted = ys + D_.T @ lam
    # minimum-norm subgradients: at each point, the value of [left slope, right slope] closest to 0
    slopes = np.diff(y_sorted) / np.diff(xs)
    lo = np.concatenate([[-np.inf], slopes])
    hi = np.concatenate([slopes, [np.inf]])
    xi_sorted = np.clip(0.0, lo, hi)
    y = np.empty(N)
    xi = np.empty(N)
    y[order], xi[order] = y_sorted, xi_sorted
    return y, xi


def test_one_dimensional_case_and_holder_continuity():
    from oracle import exact as E
    X, yb = _inst(N=20, n=1, seed=13)
    y_star, xi_star = _convex_ls_1d(X[:, 0], yb)
    B_xi = np.linalg.norm(xi_star)
    assert np.all(np.diff(np.diff(y_star[np.argsort(X[:, 0])]) / np.diff(np.sort(X[:, 0]))) >= -1e-10)
    for gamma in (1e-1, 1e-2, 1e-3, 1e-4, 1e-5):
        y_g, xi_g, _, _ = E.solve(X, yb, gamma)
        assert np.linalg.norm(y_g - y_star) <= B_xi * np.sqrt(gamma) * (1 + 1e-9)   # Lemma 1
        assert np.linalg.norm(xi_g) <= B_xi * (1 + 1e-9)                            # from its proof
    # and the P-APG oracle at gamma = 1e-3 lands on the same y(gamma)
    o = O.Solver(X, yb, gamma=1e-3, restart=True, restart_tol=1e-12)
    o.solve(1e-11, 3_000_000, check_every=100)
    y_g, _, _, _ = E.solve(X, yb, 1e-3)
    np.testing.assert_allclose(o.y_hat, y_g, rtol=0, atol=1e-8)


def test_noiseless_affine_data():
    # ybar = a^T x + b is itself feasible with the subgradients xi_l = a (at gamma = 0 it is the
    # solution, with B_xi = sqrt(N) ||a||); at gamma > 0 Lemma 1 bounds the fit's deviation
    from oracle import exact as E
    rng = np.random.default_rng(17)
    N, n = 25, 2
    X = rng.uniform(-1.0, 1.0, size=(N, n))
    a, b = np.array([0.7, -1.3]), 0.4
    yb = X @ a + b
    B_xi = np.sqrt(N) * np.linalg.norm(a)
    prev = np.inf
    for gamma in (1e-1, 1e-2, 1e-3, 1e-4):
        y_g, xi_g, _, _ = E.solve(X, yb, gamma)
        dev = np.linalg.norm(y_g - yb)
        assert dev <= B_xi * np.sqrt(gamma) * (1 + 1e-9)
        assert dev <= prev + 1e-12     # y(gamma) moves toward ybar as gamma decreases
        prev = dev
    o = O.Solver(X, yb, gamma=1e-2, restart=True, restart_tol=1e-12)
    o.solve(1e-11, 3_000_000, check_every=100)
    y_g, _, _, _ = E.solve(X, yb, 1e-2)
    np.testing.assert_allclose(o.y_hat, y_g, rtol=0, atol=1e-8)
