"""Pins of the exact-solution reference (oracle/exact.py): constraint-generation NNLS.

It must equal the full dual NNLS on every pair (tests/dense_qp.py, tiny N), the FP64 P-APG
oracle run to a far tighter KKT tolerance (small N), and the stored converged P-APG reference
of recipe (1) at N = 500.
"""
import os

import numpy as np
import pytest

from oracle import exact as E
from oracle import oracle as O
from paper_1407_7220_gb300 import datagen
from tests import dense_qp as D

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rel(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


@pytest.mark.parametrize("gamma,n", [(0.1, 2), (0.01, 2), (0.1, 1), (0.05, 3)])
def test_equals_full_dual_nnls(gamma, n):
    X, yb, _ = datagen.make("sq2", N=20, n=n, seed=21)
    s = O.shift(yb)
    y_ref, xi_ref, T_ref, _ = D.solve_regularized_nnls(X, yb + s, gamma)
    y, xi, T, info = E.solve(X, yb, gamma)
    assert info["min_constraint"] >= -1e-12 * max(1.0, np.ptp(yb))
    np.testing.assert_allclose(y, y_ref - s, rtol=0, atol=1e-10)
    np.testing.assert_allclose(xi, xi_ref, rtol=0, atol=1e-9 * max(1.0, np.abs(xi_ref).max()))
    assert T.min() >= 0.0 and info["complementarity"] <= 1e-10


def test_equals_converged_papg_oracle():
    X, yb, _ = datagen.make("sq2", N=60, seed=5)
    o = O.Solver(X, yb, gamma=0.1, restart=True, restart_tol=1e-12)
    o.solve(1e-11, 3_000_000, check_every=50)
    assert o.metrics["kkt"] <= 1e-11
    y, xi, _, info = E.solve(X, yb, 0.1)
    assert _rel(y, o.y_hat) <= 1e-8
    np.testing.assert_allclose(xi, o.xi, rtol=0, atol=1e-6 * max(1.0, np.abs(xi).max()))


def test_stored_references_agree():
    # the exact solution of recipe (1) (N = 500, gamma = 0.1) and the FP64 P-APG oracle run to
    # KKT 9.9e-9 (tests/golden/make_golden.py) are the same fit
    ex = np.load(os.path.join(GOLDEN, "sq2_N500_g0.1_exact.npz"))
    pa = np.load(os.path.join(GOLDEN, "sq2_N500_g0.1.npz"))
    X, yb, _ = datagen.make("sq2", N=500)
    assert float(ex["X_sum"]) == pytest.approx(X.sum(), rel=0, abs=1e-12)
    assert float(ex["min_constraint"]) >= -1e-12 and float(ex["complementarity"]) <= 1e-10
    assert _rel(pa["y_hat"], ex["y_hat"]) <= 3e-7
