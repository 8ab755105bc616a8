"""The library's host-side problem constants against the oracle, without a GPU.

``cr_problem_constants`` computes sigma_max^2(A_2) through the covariance eigen-decomposition
and a secular equation per point; the oracle forms every block sum_m (x_m - x_l)(x_m - x_l)^T
and takes its largest eigenvalue directly (Jacobi in ``cr_oracle.c``, LAPACK in ``alcc.py``).
CPU only.
"""
import os

import numpy as np
import pytest

import paper_1407_7220_gb300 as crg
from oracle import alcc as A
from oracle import oracle as O
from paper_1407_7220_gb300 import datagen


@pytest.fixture(scope="module")
def built():
    if not os.path.exists(crg.library_path):
        from paper_1407_7220_gb300 import _build
        _build.build()
    return crg.library_path


@pytest.mark.parametrize("recipe,N,n,gamma", [("sq2", 20, 2, 0.1), ("sumexp", 300, 5, 0.05), ("maxaff", 97, 10, 1e-2),
                                               ("lse", 33, 32, 0.1), ("xqx", 100, 5, 0.1)])
def test_constants_match_the_oracle(built, recipe, N, n, gamma):
    X, yb, _ = datagen.make(recipe, N=N, n=n)
    c = crg.problem_constants(X, yb, gamma)
    assert c["L"] == pytest.approx(O.lipschitz(X, gamma), rel=1e-10)
    assert c["shift"] == O.shift(yb)
    assert c["sigma2_A1"] == 2.0 * N == A.sigma2_A1(N)
    assert c["sigma2_A2"] == pytest.approx(A.sigma2_A2(X), rel=1e-10)


def test_bad_inputs_are_rejected(built):
    X, yb, _ = datagen.make("sq2", N=20, n=2)
    for args in ((X, yb, 0.0), (X[:2], yb[:2], 0.1), (np.where(X > 0.5, np.nan, X), yb, 0.1)):
        with pytest.raises(crg.CrError) as e:
            crg.problem_constants(*args)
        assert e.value.status == crg.CR_EINVAL


@pytest.mark.parametrize("case", ["anisotropic", "ties", "one_far_point"])
def test_largest_block_found_where_it_is_not_the_farthest_point(built, case):
    # ||A_2||^2 = max over points of the largest eigenvalue of their block.  The library bounds
    # each point's value by N (lambda_max(cov) + ||x_l - xbar||^2) and solves the secular
    # equation only where that bound reaches the best value so far; these layouts put the
    # largest block away from the farthest point, or make several points tie.
    rng = np.random.default_rng(11)
    N, n = 240, 3
    if case == "anisotropic":
        X = np.clip(rng.normal(size=(N, n)) * np.array([4.0, 0.1, 0.1]), -7.0, 7.0)
        X[0] = [0.0, 9.0, 0.0]        # farthest from the mean, along a thin axis
        X[1] = [8.5, 0.0, 0.0]        # nearer, along the wide axis: the largest block
        d = X - X.mean(axis=0)
        lam = [np.linalg.eigvalsh(d.T @ d + N * np.outer(v, v))[-1] for v in d]
        assert np.argmax(lam) == 1 and np.argmax((d * d).sum(axis=1)) == 0
    elif case == "ties":
        X = np.repeat(rng.uniform(-1, 1, size=(N // 4, n)), 4, axis=0)
    else:
        X = rng.uniform(-1, 1, size=(N, n))
        X[17] = [40.0, -3.0, 5.0]
    yb = rng.normal(size=N)
    c = crg.problem_constants(X, yb, 0.1)
    assert c["sigma2_A2"] == pytest.approx(A.sigma2_A2(X), rel=1e-10)
