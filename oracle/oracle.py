"""ctypes wrapper around ``cr_oracle.c`` (FP64 P-APG at K = N).

TEST INFRASTRUCTURE ONLY -- see the package docstring.  Every function here
marshals numpy arrays into the C oracle; the arithmetic lives in
``cr_oracle.c`` and follows Fig. 2 (P-APG) of the paper step by step.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

# OpenMP threads of the oracle sleep instead of spinning when idle, so that it
# degrades gracefully when other processes share the cores (set before load).
os.environ.setdefault("OMP_WAIT_POLICY", "PASSIVE")

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "cr_oracle.c")
_LIB = os.path.join(_HERE, "libcr_oracle.so")
_lock = threading.Lock()
_lib = None

__all__ = [
    "build_oracle", "shift", "lipschitz", "eta", "residual", "metrics", "Solver",
    "METRIC_NAMES", "num_threads", "papg_jvp", "papg_jvp_multi",
]

METRIC_NAMES = ("kkt", "pri", "comp", "infeas", "gap", "primal", "dual", "fit", "sum_check")


def build_oracle(force: bool = False) -> str:
    """Compile cr_oracle.c with gcc (OpenMP, FP64, no FMA contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        cmd = ["gcc", "-O3", "-std=c11", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
               "-o", _LIB + ".tmp", _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(_LIB + ".tmp", _LIB)
    return _LIB


class _Opts(ctypes.Structure):
    _fields_ = [("gamma", ctypes.c_double), ("L", ctypes.c_double), ("sigma", ctypes.c_double),
                ("tol", ctypes.c_double), ("momentum", ctypes.c_int32), ("restart", ctypes.c_int32),
                ("check_every", ctypes.c_int32), ("pad", ctypes.c_int32), ("restart_tol", ctypes.c_double),
                ("B_theta", ctypes.c_double)]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build_oracle()
            lib = ctypes.CDLL(_LIB)
            dp = ctypes.POINTER(ctypes.c_double)
            i64, i32, d = ctypes.c_int64, ctypes.c_int32, ctypes.c_double
            lib.orc_shift.argtypes = [dp, i64]
            lib.orc_shift.restype = d
            lib.orc_lipschitz.argtypes = [dp, i64, i32, d]
            lib.orc_lipschitz.restype = d
            lib.orc_eta.argtypes = [dp, dp, dp, dp, i64, i32, d, dp, dp]
            lib.orc_eta.restype = None
            lib.orc_residual.argtypes = [dp, dp, dp, i64, i32, dp]
            lib.orc_residual.restype = None
            lib.orc_metrics.argtypes = [dp, dp, dp, dp, dp, dp, i64, i32, d, d, dp]
            lib.orc_metrics.restype = None
            lib.orc_state_init.argtypes = [i64, dp, dp, dp, dp, dp]
            lib.orc_state_init.restype = None
            lib.orc_papg.argtypes = [dp, dp, i64, i32, ctypes.POINTER(_Opts), dp, dp, dp, dp, dp, i64,
                                     dp, dp, dp]
            lib.orc_papg.restype = i64
            lib.orc_papg_jvp.argtypes = [dp, dp, i64, i32, d, d, d, i64, dp, dp, dp, dp]
            lib.orc_papg_jvp.restype = None
            lib.orc_papg_jvp_multi.argtypes = [dp, dp, i64, i32, d, d, d, i64, dp, dp, dp, dp]
            lib.orc_papg_jvp_multi.restype = None
            lib.orc_num_threads.argtypes = []
            lib.orc_num_threads.restype = ctypes.c_int
            lib.orc_set_num_threads.argtypes = [ctypes.c_int]
            lib.orc_set_num_threads.restype = None
            _lib = lib
    return _lib


def _p(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def num_threads() -> int:
    return int(_load().orc_num_threads())


def set_num_threads(t: int) -> None:
    """Threads of the oracle's parallel loops from now on (t >= 1)."""
    _load().orc_set_num_threads(int(t))


def shift(ybar) -> float:
    """Observation shift s that keeps y(gamma) >= 0 (paragraph after Eq. (omega_primal))."""
    yb = _f64(ybar)
    return float(_load().orc_shift(_p(yb), yb.shape[0]))


def lipschitz(X, gamma: float) -> float:
    """L_g = sigma_max(C)^2 / gamma, Eq. (eq:lischitz), with the closed-form bound on sigma_max(C)^2."""
    X = _f64(X)
    return float(_load().orc_lipschitz(_p(X), X.shape[0], X.shape[1], float(gamma)))


def eta(theta, mu, X, h, gamma: float):
    """Step 1 of P-APG at K = N: y = h + A1^T theta + mu, xi = A2^T theta / gamma."""
    theta, mu, X, h = _f64(theta), _f64(mu), _f64(X), _f64(h)
    N, n = X.shape
    y = np.empty(N)
    xi = np.empty((N, n))
    _load().orc_eta(_p(theta), _p(mu), _p(X), _p(h), N, n, float(gamma), _p(y), _p(xi))
    return y, xi


def residual(y, xi, X):
    """(C eta)_p = y_l1 - y_l2 - xi_l2^T (x_l1 - x_l2) for all pairs (N x N, zero diagonal)."""
    y, xi, X = _f64(y), _f64(xi), _f64(X)
    N, n = X.shape
    G = np.empty((N, N))
    _load().orc_residual(_p(y), _p(xi), _p(X), N, n, _p(G))
    return G


def metrics(theta, mu, y, xi, X, h, gamma: float, sigma: float) -> dict:
    theta, mu, y, xi, X, h = map(_f64, (theta, mu, y, xi, X, h))
    N, n = X.shape
    out = np.empty(9)
    _load().orc_metrics(_p(theta), _p(mu), _p(y), _p(xi), _p(X), _p(h), N, n, float(gamma),
                        float(sigma), _p(out))
    return dict(zip(METRIC_NAMES, out.tolist()))


def papg_jvp(X, ybar, gamma: float, L: float, s: float, K: int, dybar, dX):
    """(yhat, d yhat) after K iterations of plain P-APG from Iteration 0, forward-mode along
    (dybar, dX), with gamma, L and the shift s held fixed."""
    X, ybar, dybar, dX = _f64(X), _f64(ybar), _f64(dybar), _f64(dX)
    N, n = X.shape
    yhat = np.empty(N)
    dyhat = np.empty(N)
    _load().orc_papg_jvp(_p(X), _p(ybar), N, n, float(gamma), float(L), float(s), int(K), _p(dybar), _p(dX),
                         _p(yhat), _p(dyhat))
    return yhat, dyhat


def papg_jvp_multi(X, ybar, gamma: float, L: float, s: float, K: int, dybar, dX):
    """papg_jvp for D directions: dybar (D, N), dX (D, N, n).  Returns (yhat (N,), dyhat (D, N)).
    The C routine takes 8 directions per call (memory: 2 N^2 x 8 doubles); the last group is
    padded with zero directions."""
    X, ybar = _f64(X), _f64(ybar)
    dybar = np.asarray(dybar, dtype=np.float64)
    dX = np.asarray(dX, dtype=np.float64)
    N, n = X.shape
    D = dybar.shape[0]
    assert dybar.shape == (D, N) and dX.shape == (D, N, n)
    G = 8
    out = np.empty((D, N))
    yhat = np.empty(N)
    for g0 in range(0, D, G):
        g1 = min(D, g0 + G)
        dyb = np.zeros((N, G))
        dxx = np.zeros((N, n, G))
        dyb[:, :g1 - g0] = dybar[g0:g1].T
        dxx[:, :, :g1 - g0] = np.transpose(dX[g0:g1], (1, 2, 0))
        dyh = np.empty((N, G))
        _load().orc_papg_jvp_multi(_p(X), _p(ybar), N, n, float(gamma), float(L), float(s), int(K), _p(dyb), _p(dxx),
                                   _p(yhat), _p(dyh))
        out[g0:g1] = dyh[:, :g1 - g0].T
    return yhat, out


def data_scale(ybar) -> float:
    yb = np.asarray(ybar, dtype=np.float64)
    return max(1.0, float(yb.max() - yb.min()))


class Solver:
    """P-APG (Fig. 2) on problem (regularize) with every pair dualized (K = N).

    State after ``iterate(k)``: ``theta1`` = theta^(1)_l, ``theta2`` = theta^(2)_{l+1},
    ``mu1``/``mu2`` the multipliers of the y >= 0 rows, ``iters`` = l.
    ``y_hat``/``xi`` are the fitted values (shift removed) and subgradients at theta^(1)_l.
    """

    def __init__(self, X, ybar, gamma: float = 1e-1, L: float | None = None, s: float | None = None,
                 momentum: bool = True, restart: bool = False, check_every: int = 0,
                 theta0=None, mu0=None, restart_tol: float = 0.0, B_theta: float = 0.0):
        self.X = _f64(X)
        self.ybar = _f64(ybar)
        self.N, self.n = self.X.shape
        if self.N < self.n + 1:
            raise ValueError("the paper assumes N >= n + 1")
        self.gamma = float(gamma)
        self.s = shift(self.ybar) if s is None else float(s)
        self.h = self.ybar + self.s
        self.L = lipschitz(self.X, self.gamma) if L is None else float(L)
        self.sigma = data_scale(self.ybar)
        self.momentum = bool(momentum)
        self.restart = bool(restart)
        self.check_every = int(check_every)
        self.restart_tol = float(restart_tol)
        self.B_theta = float(B_theta)   # > 0: Q_2 includes the ball ||lambda||_2 <= B_theta
        N = self.N
        self.P = np.zeros((N, N))
        self.T2 = np.zeros((N, N))
        self.muP = np.zeros(N)
        self.mu2 = np.zeros(N)
        self.scal = np.zeros(4)
        _load().orc_state_init(N, _p(self.P), _p(self.T2), _p(self.muP), _p(self.mu2), _p(self.scal))
        if theta0 is not None:
            # a start other than Iteration 0 of Fig. 2: theta^(1)_0 = theta^(2)_1 = theta0
            th = _f64(theta0).copy()
            np.fill_diagonal(th, 0.0)
            self.P[:] = th
            self.T2[:] = th
        if mu0 is not None:
            self.muP[:] = _f64(mu0)
            self.mu2[:] = _f64(mu0)
        self.y = np.empty(N)
        self.xi_ = np.empty((N, self.n))
        self.m = np.zeros(9)

    def _opts(self, tol):
        return _Opts(self.gamma, self.L, self.sigma, float(tol), int(self.momentum), int(self.restart),
                     int(self.check_every), 0, self.restart_tol, self.B_theta)

    def iterate(self, k: int, tol: float = -1.0) -> int:
        o = self._opts(tol)
        return int(_load().orc_papg(_p(self.X), _p(self.h), self.N, self.n, ctypes.byref(o), _p(self.P),
                                    _p(self.T2), _p(self.muP), _p(self.mu2), _p(self.scal), int(k),
                                    _p(self.y), _p(self.xi_), _p(self.m)))

    def solve(self, tol: float, max_iter: int, check_every: int = 10) -> int:
        self.check_every = check_every
        return self.iterate(max_iter, tol)

    @property
    def iters(self) -> int:
        return int(self.scal[1])

    @property
    def restarts(self) -> int:
        return int(self.scal[3])

    @property
    def theta1(self) -> np.ndarray:
        return self.P

    @property
    def theta2(self) -> np.ndarray:
        return self.T2

    @property
    def mu1(self) -> np.ndarray:
        return self.muP

    @property
    def y_shifted(self) -> np.ndarray:
        return self.y

    @property
    def y_hat(self) -> np.ndarray:
        return self.y - self.s

    @property
    def xi(self) -> np.ndarray:
        return self.xi_

    @property
    def metrics(self) -> dict:
        return dict(zip(METRIC_NAMES, self.m.tolist()))
