"""GB300 P-APG convex-regression solver: thin Python binding of libcrgpu.so.

The library implements P-APG (Fig. 2 of Aybat & Wang, arXiv:1407.7220) on the
dual of problem (regularize) with every pairwise constraint dualized; see
``include/crgpu.h`` for the C ABI.  This module only marshals arguments
(ctypes): every step of the iteration runs in the CUDA kernels of the
library.  There is no CPU fallback -- if the library is missing or no usable
GPU is present, the calls raise.

Names mirror the C ABI (``cr_create``, ``cr_iterate``, ``cr_solve``,
``cr_objective``, ``cr_kkt_residual``, ``cr_get_solution``, ...).  The
``Solver`` class wraps one handle; ``BatchSolver`` many independent fits;
``AlccSolver`` the ALCC method with its MAPG inner solver (Sec. II-D) on the
full problem; ``convex_fit`` the differentiable fit (autograd);
``problem_constants`` the host-side constants.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

__all__ = [
    "CrError", "Options", "Solver", "AlccOptions", "AlccSolver", "BlockSolver", "problem_constants", "lib", "library_path",
    "exported_symbols",
    "THETA_F32", "THETA_BF16", "THETA_F16", "THETA_F64", "DRIVER_AUTO", "DRIVER_PERSISTENT", "DRIVER_PHASES",
    "PAIR_AUTO", "PAIR_CUDA_CORES", "PAIR_TENSOR_CORES",
    "CR_OK", "CR_NOT_CONVERGED",
]

HERE = os.path.dirname(os.path.abspath(__file__))
library_path = os.path.join(HERE, "libcrgpu.so")

CR_OK, CR_NOT_CONVERGED, CR_EINVAL, CR_ENOMEM, CR_ECUDA, CR_ETIMEOUT, CR_ENUMERIC, CR_ESTATE = 0, 1, -1, -2, -3, -4, -5, -6
THETA_F32, THETA_BF16, THETA_F16, THETA_F64 = 0, 1, 2, 3
DRIVER_AUTO, DRIVER_PERSISTENT, DRIVER_PHASES = 0, 1, 2
PAIR_AUTO, PAIR_CUDA_CORES, PAIR_TENSOR_CORES = 0, 1, 2
_DTYPES = {"f32": THETA_F32, "fp32": THETA_F32, "float32": THETA_F32, "bf16": THETA_BF16,
           "bfloat16": THETA_BF16, "f16": THETA_F16, "fp16": THETA_F16, "float16": THETA_F16,
           "f64": THETA_F64, "fp64": THETA_F64, "float64": THETA_F64}

# the C-ABI entry points declared in include/crgpu.h
exported_symbols = (
    "cr_options_default", "cr_create", "cr_create_device", "cr_reset", "cr_iterate", "cr_solve",
    "cr_objective", "cr_kkt_residual", "cr_get_solution", "cr_get_info", "cr_destroy",
    "cr_status_str", "cr_last_error", "cr_profile", "cr_get_device_state", "cr_kkt_residual_noalloc",
    "cr_batch_create", "cr_batch_solve", "cr_batch_iterate", "cr_batch_reset", "cr_batch_instance",
    "cr_batch_info", "cr_batch_destroy", "cr_batch_last_error", "cr_backward", "cr_get_engine",
    "cr_alcc_options_default", "cr_alcc_create", "cr_alcc_iterate", "cr_alcc_solve", "cr_alcc_metrics",
    "cr_alcc_info", "cr_problem_constants", "cr_batch_stats", "cr_promote", "cr_blocks_create",
    "cr_blocks_iterate", "cr_blocks_solution", "cr_get_solution_device", "cr_batch_tuning",
)
PROFILE_PAIR, PROFILE_FOLD, PROFILE_KKT, PROFILE_PERSISTENT = 0, 1, 2, 3


class Options(ctypes.Structure):
    """Mirror of ``cr_options``."""
    _fields_ = [
        ("gamma", ctypes.c_double), ("L", ctypes.c_double), ("shift", ctypes.c_double),
        ("theta_dtype", ctypes.c_int32), ("stochastic_round", ctypes.c_int32),
        ("kkt_every", ctypes.c_int32), ("momentum", ctypes.c_int32), ("restart", ctypes.c_int32),
        ("driver", ctypes.c_int32), ("grid", ctypes.c_int32), ("fp16_exponent", ctypes.c_int32),
        ("seed", ctypes.c_uint64), ("stream", ctypes.c_void_p), ("barrier_timeout_ms", ctypes.c_int32),
        ("test_barrier_extra", ctypes.c_int32), ("profile", ctypes.c_int32), ("record_every", ctypes.c_int32),
        ("pair_engine", ctypes.c_int32), ("batch_stage_rows", ctypes.c_int32), ("reserved", ctypes.c_int32 * 2),
        ("restart_tol", ctypes.c_double), ("B_theta", ctypes.c_double), ("promote_at", ctypes.c_double),
    ]


class AlccOptions(ctypes.Structure):
    """Mirror of ``cr_alcc_options``."""
    _fields_ = [
        ("mu1_scale", ctypes.c_double), ("tau1_rel", ctypes.c_double), ("alpha1_rel", ctypes.c_double),
        ("c", ctypes.c_double), ("kappa", ctypes.c_double), ("lmax_cap", ctypes.c_int64),
        ("fixed_inner", ctypes.c_int64), ("launch_iters", ctypes.c_int64), ("mu_max_scale", ctypes.c_double),
        ("reserved", ctypes.c_double * 3),
    ]


class CrError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"crgpu status {status}: {msg}")
        self.status = status


_lock = threading.Lock()
_lib = None


def lib():
    """Load libcrgpu.so (built by ``__graft_entry__.build()`` / ``python -m paper_1407_7220_gb300._build``)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(library_path):
                raise RuntimeError(f"{library_path} is missing: build the CUDA library first "
                                   "(python -m paper_1407_7220_gb300._build)")
            L = ctypes.CDLL(library_path)
            H = ctypes.c_void_p
            dp = ctypes.POINTER(ctypes.c_double)
            fp = ctypes.c_void_p
            i64p = ctypes.POINTER(ctypes.c_int64)
            L.cr_options_default.argtypes = [ctypes.POINTER(Options)]
            L.cr_options_default.restype = None
            L.cr_create.argtypes = [dp, dp, ctypes.c_int64, ctypes.c_int32, ctypes.POINTER(Options),
                                    ctypes.POINTER(H)]
            L.cr_create_device.argtypes = [fp, fp, ctypes.c_int64, ctypes.c_int32, ctypes.POINTER(Options),
                                           ctypes.POINTER(H)]
            L.cr_reset.argtypes = [H]
            L.cr_blocks_create.argtypes = [dp, dp, ctypes.c_int64, ctypes.c_int32, ctypes.POINTER(ctypes.c_int32),
                                           ctypes.POINTER(Options), ctypes.c_int32, ctypes.POINTER(H)]
            L.cr_blocks_iterate.argtypes = [H, ctypes.c_int64]
            L.cr_blocks_solution.argtypes = [H, dp, dp]
            for name in ("cr_blocks_create", "cr_blocks_iterate", "cr_blocks_solution"):
                getattr(L, name).restype = ctypes.c_int
            L.cr_promote.argtypes = [H, ctypes.c_int32]
            L.cr_promote.restype = ctypes.c_int
            L.cr_iterate.argtypes = [H, ctypes.c_int64]
            L.cr_solve.argtypes = [H, ctypes.c_double, ctypes.c_int64, i64p]
            L.cr_objective.argtypes = [H, dp, dp, dp]
            L.cr_kkt_residual.argtypes = [H, dp, dp, dp]
            L.cr_get_solution.argtypes = [H, dp, dp]
            L.cr_get_solution_device.argtypes = [H, ctypes.c_void_p, ctypes.c_void_p]
            L.cr_get_solution_device.restype = ctypes.c_int
            L.cr_get_info.argtypes = [H, i64p, i64p, dp, dp]
            L.cr_get_engine.argtypes = [H, ctypes.POINTER(ctypes.c_int32)]
            vpp = ctypes.POINTER(ctypes.c_void_p)
            L.cr_get_device_state.argtypes = [H, vpp, i64p, vpp, vpp, vpp, vpp, dp]
            L.cr_get_device_state.restype = ctypes.c_int
            L.cr_kkt_residual_noalloc.argtypes = [ctypes.c_int64, ctypes.c_int32, fp, ctypes.c_int64, fp, fp, fp, fp,
                                                  ctypes.c_double, fp, fp]
            L.cr_kkt_residual_noalloc.restype = ctypes.c_int
            L.cr_batch_create.argtypes = [ctypes.c_int32, i64p, ctypes.POINTER(ctypes.c_int32),
                                          ctypes.POINTER(dp), ctypes.POINTER(dp), ctypes.POINTER(Options),
                                          ctypes.POINTER(H)]
            L.cr_batch_solve.argtypes = [H, ctypes.c_double, ctypes.c_int64, i64p]
            L.cr_batch_iterate.argtypes = [H, ctypes.c_int64]
            L.cr_batch_reset.argtypes = [H]
            L.cr_batch_instance.argtypes = [H, ctypes.c_int32, ctypes.POINTER(H)]
            L.cr_batch_info.argtypes = [H, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32), i64p]
            L.cr_batch_stats.argtypes = [H, ctypes.POINTER(ctypes.c_int32), i64p, i64p, ctypes.POINTER(ctypes.c_int32),
                                         ctypes.POINTER(ctypes.c_double)]
            L.cr_batch_stats.restype = ctypes.c_int
            i32p = ctypes.POINTER(ctypes.c_int32)
            L.cr_batch_tuning.argtypes = [H, ctypes.c_int32, i32p, i32p, i32p, i32p, i32p, ctypes.POINTER(ctypes.c_double)]
            L.cr_batch_tuning.restype = ctypes.c_int
            L.cr_batch_destroy.argtypes = [H]
            L.cr_batch_destroy.restype = None
            L.cr_batch_last_error.argtypes = [H]
            L.cr_batch_last_error.restype = ctypes.c_char_p
            for name in ("cr_batch_create", "cr_batch_solve", "cr_batch_iterate", "cr_batch_reset",
                         "cr_batch_instance", "cr_batch_info"):
                getattr(L, name).restype = ctypes.c_int
            L.cr_backward.argtypes = [H, fp, fp, fp]
            L.cr_backward.restype = ctypes.c_int
            L.cr_alcc_options_default.argtypes = [ctypes.POINTER(AlccOptions)]
            L.cr_alcc_options_default.restype = None
            L.cr_alcc_create.argtypes = [dp, dp, ctypes.c_int64, ctypes.c_int32, ctypes.POINTER(Options),
                                         ctypes.POINTER(AlccOptions), ctypes.POINTER(H)]
            L.cr_alcc_iterate.argtypes = [H, ctypes.c_int64, i64p]
            L.cr_alcc_solve.argtypes = [H, ctypes.c_double, ctypes.c_int64, i64p]
            L.cr_alcc_metrics.argtypes = [H, dp, dp, dp, dp]
            L.cr_alcc_info.argtypes = [H, i64p, i64p, dp, i64p]
            for name in ("cr_alcc_create", "cr_alcc_iterate", "cr_alcc_solve", "cr_alcc_metrics", "cr_alcc_info"):
                getattr(L, name).restype = ctypes.c_int
            L.cr_problem_constants.argtypes = [dp, dp, ctypes.c_int64, ctypes.c_int32, ctypes.c_double, dp, dp, dp, dp]
            L.cr_problem_constants.restype = ctypes.c_int
            L.cr_profile.argtypes = [H, ctypes.c_int32, dp, i64p]
            L.cr_profile.restype = ctypes.c_int
            L.cr_destroy.argtypes = [H]
            L.cr_destroy.restype = None
            L.cr_status_str.argtypes = [ctypes.c_int]
            L.cr_status_str.restype = ctypes.c_char_p
            L.cr_last_error.argtypes = [H]
            L.cr_last_error.restype = ctypes.c_char_p
            for name in ("cr_create", "cr_create_device", "cr_reset", "cr_iterate", "cr_solve", "cr_objective",
                         "cr_kkt_residual", "cr_get_solution", "cr_get_info"):
                getattr(L, name).restype = ctypes.c_int
            _lib = L
    return _lib


def default_options(**kw) -> Options:
    o = Options()
    lib().cr_options_default(ctypes.byref(o))
    for k, v in kw.items():
        if k == "theta_dtype" and isinstance(v, str):
            v = _DTYPES[v.lower()]
        if not hasattr(o, k):
            raise TypeError(f"unknown option {k!r}")
        setattr(o, k, v)
    return o


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


class Solver:
    """One problem instance on the GPU (a ``cr_handle``).

    X: (N, n) array, ybar: (N,) array -- host numpy arrays (copied as FP64) or
    CUDA torch tensors (copied as FP32 via ``cr_create_device``).  Keyword
    arguments set ``cr_options`` fields (``gamma``, ``theta_dtype`` ('f32',
    'bf16', 'f16'), ``stochastic_round``, ``kkt_every``, ``momentum``,
    ``restart``, ``driver``, ``grid``, ``L``, ``shift``, ``stream`` ...).
    """

    def __init__(self, X, ybar, **opts):
        self._h = ctypes.c_void_p()
        L = lib()
        o = default_options(**opts)
        self.options = o
        if hasattr(X, "is_cuda") and X.is_cuda:
            Xt = X.contiguous().float()
            yt = ybar.contiguous().float()
            N, n = int(Xt.shape[0]), int(Xt.shape[1])
            st = L.cr_create_device(ctypes.c_void_p(Xt.data_ptr()), ctypes.c_void_p(yt.data_ptr()), N, n,
                                    ctypes.byref(o), ctypes.byref(self._h))
        else:
            Xa = np.ascontiguousarray(np.asarray(X, dtype=np.float64))
            ya = np.ascontiguousarray(np.asarray(ybar, dtype=np.float64))
            if Xa.ndim != 2 or ya.shape != (Xa.shape[0],):
                raise ValueError("X must be (N, n) and ybar (N,)")
            N, n = Xa.shape
            st = L.cr_create(_dptr(Xa), _dptr(ya), N, n, ctypes.byref(o), ctypes.byref(self._h))
        if st != CR_OK:
            raise CrError(st, L.cr_last_error(None).decode())
        self.N, self.n = int(N), int(n)

    # -- helpers ---------------------------------------------------------
    def _check(self, st: int, allow=(CR_OK,)):
        if st not in allow:
            raise CrError(st, lib().cr_last_error(self._h).decode())
        return st

    @property
    def handle(self):
        return self._h

    def close(self):
        if self._h:
            lib().cr_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # -- C ABI -----------------------------------------------------------
    def reset(self):
        self._check(lib().cr_reset(self._h))

    def iterate(self, k: int):
        self._check(lib().cr_iterate(self._h, int(k)))

    def promote(self, theta_dtype="f32"):
        """cr_promote: continue the iteration with FP32 multipliers (from BF16 or FP16)."""
        v = _DTYPES[theta_dtype.lower()] if isinstance(theta_dtype, str) else int(theta_dtype)
        self._check(lib().cr_promote(self._h, v))
        self.options.theta_dtype = v

    def solve(self, tol: float, max_iter: int) -> tuple[bool, int]:
        done = ctypes.c_int64()
        st = self._check(lib().cr_solve(self._h, float(tol), int(max_iter), ctypes.byref(done)),
                         (CR_OK, CR_NOT_CONVERGED))
        return st == CR_OK, int(done.value)

    def objective(self) -> dict:
        p, d, g = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        self._check(lib().cr_objective(self._h, ctypes.byref(p), ctypes.byref(d), ctypes.byref(g)))
        return {"primal": p.value, "dual": d.value, "gap": g.value}

    def kkt_residual(self) -> dict:
        k, i, g = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        self._check(lib().cr_kkt_residual(self._h, ctypes.byref(k), ctypes.byref(i), ctypes.byref(g)))
        return {"kkt": k.value, "infeas_norm": i.value, "gap_norm": g.value}

    def solution(self):
        y = np.empty(self.N)
        xi = np.empty((self.N, self.n))
        self._check(lib().cr_get_solution(self._h, _dptr(y), _dptr(xi)))
        return y, xi

    def solution_device(self, yhat=None, xi=None):
        """cr_get_solution_device: the fit into device float64 torch tensors (N,) and (N, n)."""
        for t, shape in ((yhat, (self.N,)), (xi, (self.N, self.n))):
            if t is not None:
                assert t.is_cuda and t.dtype == __import__("torch").float64 and t.is_contiguous()
                assert tuple(t.shape) == shape
        self._check(lib().cr_get_solution_device(self._h, ctypes.c_void_p(yhat.data_ptr() if yhat is not None else 0),
                                                 ctypes.c_void_p(xi.data_ptr() if xi is not None else 0)))

    def info(self) -> dict:
        it, rs = ctypes.c_int64(), ctypes.c_int64()
        Lc, s = ctypes.c_double(), ctypes.c_double()
        self._check(lib().cr_get_info(self._h, ctypes.byref(it), ctypes.byref(rs), ctypes.byref(Lc), ctypes.byref(s)))
        eng = ctypes.c_int32()
        self._check(lib().cr_get_engine(self._h, ctypes.byref(eng)))
        return {"iters": it.value, "restarts": rs.value, "L": Lc.value, "shift": s.value,
                "engine": "tensor_cores" if eng.value == PAIR_TENSOR_CORES else "cuda_cores"}

    def backward(self, dL_dyhat, dL_dybar, dL_dX):
        """Reverse mode through the recorded iterations; device float32 torch tensors (N,), (N,), (N, n)."""
        for t in (dL_dyhat, dL_dybar, dL_dX):
            assert t.is_cuda and t.dtype.is_floating_point and t.is_contiguous()
        self._check(lib().cr_backward(self._h, ctypes.c_void_p(dL_dyhat.data_ptr()),
                                      ctypes.c_void_p(dL_dybar.data_ptr()), ctypes.c_void_p(dL_dX.data_ptr())))

    def profile(self, kind: int) -> tuple[float, int]:
        """(summed device ms, launches) of one kernel kind since the last read (needs profile=1)."""
        ms, n = ctypes.c_double(), ctypes.c_int64()
        self._check(lib().cr_profile(self._h, int(kind), ctypes.byref(ms), ctypes.byref(n)))
        return ms.value, n.value

    def device_state(self) -> dict:
        """Device addresses of the current iterate (see cr_get_device_state); no copy."""
        th, X, y, xi, mu = (ctypes.c_void_p() for _ in range(5))
        ld, sg = ctypes.c_int64(), ctypes.c_double()
        self._check(lib().cr_get_device_state(self._h, ctypes.byref(th), ctypes.byref(ld), ctypes.byref(X),
                                              ctypes.byref(y), ctypes.byref(xi), ctypes.byref(mu), ctypes.byref(sg)))
        return {"theta": th.value, "ld": ld.value, "X": X.value, "y": y.value, "xi": xi.value, "mu": mu.value,
                "sigma": sg.value}


def problem_constants(X, ybar, gamma: float) -> dict:
    """cr_problem_constants: L, shift, sigma_max^2(A_1), sigma_max^2(A_2) computed on the host."""
    Xa = np.ascontiguousarray(np.asarray(X, dtype=np.float64))
    ya = np.ascontiguousarray(np.asarray(ybar, dtype=np.float64))
    if Xa.ndim != 2 or ya.shape != (Xa.shape[0],):
        raise ValueError("X must be (N, n) and ybar (N,)")
    out = [ctypes.c_double() for _ in range(4)]
    st = lib().cr_problem_constants(_dptr(Xa), _dptr(ya), Xa.shape[0], Xa.shape[1], float(gamma),
                                    *(ctypes.byref(v) for v in out))
    if st != CR_OK:
        raise CrError(st, lib().cr_last_error(None).decode())
    return dict(zip(("L", "shift", "sigma2_A1", "sigma2_A2"), (v.value for v in out)))


class AlccSolver(Solver):
    """ALCC with the MAPG inner solver on the full problem (Sec. II-D; ``cr_alcc_*``).

    X, ybar: host arrays.  Keyword arguments set ``cr_alcc_options`` fields (``mu1_scale``,
    ``tau1_rel``, ``alpha1_rel``, ``c``, ``kappa``, ``lmax_cap``, ``fixed_inner``,
    ``launch_iters``) or ``cr_options`` fields (``gamma``, ``grid``, ``stream``, ``profile`` ...).
    ``solution()``, ``device_state()``, ``reset()`` and ``profile()`` are those of ``Solver``.
    """

    def __init__(self, X, ybar, **opts):
        self._h = ctypes.c_void_p()
        L = lib()
        a = AlccOptions()
        L.cr_alcc_options_default(ctypes.byref(a))
        rest = {}
        for k, v in opts.items():
            if hasattr(a, k) and k != "reserved":
                setattr(a, k, v)
            else:
                rest[k] = v
        o = default_options(**rest)
        self.options, self.alcc_options = o, a
        Xa = np.ascontiguousarray(np.asarray(X, dtype=np.float64))
        ya = np.ascontiguousarray(np.asarray(ybar, dtype=np.float64))
        if Xa.ndim != 2 or ya.shape != (Xa.shape[0],):
            raise ValueError("X must be (N, n) and ybar (N,)")
        N, n = Xa.shape
        st = L.cr_alcc_create(_dptr(Xa), _dptr(ya), N, n, ctypes.byref(o), ctypes.byref(a), ctypes.byref(self._h))
        if st != CR_OK:
            raise CrError(st, L.cr_last_error(None).decode())
        self.N, self.n = int(N), int(n)

    def iterate(self, k: int) -> list[int]:
        """k outer iterations; returns the MAPG iterations of each."""
        inner = (ctypes.c_int64 * max(int(k), 1))()
        self._check(lib().cr_alcc_iterate(self._h, int(k), inner))
        return [int(v) for v in inner[:int(k)]]

    def solve(self, tol: float, max_outer: int) -> tuple[bool, int]:
        done = ctypes.c_int64()
        st = self._check(lib().cr_alcc_solve(self._h, float(tol), int(max_outer), ctypes.byref(done)),
                         (CR_OK, CR_NOT_CONVERGED))
        return st == CR_OK, int(done.value)

    def metrics(self) -> dict:
        v = [ctypes.c_double() for _ in range(4)]
        self._check(lib().cr_alcc_metrics(self._h, *(ctypes.byref(x) for x in v)))
        return dict(zip(("kkt", "stat", "pri", "comp"), (x.value for x in v)))

    def info(self) -> dict:
        o, it, lm = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        mu = ctypes.c_double()
        self._check(lib().cr_alcc_info(self._h, ctypes.byref(o), ctypes.byref(it), ctypes.byref(mu), ctypes.byref(lm)))
        return {"outer": o.value, "inner_total": it.value, "mu": mu.value, "lmax_next": lm.value}


class BlockSolver(Solver):
    """P-APG with the points partitioned into blocks (Sec. II-A; ``cr_blocks_*``).

    blocks: list of index arrays (a partition of range(N)) or an (N,) array of block ids.
    inner_iters: inner P-APG iterations (even) per outer iteration, Step 1 of the block problems.
    Keyword arguments set ``cr_options`` (``gamma``, ``L`` ...); FP64 multipliers throughout."""

    def __init__(self, X, ybar, blocks, inner_iters: int = 100, **opts):
        self._h = ctypes.c_void_p()
        L = lib()
        o = default_options(**opts)
        self.options = o
        Xa = np.ascontiguousarray(np.asarray(X, dtype=np.float64))
        ya = np.ascontiguousarray(np.asarray(ybar, dtype=np.float64))
        N, n = Xa.shape
        if isinstance(blocks, (list, tuple)):
            ids = np.empty(N, dtype=np.int32)
            for i, b in enumerate(blocks):
                ids[np.asarray(b, dtype=np.int64)] = i
        else:
            ids = np.ascontiguousarray(np.asarray(blocks, dtype=np.int32))
        self._ids = ids
        st = L.cr_blocks_create(_dptr(Xa), _dptr(ya), N, n, ids.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                ctypes.byref(o), int(inner_iters), ctypes.byref(self._h))
        if st != CR_OK:
            raise CrError(st, L.cr_last_error(None).decode())
        self.N, self.n = int(N), int(n)

    def iterate(self, k: int):
        self._check(lib().cr_blocks_iterate(self._h, int(k)))

    def solution(self):
        y = np.empty(self.N)
        xi = np.empty((self.N, self.n))
        self._check(lib().cr_blocks_solution(self._h, _dptr(y), _dptr(xi)))
        return y, xi

    def info(self) -> dict:
        it = ctypes.c_int64()
        Lc, s = ctypes.c_double(), ctypes.c_double()
        self._check(lib().cr_get_info(self._h, ctypes.byref(it), None, ctypes.byref(Lc), ctypes.byref(s)))
        return {"iters": it.value, "L": Lc.value, "shift": s.value}


class _Member(Solver):
    """A batch member's handle (owned by the batch; read-only use)."""

    def __init__(self, h, N, n, opts):
        self._h = h
        self.N, self.n = N, n
        self.options = opts

    def close(self):
        self._h = ctypes.c_void_p()


class BatchSolver:
    """Many independent fits in one persistent launch (``cr_batch_*``).

    ``instances``: list of (X (N_i x n_i), ybar (N_i,)) host arrays.  Keyword arguments
    set ``cr_options`` shared by all members (``grid`` > 0 fixes the work granularity
    factor; 0 lets the autotuner pick it)."""

    def __init__(self, instances, **opts):
        L = lib()
        o = default_options(**opts)
        self.options = o
        self._keep = []
        B = len(instances)
        Ns = (ctypes.c_int64 * B)()
        ns = (ctypes.c_int32 * B)()
        Xs = (ctypes.POINTER(ctypes.c_double) * B)()
        ys = (ctypes.POINTER(ctypes.c_double) * B)()
        self.sizes = []
        for i, (X, yb) in enumerate(instances):
            Xa = np.ascontiguousarray(np.asarray(X, dtype=np.float64))
            ya = np.ascontiguousarray(np.asarray(yb, dtype=np.float64))
            self._keep += [Xa, ya]
            Ns[i], ns[i] = Xa.shape
            Xs[i] = _dptr(Xa)
            ys[i] = _dptr(ya)
            self.sizes.append(Xa.shape)
        self._h = ctypes.c_void_p()
        st = L.cr_batch_create(B, Ns, ns, Xs, ys, ctypes.byref(o), ctypes.byref(self._h))
        if st != CR_OK:
            raise CrError(st, L.cr_last_error(None).decode())
        self.B = B

    def _check(self, st, allow=(CR_OK,)):
        if st not in allow:
            raise CrError(st, lib().cr_batch_last_error(self._h).decode())
        return st

    def iterate(self, k: int):
        self._check(lib().cr_batch_iterate(self._h, int(k)))

    def solve(self, tol: float, max_iter: int) -> int:
        c = ctypes.c_int64()
        self._check(lib().cr_batch_solve(self._h, float(tol), int(max_iter), ctypes.byref(c)), (CR_OK, CR_NOT_CONVERGED))
        return int(c.value)

    def reset(self):
        self._check(lib().cr_batch_reset(self._h))

    def member(self, i: int) -> Solver:
        h = ctypes.c_void_p()
        self._check(lib().cr_batch_instance(self._h, int(i), ctypes.byref(h)))
        N, n = self.sizes[i]
        return _Member(h, N, n, self.options)

    def info(self) -> dict:
        f, g, it = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int64()
        self._check(lib().cr_batch_info(self._h, ctypes.byref(f), ctypes.byref(g), ctypes.byref(it)))
        return {"factor": f.value, "grid": g.value, "iters": it.value}

    def stats(self) -> dict:
        """cr_batch_stats: whether the CUDA graph is live, launches of each kind, autotuner timings."""
        live, nt = ctypes.c_int32(), ctypes.c_int32()
        gl, dl = ctypes.c_int64(), ctypes.c_int64()
        ms = (ctypes.c_double * 8)()
        self._check(lib().cr_batch_stats(self._h, ctypes.byref(live), ctypes.byref(gl), ctypes.byref(dl),
                                         ctypes.byref(nt), ms))
        return {"graph_live": bool(live.value), "graph_launches": gl.value, "direct_launches": dl.value,
                "tuned": nt.value, "tune_ms": [ms[i] for i in range(min(nt.value, 8))]}

    def tuning(self) -> dict:
        """cr_batch_tuning: the tile shape and granularity in use and every autotuner candidate."""
        cnt, rows, fac = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
        cr = (ctypes.c_int32 * 16)()
        cf = (ctypes.c_int32 * 16)()
        cm = (ctypes.c_double * 16)()
        self._check(lib().cr_batch_tuning(self._h, 16, ctypes.byref(cnt), ctypes.byref(rows), ctypes.byref(fac),
                                          cr, cf, cm))
        n = min(cnt.value, 16)
        return {"stage_rows": rows.value, "factor": fac.value,
                "candidates": [{"stage_rows": cr[i], "factor": cf[i], "ms": cm[i]} for i in range(n)]}

    def close(self):
        if getattr(self, "_h", None):
            lib().cr_batch_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def convex_fit(X, ybar, iters: int, record_every: int = 50, **opts):
    """Differentiable fitted values: yhat = P-APG(X, ybar) after ``iters`` iterations.

    X (N, n) and ybar (N,) are CUDA tensors; the result is a CUDA tensor of ybar's dtype.
    Backward runs ``cr_backward`` (reverse mode through the unrolled iterations, checkpoint
    every ``record_every``), giving dLoss/dX and dLoss/dybar.  gamma, L and the shift are
    held fixed; plain P-APG (restart = 0).  Extra keyword arguments are ``cr_options``."""
    import torch

    class _ConvexFit(torch.autograd.Function):
        @staticmethod
        def forward(ctx, X_, y_):
            s = Solver(X_.detach(), y_.detach(), record_every=int(record_every), restart=0, **opts)
            s.iterate(int(iters))
            yhat = torch.empty(X_.shape[0], dtype=torch.float64, device=y_.device)
            s.solution_device(yhat)   # device to device, no host round trip
            ctx.solver = s
            ctx.meta = (X_.shape, X_.dtype, y_.dtype)
            return yhat.to(y_.dtype)

        @staticmethod
        def backward(ctx, gy):
            shape, xdt, ydt = ctx.meta
            u = gy.detach().contiguous().to(torch.float32)
            dyb = torch.empty_like(u)
            dX = torch.empty(tuple(shape), dtype=torch.float32, device=u.device)
            ctx.solver.backward(u, dyb, dX)
            return dX.to(xdt), dyb.to(ydt)

    return _ConvexFit.apply(X, ybar)
