"""Thin ctypes binding of libkrr.so (include/krr.h).

Only argument marshalling lives here: every step of Build / Factor / Solve /
Predict runs in the CUDA library.  Tensors (CUDA or CPU) and numpy arrays are
passed as raw pointers; the library tells host and device memory apart.  If
libkrr.so has not been built the import fails loudly -- there is no CPU
fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

try:
    import torch
except ImportError:  # pragma: no cover - torch is part of the supported setup
    torch = None

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libkrr.so")

# krr_status values
OK, EINVAL, ENOMEM, ECUDA, ENOTPD, ENOCONV, ETIMEOUT, ESTATE = range(8)
STATUS_NAMES = {0: "KRR_OK", 1: "KRR_EINVAL", 2: "KRR_ENOMEM", 3: "KRR_ECUDA", 4: "KRR_ENOTPD",
                5: "KRR_ENOCONV", 6: "KRR_ETIMEOUT", 7: "KRR_ESTATE"}
MODES = {"mixed": 0, "fp32": 1}
RULES = {"lambda": 0, "knorm": 1}
KERNELS = {"gaussian": 0, "ibs": 1}
PREC_NAMES = {0: "fp64", 1: "fp32", 2: "fp16", 3: "e4m3", 255: "-"}

# Every symbol include/krr.h declares (checked by the CPU test suite).
EXPORTED = ["krr_default_options", "krr_create", "krr_build_kernel", "krr_factor", "krr_solve",
            "krr_predict", "krr_build_kernel_conf", "krr_predict_conf", "krr_rr_build", "krr_rr_rhs",
            "krr_rr_predict", "krr_get_precision_map", "krr_set_keep_distances", "krr_get_distances",
            "krr_get_kernel", "krr_get_factor", "krr_predict_noalloc", "krr_grad_hyper", "krr_set_profiling",
            "krr_get_profile", "krr_set_wait_budget", "krr_sync", "krr_last_error",
            "krr_destroy", "krr_batch_create", "krr_batch_run", "krr_batch_last_error", "krr_batch_destroy"]
PROF_CLASSES = ["pack", "build", "diag", "trsm", "cast", "update", "solve", "residual", "predict", "update_shared"]


class Options(ctypes.Structure):
    _fields_ = [("tile", ctypes.c_int64), ("mode", ctypes.c_int32), ("allow_fp8", ctypes.c_int32),
                ("eps", ctypes.c_double), ("ir_tol", ctypes.c_double), ("ir_max", ctypes.c_int32),
                ("diag_fp64", ctypes.c_int32), ("wait_budget_ns", ctypes.c_int64), ("prec_rule", ctypes.c_int32),
                ("kernel", ctypes.c_int32), ("lookahead", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class FactorInfo(ctypes.Structure):
    _fields_ = [("nt", ctypes.c_int64), ("tiles_fp32", ctypes.c_int64), ("tiles_fp16", ctypes.c_int64),
                ("tiles_e4m3", ctypes.c_int64), ("factor_bytes", ctypes.c_int64),
                ("bad_tile", ctypes.c_int64), ("bad_column", ctypes.c_int64),
                ("min_pivot", ctypes.c_double)]


class SolveInfo(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int32), ("converged", ctypes.c_int32),
                ("rel_residual", ctypes.c_double), ("history", ctypes.c_double * 32)]


class Profile(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_int64), ("count", ctypes.c_int64 * len(PROF_CLASSES)),
                ("ms", ctypes.c_double * len(PROF_CLASSES)), ("flops", ctypes.c_double * len(PROF_CLASSES)),
                ("bytes", ctypes.c_double * len(PROF_CLASSES))]


class BatchProblem(ctypes.Structure):
    _fields_ = [("G", ctypes.c_void_p), ("n", ctypes.c_int64), ("ldg", ctypes.c_int64),
                ("gamma", ctypes.c_double), ("lam", ctypes.c_double), ("Y", ctypes.c_void_p),
                ("ldy", ctypes.c_int64), ("A", ctypes.c_void_p), ("lda", ctypes.c_int64),
                ("T", ctypes.c_void_p), ("n_test", ctypes.c_int64), ("ldt", ctypes.c_int64),
                ("Yt", ctypes.c_void_p), ("ldyt", ctypes.c_int64)]


class BatchResult(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("tile", ctypes.c_int32), ("rel_residual", ctypes.c_double)]


class KRRError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


_lib = None


def load_library(path: str = LIB_PATH):
    """Load libkrr.so; raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"{path} is missing: build it with `python -c 'import __graft_entry__ as g; "
                          f"g.build()'` (there is no CPU fallback)")
    lib = ctypes.CDLL(path)
    vp, i64, i32, dbl = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_double
    lib.krr_default_options.argtypes = [ctypes.POINTER(Options)]
    lib.krr_default_options.restype = None
    lib.krr_create.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(Options), vp]
    lib.krr_build_kernel.argtypes = [vp, vp, i64, i64, i64, dbl]
    lib.krr_factor.argtypes = [vp, dbl, ctypes.POINTER(FactorInfo)]
    lib.krr_solve.argtypes = [vp, vp, i64, i64, vp, i64, ctypes.POINTER(SolveInfo)]
    lib.krr_predict.argtypes = [vp, vp, i64, i64, vp, i64, i64, vp, i64]
    lib.krr_build_kernel_conf.argtypes = [vp, vp, i64, i64, i64, vp, i64, i64, dbl]
    lib.krr_predict_conf.argtypes = [vp, vp, i64, i64, vp, i64, vp, i64, i64, vp, i64]
    lib.krr_rr_build.argtypes = [vp, vp, i64, i64, i64, vp, i64, i64]
    lib.krr_rr_rhs.argtypes = [vp, vp, i64, i64, vp, i64]
    lib.krr_rr_predict.argtypes = [vp, vp, i64, i64, vp, i64, vp, i64, i64, vp, i64]
    lib.krr_get_precision_map.argtypes = [vp, vp, i64, ctypes.POINTER(i64)]
    lib.krr_set_keep_distances.argtypes = [vp, i32]
    lib.krr_get_distances.argtypes = [vp, vp, i64]
    lib.krr_get_kernel.argtypes = [vp, vp, i64]
    lib.krr_get_factor.argtypes = [vp, vp, i64]
    lib.krr_predict_noalloc.argtypes = [vp, vp, i64, i64, vp, i64, i64, vp, i64]
    lib.krr_grad_hyper.argtypes = [vp, vp, i64, i64, vp, i64, vp, i64, i64, ctypes.POINTER(dbl)]
    lib.krr_set_profiling.argtypes = [vp, i32]
    lib.krr_get_profile.argtypes = [vp, ctypes.POINTER(Profile), i32]
    lib.krr_batch_create.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(Options), vp, i64, i64,
                                     ctypes.POINTER(BatchProblem), i32, i32]
    lib.krr_batch_create.restype = ctypes.c_int
    lib.krr_batch_run.argtypes = [vp, ctypes.POINTER(BatchResult)]
    lib.krr_batch_run.restype = ctypes.c_int
    lib.krr_batch_last_error.argtypes = [vp]
    lib.krr_batch_last_error.restype = ctypes.c_char_p
    lib.krr_batch_destroy.argtypes = [vp]
    lib.krr_batch_destroy.restype = None
    lib.krr_set_wait_budget.argtypes = [vp, i64]
    lib.krr_set_wait_budget.restype = ctypes.c_int
    lib.krr_sync.argtypes = [vp]
    lib.krr_last_error.argtypes = [vp]
    lib.krr_last_error.restype = ctypes.c_char_p
    lib.krr_destroy.argtypes = [vp]
    lib.krr_destroy.restype = None
    for name in ("krr_create", "krr_build_kernel", "krr_factor", "krr_solve", "krr_predict",
                 "krr_build_kernel_conf", "krr_predict_conf", "krr_rr_build", "krr_rr_rhs", "krr_rr_predict",
                 "krr_get_precision_map", "krr_set_keep_distances", "krr_get_distances",
                 "krr_get_kernel", "krr_get_factor", "krr_predict_noalloc", "krr_grad_hyper", "krr_set_profiling",
            "krr_get_profile", "krr_sync"):
        getattr(lib, name).restype = ctypes.c_int
    _lib = lib
    return lib


def default_options() -> Options:
    o = Options()
    load_library().krr_default_options(ctypes.byref(o))
    return o


def _ptr(x):
    """Raw pointer of a torch tensor or numpy array (must be C-contiguous rows)."""
    if torch is not None and isinstance(x, torch.Tensor):
        return x.data_ptr()
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    raise TypeError(f"expected a torch.Tensor or numpy.ndarray, got {type(x)}")


def _ld(x) -> int:
    """Leading dimension (elements) of a row-major 2-D tensor/array."""
    if torch is not None and isinstance(x, torch.Tensor):
        if x.dim() != 2 or x.stride(1) != 1:
            raise ValueError("expected a 2-D tensor with unit column stride")
        return x.stride(0)
    if x.ndim != 2 or x.strides[1] != x.itemsize:
        raise ValueError("expected a 2-D array with unit column stride")
    return x.strides[0] // x.itemsize


def _empty_like_rows(ref, rows, cols):
    if torch is not None and isinstance(ref, torch.Tensor):
        return torch.empty((rows, cols), dtype=torch.float32, device=ref.device)
    return np.empty((rows, cols), dtype=np.float32)


class KRR:
    """One KRR context: Build (Alg. 2), Associate (Alg. 3), Predict (Alg. 4)."""

    def __init__(self, tile: int = 1024, mode: str = "mixed", eps: float | None = None,
                 ir_tol: float | None = None, ir_max: int | None = None, allow_fp8: bool = True,
                 diag_fp64: bool = False, prec_rule: str = "lambda", wait_budget_ns: int | None = None,
                 kernel: str = "gaussian", lookahead: bool = True, stream=None):
        lib = load_library()
        o = default_options()
        o.tile = tile
        o.mode = MODES[mode]
        o.allow_fp8 = int(allow_fp8)
        o.diag_fp64 = int(diag_fp64)
        o.prec_rule = RULES[prec_rule]
        o.kernel = KERNELS[kernel]
        o.lookahead = int(lookahead)
        if wait_budget_ns is not None:
            o.wait_budget_ns = int(wait_budget_ns)
        if eps is not None:
            o.eps = eps
        if ir_tol is not None:
            o.ir_tol = ir_tol
        if ir_max is not None:
            o.ir_max = ir_max
        if stream is None and torch is not None and torch.cuda.is_available():
            stream = torch.cuda.current_stream().cuda_stream
        self._lib = lib
        self._ctx = ctypes.c_void_p()
        st = lib.krr_create(ctypes.byref(self._ctx), ctypes.byref(o), ctypes.c_void_p(stream or 0))
        if st != OK:
            raise KRRError(st, lib.krr_last_error(None).decode())
        self.options = o
        self.n = self.m = None

    # -- plumbing -----------------------------------------------------------
    def _check(self, st):
        if st != OK:
            raise KRRError(st, self._lib.krr_last_error(self._ctx).decode())

    def close(self):
        if self._ctx:
            self._lib.krr_destroy(self._ctx)
            self._ctx = ctypes.c_void_p()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- Alg. 2 ---------------------------------------------------------------
    def build_kernel(self, g, gamma: float, keep_distances: bool = False, conf=None):
        """Alg. 2; ``conf``: n x nc FP32 confounders whose squared distances join
        the genotype distances before the exponential (nc <= 16)."""
        n, m = g.shape
        self._check(self._lib.krr_set_keep_distances(self._ctx, int(keep_distances)))
        if conf is None:
            self._check(self._lib.krr_build_kernel(self._ctx, ctypes.c_void_p(_ptr(g)), n, m, _ld(g), gamma))
        else:
            self._check(self._lib.krr_build_kernel_conf(self._ctx, ctypes.c_void_p(_ptr(g)), n, m, _ld(g),
                                                        ctypes.c_void_p(_ptr(conf)), conf.shape[1], _ld(conf),
                                                        gamma))
        self.n, self.m = n, m

    # -- Alg. 3 ---------------------------------------------------------------
    def factor(self, lam: float) -> dict:
        info = FactorInfo()
        self._check(self._lib.krr_factor(self._ctx, lam, ctypes.byref(info)))
        return {f: getattr(info, f) for f, _ in FactorInfo._fields_}

    def solve(self, y, out=None, raise_on_noconv: bool = True):
        p = y.shape[1]
        a = _empty_like_rows(y, self.n, p) if out is None else out
        info = SolveInfo()
        st = self._lib.krr_solve(self._ctx, ctypes.c_void_p(_ptr(y)), p, _ld(y), ctypes.c_void_p(_ptr(a)),
                                 _ld(a), ctypes.byref(info))
        if st != OK and not (st == ENOCONV and not raise_on_noconv):
            self._check(st)
        d = {"iterations": info.iterations, "converged": int(info.converged),
             "rel_residual": info.rel_residual,
             "history": [info.history[i] for i in range(min(32, info.iterations + 1))]}
        return a, d

    # -- Alg. 4 ---------------------------------------------------------------
    def predict(self, t, a, out=None, conf=None):
        """Alg. 4; ``conf``: the held-out rows' confounders (kernels built with them)."""
        nt_, p = t.shape[0], a.shape[1]
        yt = _empty_like_rows(a, nt_, p) if out is None else out
        if conf is None:
            self._check(self._lib.krr_predict(self._ctx, ctypes.c_void_p(_ptr(t)), nt_, _ld(t),
                                              ctypes.c_void_p(_ptr(a)), _ld(a), p, ctypes.c_void_p(_ptr(yt)),
                                              _ld(yt)))
        else:
            self._check(self._lib.krr_predict_conf(self._ctx, ctypes.c_void_p(_ptr(t)), nt_, _ld(t),
                                                   ctypes.c_void_p(_ptr(conf)), _ld(conf),
                                                   ctypes.c_void_p(_ptr(a)), _ld(a), p, ctypes.c_void_p(_ptr(yt)),
                                                   _ld(yt)))
        return yt

    # -- ridge regression (Sec. IV-A): Gram matrix, X^T Y, predictions --------
    def rr_build(self, x, conf=None):
        """The context's matrix becomes X^T X, X = [x conf] (x: n x m int8)."""
        n, m = x.shape
        nc = 0 if conf is None else conf.shape[1]
        self._check(self._lib.krr_rr_build(self._ctx, ctypes.c_void_p(_ptr(x)), n, m, _ld(x),
                                           ctypes.c_void_p(_ptr(conf) if conf is not None else 0), nc,
                                           _ld(conf) if conf is not None else max(nc, 1)))
        self.n, self.m, self.rr_m, self.rr_nc = m + nc, n, m, nc

    def rr_rhs(self, y, out=None):
        """X^T Y ((m + nc) x p)."""
        p = y.shape[1]
        b = _empty_like_rows(y, self.n, p) if out is None else out
        self._check(self._lib.krr_rr_rhs(self._ctx, ctypes.c_void_p(_ptr(y)), p, _ld(y), ctypes.c_void_p(_ptr(b)),
                                         _ld(b)))
        return b

    def rr_predict(self, t, beta, conf=None, out=None):
        """T beta_g + Ct beta_c for held-out patients."""
        n_t, p = t.shape[0], beta.shape[1]
        yt = _empty_like_rows(beta, n_t, p) if out is None else out
        self._check(self._lib.krr_rr_predict(self._ctx, ctypes.c_void_p(_ptr(t)), n_t, _ld(t),
                                             ctypes.c_void_p(_ptr(conf) if conf is not None else 0),
                                             _ld(conf) if conf is not None else 1, ctypes.c_void_p(_ptr(beta)),
                                             _ld(beta), p, ctypes.c_void_p(_ptr(yt)), _ld(yt)))
        return yt

    # -- hyperparameter gradient (adjoint reusing the factor) ----------------
    def grad_hyper(self, t, yt, a):
        """(loss, d loss/d log gamma, d loss/d log lambda) of the held-out MSE."""
        out = (ctypes.c_double * 3)()
        self._check(self._lib.krr_grad_hyper(self._ctx, ctypes.c_void_p(_ptr(t)), t.shape[0], _ld(t),
                                             ctypes.c_void_p(_ptr(yt)), _ld(yt), ctypes.c_void_p(_ptr(a)),
                                             _ld(a), a.shape[1], out))
        return out[0], out[1], out[2]

    # -- inspection -----------------------------------------------------------
    def precision_map(self) -> np.ndarray:
        nt = ctypes.c_int64()
        self._check(self._lib.krr_get_precision_map(self._ctx, None, 0, ctypes.byref(nt)))
        out = np.empty((nt.value, nt.value), dtype=np.uint8)
        self._check(self._lib.krr_get_precision_map(self._ctx, ctypes.c_void_p(out.ctypes.data), out.size,
                                                    ctypes.byref(nt)))
        return out

    def distances(self, out=None):
        """Squared distances of the lower-triangle tiles (needs keep_distances=True)
        into ``out`` (an n x n host array or device tensor of 4-byte integers;
        its strictly-upper tiles are left as they are), or into a new zeroed
        host uint32 array."""
        if out is None:
            out = np.zeros((self.n, self.n), dtype=np.uint32)
        self._check(self._lib.krr_get_distances(self._ctx, ctypes.c_void_p(_ptr(out)), _ld(out)))
        return out

    def kernel(self, out=None):
        """FP32 kernel matrix of the lower-triangle tiles into ``out`` (an n x n
        host array or device tensor; its strictly-upper tiles are left as they
        are), or into a new zeroed host array."""
        if out is None:
            out = np.zeros((self.n, self.n), dtype=np.float32)
        self._check(self._lib.krr_get_kernel(self._ctx, ctypes.c_void_p(_ptr(out)), _ld(out)))
        return out

    def set_profiling(self, on: bool = True):
        self._check(self._lib.krr_set_profiling(self._ctx, int(on)))

    def profile(self, reset: bool = True) -> dict:
        """Per-class event times (ms), counts, algorithmic flops/bytes and launches."""
        pr = Profile()
        self._check(self._lib.krr_get_profile(self._ctx, ctypes.byref(pr), int(reset)))
        out = {"launches": pr.launches}
        for i, name in enumerate(PROF_CLASSES):
            out[name] = {"count": pr.count[i], "ms": pr.ms[i], "flops": pr.flops[i], "bytes": pr.bytes[i]}
        return out

    def factor_matrix(self) -> np.ndarray:
        """Dense copy of the stored (mixed-precision) factor L, lower triangular."""
        out = np.zeros((self.n, self.n), dtype=np.float32)
        self._check(self._lib.krr_get_factor(self._ctx, ctypes.c_void_p(out.ctypes.data), self.n))
        return out

    def set_wait_budget(self, ns: int):
        """Limit (ns) of every bounded device wait of later launches."""
        self._check(self._lib.krr_set_wait_budget(self._ctx, int(ns)))

    def sync(self):
        self._check(self._lib.krr_sync(self._ctx))


class KRRBatch:
    """Many KRR problems (cohorts x folds x lambdas) captured into one CUDA graph.

    problems: list of dicts with device tensors G (n x m int8), Y (n x p),
    optional T (n_t x m int8), and floats gamma, lam.  Outputs A and Yt are
    allocated here and refreshed by every run().
    """

    def __init__(self, problems, ir_iters: int = 3, autotune: int = 1, tile: int = 1024, stream=None):
        lib = load_library()
        self._lib = lib
        o = default_options()
        o.tile = tile
        o.ir_max = ir_iters
        if stream is None and torch is not None and torch.cuda.is_available():
            stream = torch.cuda.current_stream().cuda_stream
        m = problems[0]["G"].shape[1]
        p = problems[0]["Y"].shape[1]
        self.A, self.Yt = [], []
        arr = (BatchProblem * len(problems))()
        for i, pr in enumerate(problems):
            g, y = pr["G"], pr["Y"]
            a = torch.empty((g.shape[0], p), dtype=torch.float32, device=g.device)
            self.A.append(a)
            t = pr.get("T")
            yt = torch.empty((t.shape[0], p), dtype=torch.float32, device=g.device) if t is not None else None
            self.Yt.append(yt)
            arr[i] = BatchProblem(g.data_ptr(), g.shape[0], _ld(g), pr["gamma"], pr["lam"], y.data_ptr(), _ld(y),
                                  a.data_ptr(), _ld(a), t.data_ptr() if t is not None else None,
                                  t.shape[0] if t is not None else 0, _ld(t) if t is not None else m,
                                  yt.data_ptr() if yt is not None else None, p)
        self._problems = problems  # keep the inputs alive: the graph reads them at every run
        self._arr = arr
        self._bt = ctypes.c_void_p()
        st = lib.krr_batch_create(ctypes.byref(self._bt), ctypes.byref(o), ctypes.c_void_p(stream or 0), m, p,
                                  arr, len(problems), int(autotune))
        if st != OK:
            raise KRRError(st, "krr_batch_create failed: " + lib.krr_batch_last_error(None).decode())
        self.count = len(problems)

    def run(self):
        res = (BatchResult * self.count)()
        st = self._lib.krr_batch_run(self._bt, res)
        if st != OK:
            raise KRRError(st, self._lib.krr_batch_last_error(self._bt).decode())
        return [{"status": r.status, "tile": r.tile, "rel_residual": r.rel_residual} for r in res]

    def close(self):
        if self._bt:
            self._lib.krr_batch_destroy(self._bt)
            self._bt = ctypes.c_void_p()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
