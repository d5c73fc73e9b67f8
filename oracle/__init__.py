"""Plain CPU oracle for Gaussian-kernel ridge regression on genotypes.

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  The product path
(the CUDA library and its binding) never imports it and shares no code with it.

Everything here is the plain definition of what the method computes, in
int64 / IEEE double:

* Alg. 2 / Alg. 5 (Build with the Gaussian kernel): ``d_ij = sum_k (g_ik -
  g_jk)^2`` term by term, ``K_ij = exp(-gamma d_ij)``.
* Alg. 3 (Associate): Cholesky of ``K + alpha I`` and forward/backward
  substitution for every phenotype column.
* Alg. 4 (Predict): Build(gamma, T, G) then ``P_r = K_test W``.
* The gradient of the held-out mean-squared error with respect to log gamma
  and log lambda, from the adjoint closed form (the paper has no gradient;
  the formula is derived in ``hyper_gradient``'s docstring).

Large cases (the 16384-row subproblem of the N = 131072 workload, the
gradient at N = 16384) would take the plain loops many minutes on the host,
so the functions that carry the O(N^2 M) Gram product and the O(N^3)
factorisation also take ``method="lapack"``: the same definitions with a
library primitive as the step -- the Gram product G1 G2^T as a float64
matrix product (every partial sum is an integer below 2^53, so it is exact),
LAPACK's Cholesky and triangular solves in float64.  The tests pin each of
them against the plain loops (equal integers, and agreement to float64
rounding).

Pins (tests/test_oracle_*.py) tie each function to something other than
itself: brute force on tiny inputs, the paper's 3x2 worked example, closed
forms (gamma = 0, K = I, lambda -> infinity, min(i,j) Cholesky), invariants
(symmetry, K_ii = 1, L L^T reconstruction, the predict identity) and central
finite differences for the gradient.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "krr_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

_i64p = ctypes.POINTER(ctypes.c_int64)
_f64p = ctypes.POINTER(ctypes.c_double)
_i8p = ctypes.POINTER(ctypes.c_int8)


def build(force: bool = False) -> str:
    """Compile the C oracle into ``oracle/liboracle.so`` (gcc, OpenMP if available)."""
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    base = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            lib.oracle_num_threads.restype = ctypes.c_int
            for name in ("oracle_sqdist_bruteforce", "oracle_sqdist_gram"):
                f = getattr(lib, name)
                f.restype = None
                f.argtypes = [_i8p, ctypes.c_int64, ctypes.c_int64, _i8p, ctypes.c_int64,
                              ctypes.c_int64, ctypes.c_int64, _i64p]
            lib.oracle_gaussian_kernel.restype = None
            lib.oracle_gaussian_kernel.argtypes = [_i64p, ctypes.c_int64, ctypes.c_double, _f64p]
            lib.oracle_cholesky.restype = ctypes.c_int64
            lib.oracle_cholesky.argtypes = [_f64p, ctypes.c_int64]
            for name in ("oracle_forward_subst", "oracle_backward_subst"):
                f = getattr(lib, name)
                f.restype = None
                f.argtypes = [_f64p, ctypes.c_int64, _f64p, ctypes.c_int64]
            lib.oracle_matmul.restype = None
            lib.oracle_matmul.argtypes = [_f64p, ctypes.c_int64, ctypes.c_int64, _f64p,
                                          ctypes.c_int64, _f64p]
            lib.oracle_ibs_count.restype = None
            lib.oracle_ibs_count.argtypes = [_i8p, ctypes.c_int64, ctypes.c_int64, _i8p, ctypes.c_int64,
                                             ctypes.c_int64, ctypes.c_int64, _i64p]
            lib.oracle_conf_sqdist.restype = None
            lib.oracle_conf_sqdist.argtypes = [_f64p, ctypes.c_int64, ctypes.c_int64, _f64p, ctypes.c_int64,
                                               ctypes.c_int64, ctypes.c_int64, _f64p]
            lib.oracle_kernel_rows.restype = None
            lib.oracle_kernel_rows.argtypes = [_i8p, ctypes.c_int64, _i64p, ctypes.c_int64, _i8p,
                                               ctypes.c_int64, ctypes.c_int64, ctypes.c_int64,
                                               ctypes.c_double, _f64p]
            _lib = lib
    return _lib


def num_threads() -> int:
    """Threads the oracle's OpenMP loops use."""
    return int(_load().oracle_num_threads())


def _geno(g) -> np.ndarray:
    g = np.ascontiguousarray(np.asarray(g), dtype=np.int8)
    if g.ndim != 2:
        raise ValueError("genotype matrix must be 2-D (patients x SNPs)")
    return g


def _ptr(a, t):
    return a.ctypes.data_as(t)


def sqdist(g1, g2=None, method: str = "bruteforce") -> np.ndarray:
    """Squared Euclidean distances between the rows of ``g1`` and ``g2`` (int64).

    ``method="bruteforce"`` sums ``(g1_ik - g2_jk)^2`` term by term (the
    definition used by Alg. 5); ``method="gram"`` uses the norm-plus-Gram
    identity of the paper's distance section (Sec. IV-B).  ``method="blas"``
    is the same identity with the Gram product G1 G2^T taken by a float64
    library matrix product: its entries and partial sums are integers of at
    most 4 m < 2^53, so it is exact too.  All three are exact.
    """
    a = _geno(g1)
    b = a if g2 is None else _geno(g2)
    if a.shape[1] != b.shape[1]:
        raise ValueError("SNP counts differ")
    if method == "blas":
        af = a.astype(np.float64)
        bf = af if g2 is None else b.astype(np.float64)
        s = af @ bf.T                        # s_ij = sum_k g1_ik g2_jk (exact)
        n1 = (af * af).sum(axis=1)
        n2 = n1 if g2 is None else (bf * bf).sum(axis=1)
        d = n1[:, None] + n2[None, :] - 2.0 * s
        return d.astype(np.int64)
    out = np.empty((a.shape[0], b.shape[0]), dtype=np.int64)
    fn = {"bruteforce": _load().oracle_sqdist_bruteforce, "gram": _load().oracle_sqdist_gram}[method]
    fn(_ptr(a, _i8p), a.shape[0], a.shape[1], _ptr(b, _i8p), b.shape[0], b.shape[1], a.shape[1],
       _ptr(out, _i64p))
    return out


def gaussian_kernel(d: np.ndarray, gamma: float) -> np.ndarray:
    """Alg. 5, Gaussian branch: ``exp(-gamma * d)`` elementwise, in double."""
    d = np.ascontiguousarray(d, dtype=np.int64)
    out = np.empty(d.shape, dtype=np.float64)
    _load().oracle_gaussian_kernel(_ptr(d, _i64p), d.size, float(gamma), _ptr(out, _f64p))
    return out


# Alleles shared identical by state at one locus, by genotype (copies of the
# minor allele): row a, column b.
IBS_TABLE = np.array([[2, 1, 0], [1, 2, 1], [0, 1, 2]], dtype=np.int64)


def ibs_count(g1, g2=None, method: str = "bruteforce") -> np.ndarray:
    """``(g1_i ~ g2_j)``: alleles shared identical by state, summed over the loci (int64).

    ``method="bruteforce"`` adds ``2 - |a - b|`` locus by locus;
    ``method="blas"`` writes each genotype as its one-hot indicator (a row of
    the 3 x 3 sharing table picks the count) and sums the table lookups of all
    loci with one float64 library matrix product (integers below 2^53:
    exact)."""
    a = _geno(g1)
    b = a if g2 is None else _geno(g2)
    if a.shape[1] != b.shape[1]:
        raise ValueError("SNP counts differ")
    if method == "blas":
        m = a.shape[1]
        ea = np.zeros((a.shape[0], m, 3), np.float64)
        np.put_along_axis(ea, a.astype(np.int64)[:, :, None], 1.0, axis=2)
        eb = np.zeros((b.shape[0], m, 3), np.float64)
        np.put_along_axis(eb, b.astype(np.int64)[:, :, None], 1.0, axis=2)
        ebw = eb @ IBS_TABLE.astype(np.float64)  # row of the table for each genotype of g2
        return (ea.reshape(a.shape[0], -1) @ ebw.reshape(b.shape[0], -1).T).astype(np.int64)
    out = np.empty((a.shape[0], b.shape[0]), dtype=np.int64)
    _load().oracle_ibs_count(_ptr(a, _i8p), a.shape[0], a.shape[1], _ptr(b, _i8p), b.shape[0], b.shape[1],
                             a.shape[1], _ptr(out, _i64p))
    return out


def ibs_kernel(g1, g2=None, method: str = "bruteforce") -> np.ndarray:
    """Alg. 5, IBS branch: ``K_ij = (g1_i ~ g2_j) / N_S`` in double (K_ii = 2)."""
    m = _geno(g1).shape[1]
    return ibs_count(g1, g2, method=method).astype(np.float64) / float(m)


def conf_sqdist(c1, c2=None) -> np.ndarray:
    """Squared distances of real confounder rows, term by term in double."""
    a = np.ascontiguousarray(np.asarray(c1), dtype=np.float64)
    b = a if c2 is None else np.ascontiguousarray(np.asarray(c2), dtype=np.float64)
    if a.ndim != 2 or b.ndim != 2 or a.shape[1] != b.shape[1]:
        raise ValueError("confounder matrices must be 2-D with the same number of columns")
    out = np.empty((a.shape[0], b.shape[0]), dtype=np.float64)
    _load().oracle_conf_sqdist(_ptr(a, _f64p), a.shape[0], a.shape[1], _ptr(b, _f64p), b.shape[0], b.shape[1],
                               a.shape[1], _ptr(out, _f64p))
    return out


def build_kernel(gamma: float, g1, g2=None, method: str = "bruteforce", kernel: str = "gaussian",
                 c1=None, c2=None) -> np.ndarray:
    """Alg. 2: ``K[i, j] = KernelMatrix(type, gamma, G1[i, :], G2[j, :])`` (type
    ``"gaussian"`` or ``"ibs"``; gamma unused for IBS).  With confounders
    ``c1`` (and ``c2`` for the second set), their squared distances join the
    genotype distances before the exponential:
    ``K_ij = exp(-gamma (||g_i - g_j||^2 + ||c_i - c_j||^2))``."""
    if kernel == "ibs":
        return ibs_kernel(g1, g2, method="blas" if method in ("blas", "lapack") else "bruteforce")
    if c1 is not None:
        d = sqdist(g1, g2, method=method).astype(np.float64) + conf_sqdist(c1, c2 if g2 is not None else None)
        return np.exp(-gamma * d)
    return gaussian_kernel(sqdist(g1, g2, method=method), gamma)


class NotPositiveDefinite(ArithmeticError):
    def __init__(self, column: int):
        super().__init__(f"non-positive pivot at column {column}")
        self.column = column


def cholesky(a: np.ndarray, method: str = "plain") -> np.ndarray:
    """Alg. 3 "Factorize": lower-triangular L with ``L L^T = a`` (double).

    ``method="lapack"`` takes LAPACK's float64 Cholesky as the step (the
    failing column is not reported then: ``column`` is -1)."""
    if method == "lapack":
        try:
            return np.linalg.cholesky(np.asarray(a, dtype=np.float64))
        except np.linalg.LinAlgError:
            raise NotPositiveDefinite(-1) from None
    l = np.array(a, dtype=np.float64, order="C", copy=True)
    n = l.shape[0]
    if l.shape != (n, n):
        raise ValueError("square matrix expected")
    col = _load().oracle_cholesky(_ptr(l, _f64p), n)
    if col >= 0:
        raise NotPositiveDefinite(int(col))
    return l


def forward_subst(l: np.ndarray, y: np.ndarray, method: str = "plain") -> np.ndarray:
    """Solve ``L Z = Y`` by forward substitution (Y is n x p)."""
    if method == "lapack":
        import scipy.linalg

        yy = np.asarray(y, dtype=np.float64).reshape(len(l), -1)
        return scipy.linalg.solve_triangular(l, yy, lower=True)
    l = np.ascontiguousarray(l, dtype=np.float64)
    z = np.array(y, dtype=np.float64, order="C", copy=True).reshape(l.shape[0], -1)
    _load().oracle_forward_subst(_ptr(l, _f64p), l.shape[0], _ptr(z, _f64p), z.shape[1])
    return z


def backward_subst(l: np.ndarray, z: np.ndarray, method: str = "plain") -> np.ndarray:
    """Solve ``L^T X = Z`` by backward substitution (Z is n x p)."""
    if method == "lapack":
        import scipy.linalg

        zz = np.asarray(z, dtype=np.float64).reshape(len(l), -1)
        return scipy.linalg.solve_triangular(l, zz, lower=True, trans="T")
    l = np.ascontiguousarray(l, dtype=np.float64)
    x = np.array(z, dtype=np.float64, order="C", copy=True).reshape(l.shape[0], -1)
    _load().oracle_backward_subst(_ptr(l, _f64p), l.shape[0], _ptr(x, _f64p), x.shape[1])
    return x


def matmul(a: np.ndarray, b: np.ndarray) -> np.ndarray:
    """Plain double product ``a @ b`` accumulated in index order."""
    a = np.ascontiguousarray(a, dtype=np.float64)
    b = np.ascontiguousarray(b, dtype=np.float64).reshape(a.shape[1], -1)
    c = np.empty((a.shape[0], b.shape[1]), dtype=np.float64)
    _load().oracle_matmul(_ptr(a, _f64p), a.shape[0], a.shape[1], _ptr(b, _f64p), b.shape[1],
                          _ptr(c, _f64p))
    return c


def _lin(method: str) -> str:
    """Method of the linear-algebra steps that goes with a distance method."""
    return "lapack" if method in ("lapack", "blas") else "plain"


def _dist(method: str) -> str:
    """Method of the distance step that goes with a method name."""
    return "blas" if method in ("lapack", "blas") else method


def associate(alpha: float, k: np.ndarray, y: np.ndarray, return_factor: bool = False,
              method: str = "plain"):
    """Alg. 3: ``K~ = Factorize(K + alpha I)``; ``W = Solve(K~, P_h)``."""
    a = np.array(k, dtype=np.float64, copy=True)
    a[np.diag_indices_from(a)] += alpha
    lm = _lin(method)
    l = cholesky(a, method=lm)
    del a
    w = backward_subst(l, forward_subst(l, y, method=lm), method=lm)
    return (w, l) if return_factor else w


def predict(gamma: float, g, t, w: np.ndarray, method: str = "bruteforce", kernel: str = "gaussian",
            conf=None, conf_t=None) -> np.ndarray:
    """Alg. 4: ``K = Build(gamma, T, G)`` (N_P2 x N_P1), ``P_r = K W``."""
    return matmul(build_kernel(gamma, t, g, method=_dist(method), kernel=kernel, c1=conf_t, c2=conf), w)


def krr(gamma: float, alpha: float, g, y, t, method: str = "plain", kernel: str = "gaussian", conf=None,
        conf_t=None):
    """Alg. 1: Build, Associate, Predict.  Returns (K, W, P_r).

    ``method="lapack"``: Gram product and factorisation by library routines
    (see the module docstring); the same definitions otherwise.  ``kernel``:
    the Alg. 5 kernel type, ``"gaussian"`` or ``"ibs"``."""
    dm = "bruteforce" if method == "plain" else _dist(method)
    k = build_kernel(gamma, g, method=dm, kernel=kernel, c1=conf)
    w = associate(alpha, k, y, method=method)
    return k, w, predict(gamma, g, t, w, method=dm, kernel=kernel, conf=conf, conf_t=conf_t)


def kernel_rows(gamma: float, g1, rows, g2) -> np.ndarray:
    """Rows ``rows`` of Build(gamma, G1, G2), each entry from the definition."""
    a = _geno(g1)
    b = _geno(g2)
    r = np.ascontiguousarray(rows, dtype=np.int64)
    out = np.empty((r.size, b.shape[0]), dtype=np.float64)
    _load().oracle_kernel_rows(_ptr(a, _i8p), a.shape[1], _ptr(r, _i64p), r.size, _ptr(b, _i8p),
                               b.shape[0], b.shape[1], a.shape[1], float(gamma), _ptr(out, _f64p))
    return out


def held_out_loss(gamma: float, lam: float, g, y, t, y_t) -> float:
    """Held-out mean squared error ``||K_test A - Y_t||_F^2 / (N_t P)``, A from Alg. 3."""
    w = associate(lam, build_kernel(gamma, g), y)
    r = predict(gamma, g, t, w) - np.asarray(y_t, dtype=np.float64).reshape(len(t), -1)
    return float((r * r).sum() / r.size)


def hyper_gradient(gamma: float, lam: float, g, y, t, y_t, method: str = "plain"):
    """Gradient of the held-out MSE with respect to log gamma and log lambda.

    With M = K + lambda I, A = M^-1 Y, Yhat = K_t A and
    loss = ||Yhat - Y_t||_F^2 / (N_t P):

    * G_p = dloss/dYhat = 2 (Yhat - Y_t) / (N_t P)
    * B = dloss/dA = K_t^T G_p and Z = M^-1 B (M is symmetric)
    * dA = -M^-1 dM A, so dloss = -<Z A^T, dM>.
    * dM/dlambda = I:              dloss/dlog lambda = -lambda <Z, A>.
    * dK/dgamma = -D (.) K, for K and for K_t:
      dloss/dlog gamma = gamma * ( sum_ij D_ij K_ij (Z A^T)_ij
                                   - sum_tj D_tj K_tj (G_p A^T)_tj ).

    Returns (loss, dloss/dlog gamma, dloss/dlog lambda), all double.
    ``method="lapack"``: Gram products and factorisation by library routines.
    """
    g = _geno(g)
    t = _geno(t)
    y = np.asarray(y, dtype=np.float64).reshape(len(g), -1)
    y_t = np.asarray(y_t, dtype=np.float64).reshape(len(t), -1)
    dm = "bruteforce" if method == "plain" else _dist(method)
    lm = _lin(method)
    d = sqdist(g, method=dm)
    k = gaussian_kernel(d, gamma)
    a, l = associate(lam, k, y, return_factor=True, method=method)
    d_t = sqdist(t, g, method=dm)
    k_t = gaussian_kernel(d_t, gamma)
    yhat = matmul(k_t, a)
    r = yhat - y_t
    loss = float((r * r).sum() / r.size)
    g_p = 2.0 * r / r.size
    b = matmul(k_t.T, g_p)
    z = backward_subst(l, forward_subst(l, b, method=lm), method=lm)
    dlog_lam = -lam * float((z * a).sum())
    za = matmul(z, a.T)
    ga = matmul(g_p, a.T)
    dgamma = float((d * k * za).sum()) - float((d_t * k_t * ga).sum())
    return loss, gamma * dgamma, dlog_lam


def ridge_design(g, c=None) -> np.ndarray:
    """X = [G C]: genotype columns, then the real confounder columns (double)."""
    x = _geno(g).astype(np.float64)
    if c is not None:
        x = np.concatenate([x, np.asarray(c, dtype=np.float64).reshape(len(x), -1)], axis=1)
    return x


def ridge(lam: float, g, y, c=None, method: str = "plain"):
    """Ridge regression (Sec. IV-A, Eq. 2): ``beta = (X^T X + lambda I)^-1 X^T Y``
    with X = [G C].  The Gram matrix and X^T Y are plain double products
    (``method="lapack"``: library products and factorisation); the system is
    solved by the Cholesky factorisation and substitutions of Alg. 3.
    Returns (X^T X, X^T Y, beta)."""
    x = ridge_design(g, c)
    yy = np.asarray(y, dtype=np.float64).reshape(len(x), -1)
    xt = np.ascontiguousarray(x.T)
    if method == "lapack":
        gram, rhs = xt @ x, xt @ yy
    else:
        gram, rhs = matmul(xt, x), matmul(xt, yy)
    beta = associate(lam, gram, rhs, method=method)
    return gram, rhs, beta


def ridge_predict(t, beta, ct=None) -> np.ndarray:
    """Predictions ``[T Ct] beta`` of held-out patients."""
    return matmul(ridge_design(t, ct), beta)
