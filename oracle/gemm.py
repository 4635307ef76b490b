"""FP64 gemm oracle (definition of C = alpha*A*B + beta*C, Tiramisu paper
Section I) -- test infrastructure only; see the package docstring.

The arithmetic lives in ``gemm_oracle.c`` (plain i-k-j triple loop in double);
this module compiles it with gcc and wraps it with ctypes.  ``gemm_exact`` is an
independent exact-rational restatement for tiny shapes (pure Python loops).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from fractions import Fraction

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gemm_oracle.c")
_LIB_PATH = os.path.join(_HERE, "_build", "liboracle_gemm.so")
_lock = threading.Lock()
_lib = None


def library_path() -> str:
    return _LIB_PATH


def build(force: bool = False) -> str:
    """Compile the oracle's C file into a shared object (gcc, OpenMP)."""
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-std=c11", "-ffp-contract=off",
           "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB_PATH)
            i64, f32, vp = ctypes.c_int64, ctypes.c_float, ctypes.c_void_p
            lib.oracle_gemm_f64.argtypes = [i64, i64, i64, f32, vp, i64, vp, i64,
                                            f32, vp, i64, vp, i64]
            lib.oracle_gemm_f64.restype = None
            lib.oracle_gemm_f64_rows.argtypes = [i64, i64, f32, vp, i64, vp, i64,
                                                 f32, vp, i64, vp, i64, vp]
            lib.oracle_gemm_f64_rows.restype = None
            lib.oracle_axpby_f64.argtypes = [i64, i64, f32, vp, i64, f32, vp, i64, vp, i64]
            lib.oracle_axpby_f64.restype = None
            lib.oracle_gemm_f32_seq.argtypes = [i64, i64, i64, f32, vp, i64, vp, i64,
                                                f32, vp, i64, vp, i64]
            lib.oracle_gemm_f32_seq.restype = None
            lib.oracle_rel_frob.argtypes = [i64, i64, vp, i64, vp, i64]
            lib.oracle_rel_frob.restype = ctypes.c_double
            lib.oracle_set_num_threads.argtypes = [ctypes.c_int]
            lib.oracle_set_num_threads.restype = None
            lib.oracle_num_threads.argtypes = []
            lib.oracle_num_threads.restype = ctypes.c_int
            _lib = lib
    return _lib


def _f32(a: np.ndarray) -> np.ndarray:
    if a.dtype != np.float32 or not a.flags.c_contiguous:
        raise TypeError("oracle inputs must be C-contiguous float32 storage arrays")
    return a


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


def gemm_f64(M: int, N: int, K: int, alpha: float, A: np.ndarray, B: np.ndarray,
             beta: float, C0: np.ndarray | None) -> np.ndarray:
    """Full M x N double result.  A, B, C0 are row-major float32 storage arrays
    whose second dimension is the leading dimension (>= the row length)."""
    lib = _load()
    A = _f32(A) if K > 0 and M > 0 else None
    B = _f32(B) if K > 0 and N > 0 else None
    ldc = 1
    if beta != 0.0:
        C0 = _f32(C0)
        ldc = C0.shape[1]
    else:
        C0 = None
    out = np.empty((M, N), dtype=np.float64)
    if M == 0 or N == 0:
        return out
    lda = A.shape[1] if A is not None else max(K, 1)
    ldb = B.shape[1] if B is not None else max(N, 1)
    lib.oracle_gemm_f64(M, N, K, ctypes.c_float(alpha), _ptr(A), lda, _ptr(B), ldb,
                        ctypes.c_float(beta), _ptr(C0), ldc, _ptr(out), N)
    return out


def gemm_f64_rows(rows, N: int, K: int, alpha: float, A: np.ndarray, B: np.ndarray,
                  beta: float, C0: np.ndarray | None) -> np.ndarray:
    """Rows ``rows`` of the double result (len(rows) x N)."""
    lib = _load()
    rows = np.ascontiguousarray(np.asarray(rows, dtype=np.int64))
    A = _f32(A)
    B = _f32(B)
    ldc = 1
    if beta != 0.0:
        C0 = _f32(C0)
        ldc = C0.shape[1]
    else:
        C0 = None
    out = np.empty((len(rows), N), dtype=np.float64)
    if len(rows) == 0 or N == 0:
        return out
    lib.oracle_gemm_f64_rows(N, K, ctypes.c_float(alpha), _ptr(A), A.shape[1], _ptr(B),
                             B.shape[1], ctypes.c_float(beta), _ptr(C0), ldc,
                             _ptr(rows), len(rows), _ptr(out))
    return out


def product_f64(M: int, N: int, K: int, A: np.ndarray, B: np.ndarray) -> np.ndarray:
    """The sums sum_k A[i][k] * B[k][j] in double (M x N): gemm_f64 with
    alpha = 1 and beta = 0.  With ``axpby_f64`` it gives gemm_f64's result bit
    for bit, so that one product (the expensive part at large sizes) serves
    several (alpha, beta) pairs."""
    return gemm_f64(M, N, K, 1.0, A, B, 0.0, None)


def axpby_f64(alpha: float, P: np.ndarray, beta: float, C0: np.ndarray | None) -> np.ndarray:
    """alpha * P + beta * C0 in double, the definition's last step (C0 a
    float32 storage array, not read when beta == 0)."""
    lib = _load()
    P = np.ascontiguousarray(P, dtype=np.float64)
    M, N = P.shape
    ldc = 1
    if beta != 0.0:
        C0 = _f32(C0)
        ldc = C0.shape[1]
    else:
        C0 = None
    out = np.empty((M, N), dtype=np.float64)
    if M == 0 or N == 0:
        return out
    lib.oracle_axpby_f64(M, N, ctypes.c_float(alpha), _ptr(P), N, ctypes.c_float(beta), _ptr(C0), ldc,
                         _ptr(out), N)
    return out


def gemm_f32_seq(M: int, N: int, K: int, alpha: float, A: np.ndarray, B: np.ndarray,
                 beta: float, C0: np.ndarray | None) -> np.ndarray:
    """The definition evaluated in FP32 (k in increasing order, every product
    and sum rounded to FP32): the accuracy of a plain single-precision gemm,
    the yardstick of the six-product mode.  M x N float32."""
    lib = _load()
    A = _f32(A) if K > 0 and M > 0 else None
    B = _f32(B) if K > 0 and N > 0 else None
    ldc = 1
    if beta != 0.0:
        C0 = _f32(C0)
        ldc = C0.shape[1]
    else:
        C0 = None
    out = np.empty((M, N), dtype=np.float32)
    if M == 0 or N == 0:
        return out
    lda = A.shape[1] if A is not None else max(K, 1)
    ldb = B.shape[1] if B is not None else max(N, 1)
    lib.oracle_gemm_f32_seq(M, N, K, ctypes.c_float(alpha), _ptr(A), lda, _ptr(B), ldb,
                            ctypes.c_float(beta), _ptr(C0), ldc, _ptr(out), N)
    return out


def set_num_threads(n: int) -> None:
    """Threads the oracle's OpenMP loops use from now on."""
    _load().oracle_set_num_threads(int(n))


def num_threads() -> int:
    """OpenMP threads the oracle's loops use."""
    return int(_load().oracle_num_threads())


def rel_frob(got: np.ndarray, ref: np.ndarray) -> float:
    """||got - ref||_F / ||ref||_F in double (absolute norm if ref == 0).
    ``got`` may be a storage array wider than ``ref`` (ld > N)."""
    lib = _load()
    M, N = ref.shape
    got = np.ascontiguousarray(got, dtype=np.float32)
    ref = np.ascontiguousarray(ref, dtype=np.float64)
    if M == 0 or N == 0:
        return 0.0
    return float(lib.oracle_rel_frob(M, N, _ptr(got), got.shape[1], _ptr(ref), N))


def gemm_exact(M: int, N: int, K: int, alpha: float, A: np.ndarray, B: np.ndarray,
               beta: float, C0: np.ndarray | None) -> list[list[Fraction]]:
    """Exact rational value of alpha*A*B + beta*C0 (pure Python; tiny shapes).
    Every float is converted to the Fraction it denotes exactly."""
    fa, fb = Fraction(float(alpha)), Fraction(float(beta))
    out = []
    for i in range(M):
        row = []
        for j in range(N):
            s = Fraction(0)
            if fa != 0:
                for k in range(K):
                    s += Fraction(float(A[i, k])) * Fraction(float(B[k, j]))
            v = fa * s
            if fb != 0:
                v += fb * Fraction(float(C0[i, j]))
            row.append(v)
        out.append(row)
    return out
