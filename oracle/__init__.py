"""Plain FP64 CPU oracle for the sketch A_hat = S A and SAP least squares.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference legs of ``bench.py`` may import this package.  The
product library (``paper_2310_15419_gb300``) never imports, links or calls it,
and the oracle shares no code with the CUDA path: it is a separate C file
(``oracle.c``) compiled with gcc into its own shared object.

Functions follow the paper (arXiv 2310.15419):
  * ``philox4x32_10``            counter-based generator named in Sec. 4.2
  * ``S_entry`` / ``S_column`` / ``S_dense``  S(i, j), Sec. 1.1 + Sec. 3.3
  * ``sketch_kji``               Alg. 3 (regenerate S(:, j) per nonzero)
  * ``sketch_jki``               Alg. 4 (generate S(:, j) once per nonempty row)
  * ``householder_qr``           QR of the sketch, Sec. 5.3
  * ``lsqr``                     LSQR on A R^{-1}, Sec. 5.3
  * ``ls_error``                 Error(x) of Sec. 5.3
  * ``sap_qr_solve``             the whole SAP-QR pipeline of Sec. 5.3
  * ``jacobi_svd``               one-sided Jacobi SVD of the sketch, Sec. 5.3
  * ``sap_svd_solve``            SAP-SVD (singular values below sigma_max / 1e12
                                 dropped), Sec. 5.3
  * ``lsqr_d_solve``             LSQR-D, the diagonal-preconditioned LSQR that
                                 Sec. 5.3 compares against
  * ``sketch_jki_omp``           Alg. 4 order on all host cores (bit-identical
                                 to ``sketch_jki``)

Parity status: every function above is pinned by a ``-m "not gpu"`` test
against something other than itself (torch's Philox engine, closed forms,
brute-force dense products, LAPACK QR, SciPy LSQR, numpy lstsq, moments).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

PM1, UNIFORM, NORMAL = 0, 1, 2

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile oracle.c with gcc into oracle/_build/liboracle.so."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + ".tmp.%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-Wall", "-fopenmp", "-shared", "-fPIC", "-o", tmp,
           _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        i64, u64, u32, i32 = (ctypes.c_int64, ctypes.c_uint64, ctypes.c_uint32,
                              ctypes.c_int)
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int32)
        up = ctypes.POINTER(ctypes.c_uint32)
        lib.oracle_philox4x32_10.argtypes = [up, up, up]
        lib.oracle_philox4x32_10.restype = None
        lib.oracle_S_entry.argtypes = [i32, u64, u32, i64, i64]
        lib.oracle_S_entry.restype = ctypes.c_double
        lib.oracle_S_column.argtypes = [i32, u64, u32, i64, i64, dp]
        lib.oracle_S_column.restype = None
        lib.oracle_S_dense.argtypes = [i32, u64, u32, i64, i64, dp]
        lib.oracle_S_dense.restype = None
        lib.oracle_uniform_from_word.argtypes = [u32]
        lib.oracle_uniform_from_word.restype = ctypes.c_double
        lib.oracle_normal_from_words.argtypes = [u32, u32, i32]
        lib.oracle_normal_from_words.restype = ctypes.c_double
        lib.oracle_sketch_kji.argtypes = [i64, i64, i64, i32, u64, u32, ip, ip,
                                          dp, dp]
        lib.oracle_sketch_kji.restype = i64
        lib.oracle_sketch_jki_rows.argtypes = [i64, i64, i64, i32, u64, u32, ip,
                                               ip, dp, dp, i64, i64]
        lib.oracle_sketch_jki_rows.restype = i64
        lib.oracle_sketch_jki_omp.argtypes = [i64, i64, i64, i32, u64, u32, ip,
                                              ip, dp, dp, i64, i64, i32]
        lib.oracle_sketch_jki_omp.restype = i64
        lib.oracle_max_threads.argtypes = []
        lib.oracle_max_threads.restype = i32
        lib.oracle_householder_qr.argtypes = [i64, i64, dp, dp]
        lib.oracle_householder_qr.restype = i32
        lib.oracle_ls_error.argtypes = [i64, i64, ip, ip, dp, dp, dp]
        lib.oracle_ls_error.restype = ctypes.c_double
        lib.oracle_lsqr.argtypes = [i64, i64, ip, ip, dp, dp, dp,
                                    ctypes.c_double, i64, dp, dp]
        lib.oracle_lsqr.restype = i32
        lib.oracle_sap_qr_solve.argtypes = [i64, i64, i64, i32, u64, u32, ip,
                                            ip, dp, dp, ctypes.c_double, i64,
                                            dp, dp]
        lib.oracle_sap_qr_solve.restype = i32
        lib.oracle_jacobi_svd.argtypes = [i64, i64, dp, dp, dp]
        lib.oracle_jacobi_svd.restype = i32
        lib.oracle_sap_svd_solve.argtypes = [i64, i64, i64, i32, u64, u32, ip,
                                             ip, dp, dp, ctypes.c_double, i64,
                                             dp, dp]
        lib.oracle_sap_svd_solve.restype = i32
        lib.oracle_lsqr_d_solve.argtypes = [i64, i64, ip, ip, dp, dp,
                                            ctypes.c_double, i64, dp, dp]
        lib.oracle_lsqr_d_solve.restype = i32
        _lib = lib
        return lib


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def _ptr(a, ctype):
    return a.ctypes.data_as(ctypes.POINTER(ctype))


def philox4x32_10(ctr, key):
    """Philox4x32-10 block for counter (4 x u32) and key (2 x u32)."""
    lib = _load()
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib.oracle_philox4x32_10(_ptr(c, ctypes.c_uint32), _ptr(k, ctypes.c_uint32),
                             _ptr(out, ctypes.c_uint32))
    return out


def uniform_from_word(w: int) -> float:
    return _load().oracle_uniform_from_word(int(w))


def normal_from_words(w_radius: int, w_angle: int, sel: int) -> float:
    return _load().oracle_normal_from_words(int(w_radius), int(w_angle), int(sel))


def S_entry(dist: int, seed: int, stream: int, i: int, j: int) -> float:
    return _load().oracle_S_entry(dist, seed, stream, i, j)


def S_column(dist: int, seed: int, stream: int, d: int, j: int) -> np.ndarray:
    out = np.zeros(d, dtype=np.float64)
    _load().oracle_S_column(dist, seed, stream, d, j, _ptr(out, ctypes.c_double))
    return out


def S_dense(dist: int, seed: int, stream: int, d: int, m: int) -> np.ndarray:
    """Materialised S, d x m (only for small brute-force checks)."""
    out = np.zeros((m, d), dtype=np.float64)  # column-major d x m == row-major m x d
    _load().oracle_S_dense(dist, seed, stream, d, m, _ptr(out, ctypes.c_double))
    return out.T


def sketch_kji(m, n, d, dist, seed, stream, colptr, rowidx, values):
    """Alg. 3 order.  Returns (A_hat (d x n float64), S entries generated)."""
    cp, ri, va = _i32(colptr), _i32(rowidx), _f64(values)
    out = np.zeros((n, d), dtype=np.float64)
    gen = _load().oracle_sketch_kji(m, n, d, dist, seed, stream,
                                    _ptr(cp, ctypes.c_int32),
                                    _ptr(ri, ctypes.c_int32),
                                    _ptr(va, ctypes.c_double),
                                    _ptr(out, ctypes.c_double))
    return out.T, int(gen)


def sketch_jki_omp(m, n, d, dist, seed, stream, colptr, rowidx, values,
                   row_lo: int = 0, row_hi: int = -1, threads: int = 0):
    """Alg. 4 order on all host cores (OpenMP; `threads` <= 0: the default
    count), bit-identical to ``sketch_jki``: the rows of A_hat are split
    between the threads, so each element's additions keep the serial order.
    Returns (A_hat (d x n float64), S entries generated)."""
    cp, ri, va = _i32(colptr), _i32(rowidx), _f64(values)
    out = np.zeros((n, d), dtype=np.float64)
    gen = _load().oracle_sketch_jki_omp(m, n, d, dist, seed, stream,
                                        _ptr(cp, ctypes.c_int32),
                                        _ptr(ri, ctypes.c_int32),
                                        _ptr(va, ctypes.c_double),
                                        _ptr(out, ctypes.c_double),
                                        row_lo, row_hi, int(threads))
    if gen < 0:
        raise MemoryError("oracle_sketch_jki_omp: allocation failed")
    return out.T, int(gen)


def max_threads() -> int:
    """Threads the oracle's OpenMP regions use by default."""
    return int(_load().oracle_max_threads())


def sketch_jki(m, n, d, dist, seed, stream, colptr, rowidx, values,
               row_lo: int = 0, row_hi: int = -1):
    """Alg. 4 order.  Returns (A_hat (d x n float64), S entries generated)."""
    cp, ri, va = _i32(colptr), _i32(rowidx), _f64(values)
    out = np.zeros((n, d), dtype=np.float64)
    gen = _load().oracle_sketch_jki_rows(m, n, d, dist, seed, stream,
                                         _ptr(cp, ctypes.c_int32),
                                         _ptr(ri, ctypes.c_int32),
                                         _ptr(va, ctypes.c_double),
                                         _ptr(out, ctypes.c_double),
                                         row_lo, row_hi)
    if gen < 0:
        raise MemoryError("oracle_sketch_jki_rows: allocation failed")
    return out.T, int(gen)


sketch = sketch_jki


def householder_qr(A: np.ndarray) -> np.ndarray:
    """R (n x n upper triangular) of the Householder QR of A (d x n)."""
    d, n = A.shape
    a = np.asfortranarray(A, dtype=np.float64)
    R = np.zeros((n, n), dtype=np.float64, order="F")
    st = _load().oracle_householder_qr(d, n, a.ctypes.data_as(
        ctypes.POINTER(ctypes.c_double)), R.ctypes.data_as(
            ctypes.POINTER(ctypes.c_double)))
    if st == -2:
        raise MemoryError("oracle_householder_qr: allocation failed")
    return np.array(R)


def ls_error(m, n, colptr, rowidx, values, b, x) -> float:
    cp, ri, va = _i32(colptr), _i32(rowidx), _f64(values)
    bb, xx = _f64(b), _f64(x)
    return _load().oracle_ls_error(m, n, _ptr(cp, ctypes.c_int32),
                                   _ptr(ri, ctypes.c_int32),
                                   _ptr(va, ctypes.c_double),
                                   _ptr(bb, ctypes.c_double),
                                   _ptr(xx, ctypes.c_double))


def lsqr(m, n, colptr, rowidx, values, b, R=None, tol=1e-10, maxit=1000):
    """LSQR on A R^{-1} (A if R is None).  Returns (x, info dict)."""
    cp, ri, va = _i32(colptr), _i32(rowidx), _f64(values)
    bb = _f64(b)
    x = np.zeros(n, dtype=np.float64)
    info = np.zeros(8, dtype=np.float64)
    Rp = None
    if R is not None:
        Rf = np.asfortranarray(R, dtype=np.float64)
        Rp = Rf.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    st = _load().oracle_lsqr(m, n, _ptr(cp, ctypes.c_int32),
                             _ptr(ri, ctypes.c_int32), _ptr(va, ctypes.c_double),
                             _ptr(bb, ctypes.c_double), Rp, tol, maxit,
                             _ptr(x, ctypes.c_double),
                             _ptr(info, ctypes.c_double))
    if st == -2:
        raise MemoryError("oracle_lsqr: allocation failed")
    return x, {"iters": int(info[0]), "istop": int(info[1]),
               "test2": float(info[2]), "anorm": float(info[3]),
               "converged": st == 0}


def sap_qr_solve(m, n, d, dist, seed, stream, colptr, rowidx, values, b,
                 tol=1e-10, maxit=1000):
    """Sec. 5.3 SAP-QR.  Returns (x, info dict with 'error' = Error(x))."""
    cp, ri, va = _i32(colptr), _i32(rowidx), _f64(values)
    bb = _f64(b)
    x = np.zeros(n, dtype=np.float64)
    info = np.zeros(8, dtype=np.float64)
    st = _load().oracle_sap_qr_solve(m, n, d, dist, seed, stream,
                                     _ptr(cp, ctypes.c_int32),
                                     _ptr(ri, ctypes.c_int32),
                                     _ptr(va, ctypes.c_double),
                                     _ptr(bb, ctypes.c_double), tol, maxit,
                                     _ptr(x, ctypes.c_double),
                                     _ptr(info, ctypes.c_double))
    if st == -2:
        raise MemoryError("oracle_sap_qr_solve: allocation failed")
    return x, {"iters": int(info[0]), "istop": int(info[1]),
               "test2": float(info[2]), "anorm": float(info[3]),
               "error": float(info[4]), "converged": st == 0}


def jacobi_svd(A):
    """One-sided Jacobi SVD of a dense d x n array (d >= n): (sigma
    decreasing, V n x n, sweeps).  Sec. 5.3's SVD of the sketch."""
    A = np.asarray(A, dtype=np.float64)
    d, n = A.shape
    a = np.ascontiguousarray(A.T)          # column-major d x n
    sigma = np.zeros(n, dtype=np.float64)
    V = np.zeros((n, n), dtype=np.float64)  # row j = column j of V
    sw = _load().oracle_jacobi_svd(d, n, _ptr(a, ctypes.c_double),
                                   _ptr(sigma, ctypes.c_double), _ptr(V, ctypes.c_double))
    if sw == -2:
        raise MemoryError("oracle_jacobi_svd: allocation failed")
    return sigma, V.T.copy(), int(sw)


def sap_svd_solve(m, n, d, dist, seed, stream, colptr, rowidx, values, b,
                  tol=1e-10, maxit=1000):
    """Sec. 5.3 SAP-SVD.  Returns (x, info) with 'error' = Error(x), 'rank'
    = singular values kept (>= sigma_max / 1e12) and the Jacobi 'sweeps'."""
    cp, ri, va = _i32(colptr), _i32(rowidx), _f64(values)
    bb = _f64(b)
    x = np.zeros(n, dtype=np.float64)
    info = np.zeros(8, dtype=np.float64)
    st = _load().oracle_sap_svd_solve(m, n, d, dist, seed, stream,
                                      _ptr(cp, ctypes.c_int32), _ptr(ri, ctypes.c_int32),
                                      _ptr(va, ctypes.c_double), _ptr(bb, ctypes.c_double),
                                      tol, maxit, _ptr(x, ctypes.c_double),
                                      _ptr(info, ctypes.c_double))
    if st == -2:
        raise MemoryError("oracle_sap_svd_solve: allocation failed")
    if st == -1:
        raise RuntimeError("oracle_sap_svd_solve: the Jacobi SVD did not converge")
    return x, {"iters": int(info[0]), "istop": int(info[1]), "test2": float(info[2]),
               "anorm": float(info[3]), "error": float(info[4]), "rank": int(info[5]),
               "sweeps": int(info[6]), "converged": st == 0}


def lsqr_d_solve(m, n, colptr, rowidx, values, b, tol=1e-10, maxit=1000):
    """Sec. 5.3 LSQR-D (LSQR with D_ii = 1 / ||A_i||).  Returns (x, info)."""
    cp, ri, va = _i32(colptr), _i32(rowidx), _f64(values)
    bb = _f64(b)
    x = np.zeros(n, dtype=np.float64)
    info = np.zeros(8, dtype=np.float64)
    st = _load().oracle_lsqr_d_solve(m, n, _ptr(cp, ctypes.c_int32), _ptr(ri, ctypes.c_int32),
                                     _ptr(va, ctypes.c_double), _ptr(bb, ctypes.c_double),
                                     tol, maxit, _ptr(x, ctypes.c_double),
                                     _ptr(info, ctypes.c_double))
    if st == -2:
        raise MemoryError("oracle_lsqr_d_solve: allocation failed")
    return x, {"iters": int(info[0]), "istop": int(info[1]), "test2": float(info[2]),
               "anorm": float(info[3]), "error": float(info[4]), "converged": st == 0}
