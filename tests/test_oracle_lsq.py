"""Pins for the oracle's SAP least-squares pieces (Sec. 5.3); CPU only.

Householder QR is pinned to LAPACK (numpy.linalg.qr uses the same sign
convention R(k,k) = -sign(x_0) ||x||); LSQR to SciPy's independent LSQR and
to numpy.linalg.lstsq; Error(x) to a hand-worked example; the SAP pipeline to
lstsq, to the condition-number iteration bound of Sec. 5 (d = gamma n gives a
preconditioned condition number near (sqrt(gamma)+1)/(sqrt(gamma)-1)) and to
the iteration counts the paper prints (tests/golden/paper_tables.txt).
"""
import os

import numpy as np
import pytest

import oracle
from paper_2310_15419_gb300 import inputs


def test_qr_matches_lapack():
    rng = np.random.default_rng(0)
    for d, n in [(10, 10), (40, 7), (200, 100), (3, 1)]:
        A = rng.standard_normal((d, n))
        R = oracle.householder_qr(A)
        Rl = np.linalg.qr(A, mode="r")
        assert np.allclose(R, Rl, rtol=0, atol=1e-12 * np.linalg.norm(A))
        assert np.allclose(np.tril(R, -1), 0)
        assert np.allclose(R.T @ R, A.T @ A, rtol=0, atol=1e-11 * np.linalg.norm(A) ** 2)


def test_qr_rank_deficient_column():
    A = np.zeros((6, 3))
    A[:, 0] = 1.0
    A[:, 2] = np.arange(6)
    R = oracle.householder_qr(A)
    assert R[1, 1] == 0.0


def test_error_metric_worked_example():
    """A = [1; 1], b = [1; 3], x = 0: A x - b = [-1; -3], A^T r = -4,
    ||A||_F = sqrt 2, ||r|| = sqrt 10 -> Error = 4 / sqrt(20)."""
    colptr = np.array([0, 2], np.int32)
    rowidx = np.array([0, 1], np.int32)
    vals = np.array([1.0, 1.0])
    e = oracle.ls_error(2, 1, colptr, rowidx, vals, np.array([1.0, 3.0]), np.zeros(1))
    assert abs(e - 4.0 / np.sqrt(20.0)) < 1e-15
    # at the LS solution x = 2 the residual is orthogonal to range(A)
    e2 = oracle.ls_error(2, 1, colptr, rowidx, vals, np.array([1.0, 3.0]), np.array([2.0]))
    assert e2 == 0.0


def test_lsqr_matches_scipy_lsqr():
    from scipy.sparse.linalg import lsqr as sp_lsqr
    A, b, _ = inputs.lsq_problem(3000, 40, 0.05, seed=1, noise=1e-2)
    x, info = oracle.lsqr(A.m, A.n, A.colptr, A.rowidx, A.values, b, None,
                          tol=1e-12, maxit=2000)
    res = sp_lsqr(A.to_scipy(), b, atol=1e-12, btol=1e-12, iter_lim=2000)
    xs, istop, itn = res[0], res[1], res[2]
    assert np.linalg.norm(x - xs) <= 1e-8 * np.linalg.norm(xs)
    assert abs(info["iters"] - itn) <= 3


def test_lsqr_with_exact_R_converges_immediately():
    """With R from the QR of A itself, A R^{-1} has orthonormal columns
    (condition number 1), so LSQR needs only a couple of iterations."""
    A, b, _ = inputs.lsq_problem(800, 20, 0.1, seed=2, noise=1e-1)
    R = oracle.householder_qr(A.to_scipy().toarray())
    x, info = oracle.lsqr(A.m, A.n, A.colptr, A.rowidx, A.values, b, R,
                          tol=1e-12, maxit=100)
    xl = np.linalg.lstsq(A.to_scipy().toarray(), b, rcond=None)[0]
    assert info["iters"] <= 3
    assert np.linalg.norm(x - xl) <= 1e-10 * np.linalg.norm(xl)


@pytest.mark.parametrize("dist", [oracle.PM1, oracle.UNIFORM, oracle.NORMAL])
def test_sap_qr_matches_lstsq(dist):
    m, n = 2000, 50
    A, b, _ = inputs.lsq_problem(m, n, 0.05, seed=3, noise=1e-1,
                                 col_scale_decades=2.0)
    x, info = oracle.sap_qr_solve(m, n, 2 * n, dist, 17, 0, A.colptr, A.rowidx,
                                  A.values, b, tol=1e-10, maxit=500)
    Ad = A.to_scipy().toarray()
    xl = np.linalg.lstsq(Ad, b, rcond=None)[0]
    el = oracle.ls_error(m, n, A.colptr, A.rowidx, A.values, b, xl)
    assert info["converged"]
    # LSQR stops on its estimate for the preconditioned system; the true
    # Error(x) may sit slightly above the stopping tolerance (the paper's
    # Table "lsquality" caption notes the same deviation)
    assert info["error"] <= max(10 * 1e-10, 10 * el)
    cond = np.linalg.cond(Ad)
    assert np.linalg.norm(x - xl) <= 1e-9 * cond * np.linalg.norm(xl)
    # gamma = 2: kappa <= ~5.83 -> ~66 iterations to 1e-10; allow slack for
    # the finite-n distortion
    assert info["iters"] <= 90


def test_sap_iterations_comparable_to_paper():
    """The paper's SAP-QR needed 80-88 LSQR iterations at tolerance 1e-14 with
    d = 2n and reached Error(x) ~ 1e-15 (tests/golden/paper_tables.txt)."""
    path = os.path.join(os.path.dirname(__file__), "golden", "paper_tables.txt")
    rows = [l.split() for l in open(path) if l.startswith("sap_iters")]
    iters = [int(r[2]) for r in rows]
    errs = [float(r[3]) for r in rows]
    m, n = 20_000, 100
    A, b, _ = inputs.lsq_problem(m, n, 0.01, seed=5, noise=1.0)
    x, info = oracle.sap_qr_solve(m, n, 2 * n, oracle.UNIFORM, 1, 0, A.colptr,
                                  A.rowidx, A.values, b, tol=1e-14, maxit=500)
    assert 0.5 * min(iters) <= info["iters"] <= 1.5 * max(iters)
    assert info["error"] <= 100 * max(errs)


# ------------------------------------------------------------ SAP-SVD, LSQR-D
def test_jacobi_svd_matches_lapack():
    """Singular values and right singular vectors against numpy's LAPACK SVD
    (vectors up to sign), at several shapes including a graded matrix."""
    rng = np.random.default_rng(3)
    for d, n, grade in [(10, 10, 0), (40, 7, 0), (120, 60, 6), (5, 1, 0)]:
        A = rng.standard_normal((d, n)) * 10.0 ** np.linspace(0, -grade, n)[None, :]
        s, V, sweeps = oracle.jacobi_svd(A)
        _, sl, Vt = np.linalg.svd(A)
        assert sweeps > 0
        assert np.allclose(s, sl, rtol=1e-12, atol=0)
        # A V = U diag(s) with orthonormal U, and |V^T V_lapack| = I
        U = (A @ V) / s
        assert np.allclose(U.T @ U, np.eye(n), atol=1e-10)
        assert np.allclose(np.abs(V.T @ Vt.T), np.eye(n), atol=1e-8)


def test_jacobi_svd_rank_deficient():
    """A duplicated (scaled) column and a zero column: two singular values
    at the FP64 noise level, the rest equal to LAPACK's."""
    rng = np.random.default_rng(4)
    A = rng.standard_normal((50, 12))
    A[:, 5] = 3.0 * A[:, 2]
    A[:, 9] = 0.0
    s, V, _ = oracle.jacobi_svd(A)
    sl = np.linalg.svd(A, compute_uv=False)
    assert np.allclose(s[:10], sl[:10], rtol=1e-12)
    assert np.all(s[10:] <= 1e-13 * s[0])


def _dense(A):
    return A.to_scipy().toarray()


@pytest.mark.parametrize("dist", [oracle.PM1, oracle.UNIFORM, oracle.NORMAL])
def test_sap_svd_full_rank_matches_lstsq(dist):
    A, b, _ = inputs.lsq_problem(3000, 40, 0.05, seed=21, noise=1e-2,
                                 col_scale_decades=2.0)
    x, info = oracle.sap_svd_solve(A.m, A.n, 2 * A.n, dist, 1, 0, A.colptr, A.rowidx,
                                   A.values, b, tol=1e-12, maxit=500)
    xl = np.linalg.lstsq(_dense(A), b, rcond=None)[0]
    assert info["converged"] and info["rank"] == A.n
    assert np.linalg.norm(x - xl) <= 1e-9 * np.linalg.norm(xl)
    assert info["error"] <= 1e-11
    # the sketch preconditions as well as the QR one: few iterations
    assert info["iters"] <= 80


def test_sap_svd_rank_deficient_gives_the_minimum_norm_solution():
    """With a duplicated column and a zero column, the kept singular
    directions span the row space of A, so x = P y is the minimum-norm
    least-squares solution, numpy's pinv(A) b."""
    A, b, _ = inputs.lsq_problem(2000, 30, 0.08, seed=22, noise=1e-1)
    Ad = _dense(A)
    Ad[:, 7] = -2.0 * Ad[:, 3]
    Ad[:, 20] = 0.0
    import scipy.sparse as sp
    C = sp.csc_matrix(Ad)
    C.sort_indices()
    B = inputs.CSC(A.m, A.n, C.indptr.astype(np.int32), C.indices.astype(np.int32),
                   C.data.astype(np.float32))
    Ad = B.to_scipy().toarray()
    x, info = oracle.sap_svd_solve(B.m, B.n, 2 * B.n, oracle.UNIFORM, 3, 0, B.colptr,
                                   B.rowidx, B.values, b, tol=1e-12, maxit=500)
    xp = np.linalg.pinv(Ad, rcond=1e-12) @ b
    assert info["rank"] == B.n - 2
    assert np.linalg.norm(x - xp) <= 1e-8 * np.linalg.norm(xp)
    assert abs(x[20]) <= 1e-12 * np.linalg.norm(xp)


def test_lsqr_d_matches_lstsq_and_scales_columns():
    """LSQR-D reaches lstsq's solution; on columns scaled over four decades
    it needs far fewer iterations than unpreconditioned LSQR (so D_ii is
    1 / ||A_i||, not ||A_i||), and a zero column takes D_ii = 1."""
    A, b, _ = inputs.lsq_problem(4000, 30, 0.05, seed=23, noise=1e-2,
                                 col_scale_decades=2.0)
    xl = np.linalg.lstsq(_dense(A), b, rcond=None)[0]
    x, info = oracle.lsqr_d_solve(A.m, A.n, A.colptr, A.rowidx, A.values, b,
                                  tol=1e-12, maxit=5000)
    assert info["converged"]
    assert np.linalg.norm(x - xl) <= 1e-8 * np.linalg.norm(xl)
    x0, i0 = oracle.lsqr(A.m, A.n, A.colptr, A.rowidx, A.values, b, None,
                         tol=1e-12, maxit=5000)
    assert info["iters"] * 3 < i0["iters"]
    # a zero column: D = 1 there and its solution entry stays 0
    cp = np.concatenate([A.colptr, A.colptr[-1:]])
    Z = inputs.CSC(A.m, A.n + 1, cp, A.rowidx, A.values)
    xz, iz = oracle.lsqr_d_solve(Z.m, Z.n, Z.colptr, Z.rowidx, Z.values, b,
                                 tol=1e-12, maxit=5000)
    assert np.isfinite(xz).all() and xz[-1] == 0.0
    assert np.linalg.norm(xz[:-1] - xl) <= 1e-8 * np.linalg.norm(xl)
