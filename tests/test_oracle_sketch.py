"""Pins for the oracle's sketch A_hat = S A (Eq. 1, Alg. 3, Alg. 4); CPU only.

Pinned against: brute-force dense products (numpy matmul of the materialised
S with the densified A), exact integer arithmetic, special cases (unit columns
pick out columns of S), linearity, the generation counts stated in Sec. 3.2,
and the expected-nonempty-rows formula of Sec. 3.1.
"""
import numpy as np
import pytest

import oracle
from paper_2310_15419_gb300 import inputs


def _dense(A):
    return A.to_scipy().toarray()


@pytest.mark.parametrize("dist", [oracle.PM1, oracle.UNIFORM, oracle.NORMAL])
@pytest.mark.parametrize("m,n,d,dens", [(60, 9, 17, 0.2), (64, 64, 64, 0.1),
                                        (300, 5, 130, 0.05), (1, 1, 1, 1.0)])
def test_brute_force_dense(dist, m, n, d, dens):
    A = inputs.integer_uniform(m, n, dens, seed=m * 7 + n)
    S = oracle.S_dense(dist, 11, 2, d, m)
    ref = S @ _dense(A)
    got3, _ = oracle.sketch_kji(m, n, d, dist, 11, 2, A.colptr, A.rowidx, A.values)
    got4, _ = oracle.sketch_jki(m, n, d, dist, 11, 2, A.colptr, A.rowidx, A.values)
    if dist == oracle.PM1:
        # +-1 S and integer A: every partial sum is an exact integer
        assert np.array_equal(got3, ref) and np.array_equal(got4, ref)
    else:
        scale = np.abs(S) @ np.abs(_dense(A)) + 1e-300
        assert np.all(np.abs(got3 - ref) <= 1e-13 * scale)
        assert np.all(np.abs(got4 - ref) <= 1e-13 * scale)


def test_unit_columns_select_columns_of_S():
    """A = [e_{j_0}, ..., e_{j_{n-1}}] gives A_hat(:, k) = S(:, j_k)."""
    m, d = 1000, 259
    js = np.array([0, 3, 127, 128, 999, 500], dtype=np.int32)
    colptr = np.arange(len(js) + 1, dtype=np.int32)
    for dist in (oracle.PM1, oracle.UNIFORM, oracle.NORMAL):
        got, _ = oracle.sketch_jki(m, len(js), d, dist, 5, 0, colptr, js,
                                   np.ones(len(js)))
        for k, j in enumerate(js):
            assert np.array_equal(got[:, k], oracle.S_column(dist, 5, 0, d, int(j)))


def test_linearity():
    m, n, d = 500, 12, 40
    A1 = inputs.float_uniform(m, n, 0.05, seed=1)
    A2 = inputs.float_uniform(m, n, 0.05, seed=2)
    S = A1.to_scipy() + A2.to_scipy()
    S.sort_indices()
    s1, _ = oracle.sketch_jki(m, n, d, oracle.UNIFORM, 3, 0, A1.colptr, A1.rowidx, A1.values)
    s2, _ = oracle.sketch_jki(m, n, d, oracle.UNIFORM, 3, 0, A2.colptr, A2.rowidx, A2.values)
    s12, _ = oracle.sketch_jki(m, n, d, oracle.UNIFORM, 3, 0, S.indptr, S.indices, S.data)
    assert np.allclose(s12, s1 + s2, rtol=0, atol=1e-12)


def test_generation_counts():
    """Sec. 3.2: Alg. 3 generates d*nnz numbers; Alg. 4 generates d per
    nonempty row (zero rows need no column of S)."""
    m, n, d = 2000, 30, 50
    A = inputs.integer_uniform(m, n, 0.01, seed=9)
    _, g3 = oracle.sketch_kji(m, n, d, oracle.PM1, 1, 0, A.colptr, A.rowidx, A.values)
    _, g4 = oracle.sketch_jki(m, n, d, oracle.PM1, 1, 0, A.colptr, A.rowidx, A.values)
    nonempty = np.unique(A.rowidx).size
    assert g3 == d * A.nnz
    assert g4 == d * nonempty
    assert nonempty < m  # this pattern has zero rows


def test_expected_nonempty_rows_formula():
    """Sec. 3.1: E[Y] = m1 (1 - (1 - rho)^n1) for a uniformly random pattern
    (using the parenthesisation of the optimisation problem, Eq. 3)."""
    m, n, rho = 200_000, 40, 0.01
    A = inputs.integer_uniform(m, n, rho, seed=4)
    Y = np.unique(A.rowidx).size
    EY = m * (1 - (1 - rho) ** n)
    sd = np.sqrt(m * (1 - (1 - rho) ** n) * (1 - rho) ** n)
    assert abs(Y - EY) < 6 * sd


def test_row_range_sample_equals_row_slice():
    m, n, d = 3000, 20, 33
    A = inputs.float_uniform(m, n, 0.02, seed=8)
    sub = A.row_slice(1200)
    a, _ = oracle.sketch_jki(m, n, d, oracle.NORMAL, 2, 0, A.colptr, A.rowidx,
                             A.values, 0, 1200)
    b, _ = oracle.sketch_jki(1200, n, d, oracle.NORMAL, 2, 0, sub.colptr,
                             sub.rowidx, sub.values)
    assert np.array_equal(a, b)


def test_empty_matrix_and_empty_columns():
    m, n, d = 100, 6, 10
    colptr = np.zeros(n + 1, dtype=np.int32)
    got, g = oracle.sketch_jki(m, n, d, oracle.UNIFORM, 1, 0, colptr,
                               np.zeros(0, np.int32), np.zeros(0))
    assert g == 0 and np.all(got == 0)


def test_scaling_trick_is_exact_for_uniform():
    """Sec. 3.3 'scaling trick': (S f)(A / f) = S A.  With f = 2^-24 and the
    odd-integer form of U(-1,1) the integer matrix S/f = 2u+1 is exact, so the
    product is unchanged bit for bit (powers of two scale exactly)."""
    m, n, d = 400, 7, 21
    A = inputs.float_uniform(m, n, 0.05, seed=12)
    S = oracle.S_dense(oracle.UNIFORM, 77, 0, d, m)
    Sint = S * 2.0**24
    assert np.all(Sint == np.round(Sint)) and np.all(np.abs(Sint) < 2**24)
    assert np.all(np.mod(Sint, 2) != 0)   # odd integers
    got, _ = oracle.sketch_kji(m, n, d, oracle.UNIFORM, 77, 0, A.colptr,
                               A.rowidx, A.values)
    ref = (Sint @ _dense(A)) * 2.0**-24
    assert np.allclose(got, ref, rtol=1e-14, atol=1e-14)


def test_paper_gflops_definition():
    """tests/golden/paper_tables.txt: the paper's GFLOP/s column equals
    2 d nnz / time (Table 'parallel', 1 thread, shar_te2-b2, d = 3n)."""
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "paper_tables.txt")
    rows = [l.split() for l in open(path) if l.strip() and not l.startswith("#")]
    for r in rows:
        if r[0] != "gflops":
            continue
        d, nnz, t, gf = int(r[2]), int(r[3]), float(r[4]), float(r[5])
        assert abs(2 * d * nnz / t / 1e9 - gf) < 0.01 * gf


@pytest.mark.parametrize("dist", [oracle.PM1, oracle.UNIFORM, oracle.NORMAL])
@pytest.mark.parametrize("threads", [1, 2, 3, 8])
def test_all_core_oracle_is_bit_identical_to_the_serial_one(dist, threads):
    """The OpenMP oracle splits the rows of A_hat between threads, so each
    element's additions keep the serial order: equal bits for float values,
    ragged d (not a multiple of the Philox block), dense-ish and empty rows,
    and a row sample."""
    A = inputs.float_uniform(3000, 37, 0.03, seed=41)
    for d in (1, 131, 517):
        ref, g1 = oracle.sketch_jki(A.m, A.n, d, dist, 9, 4, A.colptr, A.rowidx, A.values)
        got, g2 = oracle.sketch_jki_omp(A.m, A.n, d, dist, 9, 4, A.colptr, A.rowidx,
                                        A.values, threads=threads)
        assert g1 == g2 and np.array_equal(got, ref), d
    ref, _ = oracle.sketch_jki(A.m, A.n, 300, dist, 9, 0, A.colptr, A.rowidx, A.values,
                               700, 2100)
    got, _ = oracle.sketch_jki_omp(A.m, A.n, 300, dist, 9, 0, A.colptr, A.rowidx,
                                   A.values, 700, 2100, threads=threads)
    assert np.array_equal(got, ref)


def test_all_core_oracle_matches_brute_force():
    """Pinned on its own too: the materialised S times the dense A."""
    A = inputs.integer_uniform(200, 11, 0.1, seed=42)
    S = oracle.S_dense(oracle.PM1, 3, 1, 300, A.m)
    got, _ = oracle.sketch_jki_omp(A.m, A.n, 300, oracle.PM1, 3, 1, A.colptr, A.rowidx,
                                   A.values, threads=4)
    assert np.array_equal(got, S @ _dense(A))
    assert oracle.max_threads() >= 1
