"""Seeded synthetic inputs for the sketch and least-squares workloads.

This module only draws test matrices and right-hand sides.  It holds none of
the sketch's or the solver's arithmetic, and it is the one module that both the
CPU oracle's tests and the CUDA path's tests/benchmark use.  The random matrix
S is NOT drawn here: S is a pure function of (seed, stream, i, j) computed
independently by the CUDA kernels and by the oracle.

Workloads (synthetic stand-ins for the SuiteSparse matrices of the paper's
Tables "matrix:name" and "matrix:name_extended", which are not available):

  plain_small   m=50,000  n=200   density 1%, values uniform on {-3..3}\\{0}
                (FP32), d=400, +-1 S, seed 1.
  skew_large    m=2,000,000  n=1,000  d=3,000; per-row nnz k = min(n, ceil(X))
                with X Pareto(alpha=2.1) scaled so E[k] = 5 (~1e7 nnz); the k
                columns of a row are uniform without replacement; values
                U(-1,1) FP32.
  batched       256 instances: m ~ logU[1e4, 5e5], n ~ U[50, 1000],
                d = round(c n) with c ~ U[1.5, 4], density ~ logU[5e-4, 2e-2],
                values N(0,1) FP32.
  lsq_mixed     m=1,000,000  n=500  density 0.2%, values BF16(z * s_k) with
                z ~ N(0,1) and column scales s_k ~ logU[1e-2, 1e2];
                b = A x* + 1e-6 noise, x* ~ N(0, I); d = 2n.
  serve         Poisson arrivals, m ~ logU[5e4, 2e6], n ~ U[100, 2000],
                density ~ logU[5e-4, 1e-2], values N(0,1) FP32, d = 2n.
  abnormal_a/b/c  the exotic patterns of the paper's Table "extreme_examples"
                (m=100,000, n=10,000, density ~1e-3).

All draws use numpy's PCG64 seeded explicitly.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

DTYPE_F32 = 0
DTYPE_BF16 = 1


@dataclasses.dataclass
class CSC:
    """A sparse m x n matrix in CSC (0-based, rows sorted within a column)."""
    m: int
    n: int
    colptr: np.ndarray          # int32, n + 1
    rowidx: np.ndarray          # int32, nnz
    values: np.ndarray          # float32, nnz (exact values of the stored dtype)
    dtype: int = DTYPE_F32      # storage dtype of the device copy
    values_bf16: np.ndarray | None = None  # uint16 bit patterns when dtype=BF16

    @property
    def nnz(self) -> int:
        return int(self.colptr[-1])

    def row_slice(self, row_hi: int) -> "CSC":
        """The submatrix of rows [0, row_hi) (same n), as a new CSC."""
        keep = self.rowidx < row_hi
        counts = np.add.reduceat(keep.astype(np.int64), self.colptr[:-1]) \
            if self.nnz else np.zeros(self.n, np.int64)
        # reduceat on empty segments returns the element at the index; fix up
        seglen = np.diff(self.colptr)
        counts = np.where(seglen == 0, 0, counts)
        colptr = np.zeros(self.n + 1, dtype=np.int64)
        np.cumsum(counts, out=colptr[1:])
        vb = None if self.values_bf16 is None else self.values_bf16[keep]
        return CSC(row_hi, self.n, colptr.astype(np.int32),
                   self.rowidx[keep].copy(), self.values[keep].copy(),
                   self.dtype, vb)

    def columns(self, cols) -> "CSC":
        """The submatrix of the given columns (same m, columns in the given
        order), as a new CSC: column t of the result is column cols[t]."""
        cols = np.asarray(cols, dtype=np.int64)
        lens = (self.colptr[cols + 1] - self.colptr[cols]).astype(np.int64)
        colptr = np.zeros(cols.size + 1, dtype=np.int64)
        np.cumsum(lens, out=colptr[1:])
        take = np.concatenate([np.arange(self.colptr[k], self.colptr[k + 1])
                               for k in cols]) if cols.size else np.zeros(0, np.int64)
        take = take.astype(np.int64)
        vb = None if self.values_bf16 is None else self.values_bf16[take]
        return CSC(self.m, int(cols.size), colptr.astype(np.int32),
                   self.rowidx[take].copy(), self.values[take].copy(), self.dtype, vb)

    def to_scipy(self):
        import scipy.sparse as sp
        return sp.csc_matrix((self.values.astype(np.float64), self.rowidx,
                              self.colptr), shape=(self.m, self.n))


def _rng(seed) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def _csc_from_keys(keys: np.ndarray, m: int, n: int):
    """keys = col * m + row, unique and sorted -> (colptr, rowidx)."""
    cols = keys // m
    rows = (keys - cols * m).astype(np.int32)
    counts = np.bincount(cols, minlength=n)
    colptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=colptr[1:])
    if colptr[-1] >= 2**31:
        raise ValueError("nnz does not fit int32")
    return colptr.astype(np.int32), rows


def uniform_pattern(m: int, n: int, density: float, rng) -> tuple:
    """Each entry nonzero independently with probability `density`.

    Walks the m x n positions in column-major order with Geometric(density)
    gaps between successive nonzeros -- exactly the iid Bernoulli pattern,
    produced already sorted by (column, row)."""
    total = int(m) * int(n)
    if density <= 0.0 or total == 0:
        return _csc_from_keys(np.zeros(0, dtype=np.int64), m, n)
    if density >= 1.0:
        return _csc_from_keys(np.arange(total, dtype=np.int64), m, n)
    parts, last = [], -1
    while True:
        want = int((total - last) * density * 1.05) + 64
        pos = last + np.cumsum(rng.geometric(density, size=want))
        if pos[-1] >= total:
            parts.append(pos[pos < total])
            break
        parts.append(pos)
        last = int(pos[-1])
    keys = np.concatenate(parts).astype(np.int64)   # col * m + row
    return _csc_from_keys(keys, m, n)


def pareto_xmin_for_mean(alpha: float, mean: float, n: int) -> float:
    """x_min such that E[min(n, ceil(X))] = mean, X ~ Pareto(alpha, x_min).

    P(ceil X >= t) = P(X > t - 1) = min(1, (x_min / (t - 1))^(alpha - 1))."""
    t = np.arange(2, n + 1, dtype=np.float64) - 1.0

    def expect(xm):
        return 1.0 + np.minimum(1.0, (xm / t) ** (alpha - 1.0)).sum()

    lo, hi = 1e-6, float(n)
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if expect(mid) < mean:
            lo = mid
        else:
            hi = mid
    return 0.5 * (lo + hi)


def _distinct_per_row(rows: np.ndarray, k: np.ndarray, n: int, rng):
    """For each row r in `rows`, k[r] distinct columns uniform in [0, n).

    Exact uniform k-subsets: draw with replacement, drop duplicates, re-draw
    the deficit (rows are independent, so the accepted set stays uniform).
    Returns sorted row-major keys row * n + col."""
    need = k.astype(np.int64).copy()
    base = np.zeros(0, dtype=np.int64)      # sorted, unique
    extra = []
    have = np.zeros(rows.size, dtype=np.int64)
    for it in range(200):
        todo = need - have
        sel = np.nonzero(todo > 0)[0]
        if sel.size == 0:
            break
        r = np.repeat(rows[sel], todo[sel])
        new = np.unique(r * n + rng.integers(0, n, size=r.size, dtype=np.int64))
        if it == 0:
            base = new
        else:
            pos = np.searchsorted(base, new)
            pos = np.minimum(pos, base.size - 1)
            fresh = new[base[pos] != new] if base.size else new
            for e in extra:
                if fresh.size == 0:
                    break
                if e.size == 0:
                    continue
                p2 = np.minimum(np.searchsorted(e, fresh), e.size - 1)
                fresh = fresh[e[p2] != fresh]
            extra.append(fresh)
            new = fresh
        # each round draws at most a row's deficit, so no row overflows
        add = np.bincount(np.searchsorted(rows, new // n), minlength=rows.size)
        have += add
    keys = np.concatenate([base] + extra) if extra else base
    keys.sort()
    return keys


def powerlaw_row_pattern(m: int, n: int, alpha: float, mean: float, rng):
    """Per-row nnz k = min(n, ceil(X)), X ~ Pareto(alpha, x_min) with
    E[k] = mean; the k columns of each row uniform without replacement."""
    xmin = pareto_xmin_for_mean(alpha, mean, n)
    u = 1.0 - rng.random(m)                       # (0, 1]
    x = xmin * u ** (-1.0 / (alpha - 1.0))
    k = np.minimum(n, np.ceil(x)).astype(np.int64)
    rows = np.arange(m, dtype=np.int64)
    heavy = k > n // 4
    parts = []
    # heavy rows: the first k entries of a random permutation of the columns
    hrows = rows[heavy]
    for c0 in range(0, hrows.size, 4096):
        hr = hrows[c0:c0 + 4096]
        perm = np.argsort(rng.random((hr.size, n)), axis=1)
        take = np.arange(n)[None, :] < k[hr][:, None]
        parts.append((hr[:, None] * n + perm)[take])
    lrows = rows[~heavy]
    parts.append(_distinct_per_row(lrows, k[lrows], n, rng))
    rk = np.concatenate(parts)
    r, c = rk // n, rk % n
    keys = np.sort(c * m + r)                     # column-major order
    return _csc_from_keys(keys, m, n)


def to_bf16_bits(x: np.ndarray) -> np.ndarray:
    """Round float32 to bfloat16 (nearest, ties to even); return uint16 bits."""
    b = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32)
    rounding = ((b >> 16) & 1) + np.uint32(0x7FFF)
    return ((b + rounding) >> 16).astype(np.uint16)


def bf16_bits_to_f32(h: np.ndarray) -> np.ndarray:
    return (h.astype(np.uint32) << 16).view(np.float32)


# --------------------------------------------------------------------------
# Named workloads
# --------------------------------------------------------------------------
def plain_small(seed: int = 1, m: int = 50_000, n: int = 200,
                density: float = 0.01) -> CSC:
    rng = _rng(seed)
    colptr, rowidx = uniform_pattern(m, n, density, rng)
    nz = rng.integers(1, 4, size=rowidx.size) * rng.choice([-1, 1], size=rowidx.size)
    return CSC(m, n, colptr, rowidx, nz.astype(np.float32))


def integer_uniform(m: int, n: int, density: float, seed: int) -> CSC:
    """Uniform pattern with integer values in {-3..3}\\{0} (any size)."""
    return plain_small(seed=seed, m=m, n=n, density=density)


def float_uniform(m: int, n: int, density: float, seed: int,
                  law: str = "uniform") -> CSC:
    rng = _rng(seed)
    colptr, rowidx = uniform_pattern(m, n, density, rng)
    if law == "uniform":
        v = rng.uniform(-1.0, 1.0, size=rowidx.size)
    else:
        v = rng.standard_normal(size=rowidx.size)
    return CSC(m, n, colptr, rowidx, v.astype(np.float32))


def heavy_column(m: int, n: int, heavy_nnz: int, density: float, seed: int,
                 heavy_col: int = 0) -> CSC:
    """A uniform pattern of the given density whose column `heavy_col` is
    replaced by `heavy_nnz` distinct rows chosen uniformly; values U(-1,1)."""
    rng = _rng(seed)
    colptr, rowidx = uniform_pattern(m, n, density, rng)
    heavy = np.sort(rng.choice(m, size=heavy_nnz, replace=False)).astype(np.int32)
    lens = np.diff(colptr).astype(np.int64)
    parts = [rowidx[colptr[k]:colptr[k + 1]] if k != heavy_col else heavy for k in range(n)]
    lens[heavy_col] = heavy_nnz
    cp = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(lens, out=cp[1:])
    rows = np.concatenate(parts).astype(np.int32)
    v = rng.uniform(-1.0, 1.0, size=rows.size).astype(np.float32)
    return CSC(m, n, cp.astype(np.int32), rows, v)


def skew_large(seed: int = 2, m: int = 2_000_000, n: int = 1000,
               alpha: float = 2.1, mean: float = 5.0) -> CSC:
    rng = _rng(seed)
    colptr, rowidx = powerlaw_row_pattern(m, n, alpha, mean, rng)
    v = rng.uniform(-1.0, 1.0, size=rowidx.size).astype(np.float32)
    return CSC(m, n, colptr, rowidx, v)


SKEW_LARGE_D = 3000
PLAIN_SMALL_D = 400


def batched_specs(seed: int = 3, count: int = 256, scale: float = 1.0):
    """(m, n, d, density) per instance; `scale` shrinks m for quick tests."""
    rng = _rng(seed)
    m = np.exp(rng.uniform(math.log(1e4), math.log(5e5), size=count))
    n = rng.integers(50, 1001, size=count)
    c = rng.uniform(1.5, 4.0, size=count)
    dens = np.exp(rng.uniform(math.log(5e-4), math.log(2e-2), size=count))
    out = []
    for t in range(count):
        mm = max(int(n[t]) + 1, int(round(m[t] * scale)))
        out.append((mm, int(n[t]), int(round(c[t] * n[t])), float(dens[t])))
    return out


def batched(seed: int = 3, count: int = 256, scale: float = 1.0):
    """List of (CSC, d) for the batched uneven workload; values N(0,1)."""
    specs = batched_specs(seed, count, scale)
    out = []
    for t, (m, n, d, dens) in enumerate(specs):
        a = float_uniform(m, n, dens, seed=seed * 100_003 + t, law="normal")
        out.append((a, d))
    return out


def lsq_mixed(seed: int = 4, m: int = 1_000_000, n: int = 500,
              density: float = 0.002, noise: float = 1e-6):
    """(CSC with BF16 values, b (float64), x_star (float64))."""
    rng = _rng(seed)
    colptr, rowidx = uniform_pattern(m, n, density, rng)
    z = rng.standard_normal(size=rowidx.size)
    scales = np.exp(rng.uniform(math.log(1e-2), math.log(1e2), size=n))
    col_of = np.repeat(np.arange(n), np.diff(colptr))
    bits = to_bf16_bits((z * scales[col_of]).astype(np.float32))
    vals = bf16_bits_to_f32(bits)
    A = CSC(m, n, colptr, rowidx, vals, DTYPE_BF16, bits)
    x_star = rng.standard_normal(size=n)
    b = A.to_scipy() @ x_star + noise * rng.standard_normal(size=m)
    return A, b, x_star


def lsq_problem(m: int, n: int, density: float, seed: int, noise: float = 1e-6,
                law: str = "normal", col_scale_decades: float = 0.0):
    """A generic overdetermined LS problem: (CSC f32, b, x_star)."""
    rng = _rng(seed)
    colptr, rowidx = uniform_pattern(m, n, density, rng)
    z = rng.standard_normal(size=rowidx.size) if law == "normal" else \
        rng.uniform(-1, 1, size=rowidx.size)
    if col_scale_decades > 0:
        s = 10.0 ** rng.uniform(-col_scale_decades, col_scale_decades, size=n)
        z = z * s[np.repeat(np.arange(n), np.diff(colptr))]
    A = CSC(m, n, colptr, rowidx, z.astype(np.float32))
    x_star = rng.standard_normal(size=n)
    b = A.to_scipy() @ x_star + noise * rng.standard_normal(size=m)
    return A, b, x_star


def serve_requests(seed: int = 5, rate: float = 200.0, duration_s: float = 60.0,
                   m_range=(5e4, 2e6), n_range=(100, 2000),
                   dens_range=(5e-4, 1e-2), count: int | None = None):
    """Poisson arrival times and (m, n, density) per request: the arrivals
    within `duration_s`, or the first `count` arrivals when count is given."""
    rng = _rng(seed)
    t, out = 0.0, []
    while True:
        t += rng.exponential(1.0 / rate)
        if (count is None and t > duration_s) or (count is not None and len(out) >= count):
            break
        m = int(np.exp(rng.uniform(math.log(m_range[0]), math.log(m_range[1]))))
        n = int(rng.integers(n_range[0], n_range[1] + 1))
        dens = float(np.exp(rng.uniform(math.log(dens_range[0]),
                                        math.log(dens_range[1]))))
        out.append((t, max(m, 2 * n + 1), n, dens))
    return out


def abnormal(kind: str, seed: int = 6, m: int = 100_000, n: int = 10_000,
             every: int = 1000) -> CSC:
    """Table 'extreme_examples' patterns, density ~1e-3, values U(-1,1).

    a: every `every`-th row dense, all other rows zero
    b: ~2998/3000 of the nonzeros in the middle third of the columns
    c: every `every`-th column dense, all other columns zero"""
    rng = _rng(seed)
    if kind == "a":
        rows = np.arange(0, m, every, dtype=np.int64)
        keys = (np.arange(n, dtype=np.int64)[:, None] * m + rows[None, :]).ravel()
        keys.sort()
        colptr, rowidx = _csc_from_keys(keys, m, n)
    elif kind == "c":
        cols = np.arange(0, n, every, dtype=np.int64)
        keys = (cols[:, None] * m + np.arange(m, dtype=np.int64)[None, :]).ravel()
        colptr, rowidx = _csc_from_keys(keys, m, n)
    elif kind == "b":
        total = int(1e-3 * m * n)
        mid = total * 2998 // 3000
        lo, hi = n // 3, 2 * n // 3
        c_mid = rng.integers(lo, hi, size=mid)
        c_rest = rng.integers(0, n, size=total - mid)
        cols = np.concatenate([c_mid, c_rest]).astype(np.int64)
        rows = rng.integers(0, m, size=cols.size, dtype=np.int64)
        keys = np.unique(cols * m + rows)
        colptr, rowidx = _csc_from_keys(keys, m, n)
    else:
        raise ValueError(kind)
    v = rng.uniform(-1.0, 1.0, size=rowidx.size).astype(np.float32)
    return CSC(m, n, colptr, rowidx, v)
