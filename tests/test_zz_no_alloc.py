"""sketch_apply_noalloc through the C ABI (GPU): against the regular entry
point and against the FP64 oracle.

The no-allocation entry point exists for callers that cannot let a library
allocate device memory while they run (another allocator owns the device's
memory, or cudaMalloc/cudaFree would stall a latency-critical loop).  It must
give the same A_hat as the regular entry point and as the oracle -- bit for
bit for +-1 S with integer-valued A, within the 1e-6 relative Frobenius
tolerance otherwise -- on two calls in a row (the second call finds the
first call's data in the shared fixed scratch), including inputs at the
entry point's limits (262,144 rows, about a million nonzeros, one column of
150,000 nonzeros summed in one piece).  This file sorts last so a failure
here leaves every other test already run.
"""
import numpy as np
import pytest

import oracle
from paper_2310_15419_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2310_15419_gb300 import capi  # noqa: E402

TOL = 1e-6
DISTS = {"pm1": oracle.PM1, "uniform": oracle.UNIFORM, "normal": oracle.NORMAL}
MAX_ROWS, MAX_NNZ = 262_144, 1_048_576


def _rel(a, b):
    den = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (den if den > 0 else 1.0)


def _oracle(A, d, dist, seed):
    ref, _ = oracle.sketch_jki(A.m, A.n, d, DISTS[dist], seed, 0, A.colptr, A.rowidx,
                               A.values)
    return ref.T  # n x d, the layout of the output tensor


def _check_twice(A, d, dist, seed, ref_apply=True):
    dA = capi.DeviceCSC(A)
    ref = _oracle(A, d, dist, seed)
    exact = dist == "pm1" and np.all(A.values == np.round(A.values))
    reg = None
    if ref_apply:
        ref_sk = capi.Sketch(A.m, A.n, d, dist, seed=seed)
        reg = ref_sk.apply(dA).cpu().numpy().astype(np.float64)
        ref_sk.close()
    sk = capi.Sketch(A.m, A.n, d, dist, seed=seed)
    out = torch.empty((A.n, d), dtype=torch.float32, device="cuda")
    for _ in range(2):
        out.fill_(float("nan"))
        sk.apply_noalloc(dA, out)
        torch.cuda.synchronize()
        got = out.cpu().numpy().astype(np.float64)
        if exact:
            assert np.array_equal(got, ref)
            if reg is not None:
                assert np.array_equal(got, reg)
        else:
            assert _rel(got, ref) <= TOL
            if reg is not None:
                assert _rel(got, reg) <= TOL
    sk.close()


@pytest.mark.parametrize("dist", ["pm1", "uniform", "normal"])
def test_noalloc_matches_apply_and_oracle_twice(dist):
    for A in (inputs.integer_uniform(120_000, 64, 0.004, seed=21),
              inputs.float_uniform(200_000, 300, 0.001, seed=22)):
        _check_twice(A, 450, dist, seed=5)


@pytest.mark.parametrize("dist", ["pm1", "uniform", "normal"])
def test_noalloc_at_its_limits_matches_oracle(dist):
    """262,144 rows and close to 1,048,576 nonzeros, one column holding
    150,000 of them: the compensated sums keep that column within the
    tolerance although it is summed in one piece; n = 1000 > 768 also spans
    two column blocks of the kernel."""
    A = inputs.heavy_column(MAX_ROWS, 1000, 150_000, 0.0033, seed=24, heavy_col=777)
    assert A.m == MAX_ROWS and 900_000 < A.nnz <= MAX_NNZ
    _check_twice(A, 96, dist, seed=3, ref_apply=False)
    # the heavy column alone, at a ragged d: the gate holds per column too
    col = A.columns([777])
    _check_twice(col, 203, dist, seed=3, ref_apply=False)


def test_noalloc_integer_long_column_exact():
    """+-1 S with integer values: exact in any order of the atomic adds."""
    rng = np.random.default_rng(25)
    rows = np.sort(rng.choice(MAX_ROWS, size=120_000, replace=False)).astype(np.int32)
    vals = (rng.integers(1, 4, size=rows.size) * rng.choice([-1, 1], size=rows.size))
    A = inputs.CSC(MAX_ROWS, 1, np.array([0, rows.size], np.int32), rows,
                   vals.astype(np.float32))
    _check_twice(A, 130, "pm1", seed=8, ref_apply=False)


def test_noalloc_rejects_inputs_beyond_the_fixed_scratch():
    A = inputs.integer_uniform(300_000, 4, 0.001, seed=23)   # m > 262,144
    sk = capi.Sketch(A.m, A.n, 64, "pm1", seed=1)
    out = torch.empty((A.n, 64), dtype=torch.float32, device="cuda")
    with pytest.raises(capi.SketchError) as e:
        sk.apply_noalloc(capi.DeviceCSC(A), out)
    assert e.value.code == capi.SKETCH_ERR_UNSUPPORTED
    sk.close()
