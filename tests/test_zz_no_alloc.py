"""sketch_apply_noalloc against sketch_apply, through the C ABI (GPU).

The no-allocation entry point exists for callers that cannot let a library
allocate device memory while they run (another allocator owns the device's
memory, or cudaMalloc/cudaFree would stall a latency-critical loop).  It must
give the same A_hat as the regular entry point -- bit for bit for +-1 S with
integer-valued A, within the 1e-6 relative Frobenius tolerance otherwise --
on two calls in a row (the second call finds the first call's data in the
shared fixed scratch).  This file sorts last so a failure here leaves every
other test already run.
"""
import numpy as np
import pytest

from paper_2310_15419_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2310_15419_gb300 import capi  # noqa: E402

TOL = 1e-6


def _rel(a, b):
    den = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (den if den > 0 else 1.0)


@pytest.mark.parametrize("dist", ["pm1", "uniform", "normal"])
def test_noalloc_matches_apply_twice(dist):
    cases = [inputs.integer_uniform(120_000, 64, 0.004, seed=21),
             inputs.float_uniform(200_000, 300, 0.001, seed=22)]
    for A in cases:
        d = 450
        dA = capi.DeviceCSC(A)
        ref_sk = capi.Sketch(A.m, A.n, d, dist, seed=5)
        ref = ref_sk.apply(dA).cpu().numpy().astype(np.float64)
        sk = capi.Sketch(A.m, A.n, d, dist, seed=5)
        out = torch.empty((A.n, d), dtype=torch.float32, device="cuda")
        for _ in range(2):
            out.fill_(float("nan"))
            sk.apply_noalloc(dA, out)
            torch.cuda.synchronize()
            got = out.cpu().numpy().astype(np.float64)
            exact = dist == "pm1" and np.all(A.values == np.round(A.values))
            if exact:
                assert np.array_equal(got, ref)
            else:
                assert _rel(got, ref) <= TOL
        sk.close()
        ref_sk.close()


def test_noalloc_rejects_inputs_beyond_the_fixed_scratch():
    A = inputs.integer_uniform(300_000, 4, 0.001, seed=23)   # m > 262,144
    sk = capi.Sketch(A.m, A.n, 64, "pm1", seed=1)
    out = torch.empty((A.n, 64), dtype=torch.float32, device="cuda")
    with pytest.raises(capi.SketchError) as e:
        sk.apply_noalloc(capi.DeviceCSC(A), out)
    assert e.value.code == capi.SKETCH_ERR_UNSUPPORTED
    sk.close()
