"""Batched uneven sketches in one persistent launch (through the C ABI):
every instance equals its own single-instance sketch and the oracle, the
tuned launch replays from a captured CUDA graph, and instance i uses Philox
stream id i (one seed, independent S per instance)."""
import numpy as np
import pytest

import oracle
from paper_2310_15419_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2310_15419_gb300 import capi  # noqa: E402

DISTS = {"pm1": oracle.PM1, "uniform": oracle.UNIFORM, "normal": oracle.NORMAL}


def _instances(count, integer, seed=3, scale=0.04):
    specs = inputs.batched_specs(seed, count, scale)
    out = []
    for t, (m, n, d, dens) in enumerate(specs):
        if integer:
            A = inputs.integer_uniform(m, n, dens, seed=1000 + t)
        else:
            A = inputs.float_uniform(m, n, dens, seed=1000 + t, law="normal")
        out.append((A, d))
    return out


@pytest.mark.parametrize("dist", ["pm1", "uniform", "normal"])
def test_batch_matches_single_and_oracle(dist):
    integer = dist == "pm1"
    inst = _instances(24, integer)
    sks = [capi.Sketch(A.m, A.n, d, dist, seed=1, stream_id=t)
           for t, (A, d) in enumerate(inst)]
    mats = [capi.DeviceCSC(A) for A, _ in inst]
    batch = capi.Batch(sks, mats)
    outs = batch.apply()
    torch.cuda.synchronize()
    assert batch.status() == capi.SKETCH_OK
    for t, ((A, d), sk, dA, o) in enumerate(zip(inst, sks, mats, outs)):
        got = o.cpu().numpy().astype(np.float64).T
        single = sk.apply(dA).cpu().numpy().astype(np.float64).T
        if t % 6 == 0:
            ref, _ = oracle.sketch_jki(A.m, A.n, d, DISTS[dist], 1, t, A.colptr,
                                       A.rowidx, A.values)
        else:
            ref = None
        if integer:
            assert np.array_equal(got, single)
            if ref is not None:
                assert np.array_equal(got, ref)
        else:
            den = np.linalg.norm(single)
            assert np.linalg.norm(got - single) <= 1e-6 * den
            if ref is not None:
                assert np.linalg.norm(got - ref) <= 1e-6 * np.linalg.norm(ref)
    batch.close()


def test_batch_graph_replay():
    inst = _instances(16, True, seed=5)
    sks = [capi.Sketch(A.m, A.n, d, "pm1", seed=9, stream_id=t)
           for t, (A, d) in enumerate(inst)]
    mats = [capi.DeviceCSC(A) for A, _ in inst]
    batch = capi.Batch(sks, mats)
    first = [o.clone() for o in batch.apply()]
    for o in batch.outs:
        o.zero_()
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            batch.apply(stream=s)
    for o in batch.outs:
        o.zero_()
    torch.cuda.synchronize()
    for _ in range(3):
        g.replay()
    torch.cuda.synchronize()
    for a, b in zip(first, batch.outs):
        assert torch.equal(a, b)
    info = batch.info()
    assert info["q_tiles"] in (1, 2, 4) and info["items"] > 0
    batch.close()


def test_batch_rejects_mixed_distributions():
    A = inputs.integer_uniform(500, 5, 0.05, seed=1)
    sks = [capi.Sketch(500, 5, 16, "pm1"), capi.Sketch(500, 5, 16, "uniform")]
    mats = [capi.DeviceCSC(A), capi.DeviceCSC(A)]
    with pytest.raises(capi.SketchError) as e:
        capi.Batch(sks, mats)
    assert e.value.code == capi.SKETCH_ERR_UNSUPPORTED
