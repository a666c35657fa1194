"""Continuous-batching least-squares server (through the C ABI): requests of
mixed (m, n, density) overlap on the GPU; every result equals the same
request solved alone (same kernels, deterministic reductions), reaches the
error gate, and carries consistent timestamps; a request larger than the
memory budget is refused without being run."""
import numpy as np
import pytest

import oracle
from paper_2310_15419_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2310_15419_gb300 import capi  # noqa: E402


def _problems(count, seed=40):
    rng = np.random.default_rng(seed)
    out = []
    for t in range(count):
        m = int(np.exp(rng.uniform(np.log(5_000), np.log(60_000))))
        n = int(rng.integers(20, 200))
        dens = float(np.exp(rng.uniform(np.log(2e-3), np.log(2e-2))))
        A, b, _ = inputs.lsq_problem(m, n, dens, seed=seed * 1000 + t, noise=1e-3)
        out.append((A, b))
    return out


def _alone(A, b, dist, seed):
    sk = capi.Sketch(A.m, A.n, 2 * A.n, dist, seed=seed)
    sk.set_autotune(False)
    x, info = sk.lsq_solve(capi.DeviceCSC(A), torch.from_numpy(b).cuda(), tol=1e-10)
    sk.close()
    return x.cpu().numpy(), info


def test_mixed_requests_equal_alone_results():
    probs = _problems(12)
    srv = capi.Server(slots=4, mem_budget=8 << 30, dist="uniform", seed=7)
    ids = [srv.submit(A, b) for A, b in probs]
    srv.drain()
    res = {}
    while len(res) < len(ids):
        for r in srv.poll(64, wait_ms=100):
            res[r["id"]] = r
    srv.close()
    for rid, (A, b) in zip(ids, probs):
        r = res[rid]
        assert r["status"] == capi.SKETCH_OK
        assert r["t_submit"] <= r["t_start"] <= r["t_done"]
        xa, ia = _alone(A, b, "uniform", 7)
        assert np.array_equal(r["x"], xa)
        assert r["iters"] == ia["iters"]
        e = oracle.ls_error(A.m, A.n, A.colptr, A.rowidx, A.values, b, r["x"])
        assert e <= 1e-10


def test_requests_overlap_and_budget_refusal():
    probs = _problems(8, seed=41)
    srv = capi.Server(slots=4, mem_budget=8 << 30, dist="pm1", seed=1)
    for A, b in probs:
        srv.submit(A, b)
    srv.drain()
    res = srv.poll(64)
    srv.close()
    # some requests ran at the same time (their [start, done] intervals meet)
    spans = sorted((r["t_start"], r["t_done"]) for r in res)
    overlap = any(spans[i + 1][0] < spans[i][1] for i in range(len(spans) - 1))
    assert overlap
    # a budget below one request's footprint: refused, never run
    A, b = probs[0]
    tiny = capi.Server(slots=1, mem_budget=1 << 10, dist="pm1", seed=1)
    tiny.submit(A, b)
    tiny.drain()
    (r,) = tiny.poll(4)
    tiny.close()
    assert r["status"] == capi.SKETCH_ERR_OOM
