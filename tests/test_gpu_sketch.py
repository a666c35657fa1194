"""Parity of the CUDA sketch (through the C ABI) with the FP64 CPU oracle.

Bar: bit-exact for +-1 S with integer-valued A (every partial sum is an
exact integer in FP32); relative Frobenius error <= 1e-6 against FP64 for
FP32 values and U / N entries of S; S itself bit-exact for +-1 and U and
within a few FP32 ulps for N (Box-Muller uses CUDA's logf / sqrtf /
sincospif on the device and FP64 libm in the oracle).
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

DISTS = {"pm1": oracle.PM1, "uniform": oracle.UNIFORM, "normal": oracle.NORMAL}
TOL = 1e-6


def rel_fro(got, ref):
    den = np.linalg.norm(ref)
    return np.linalg.norm(got - ref) / (den if den > 0 else 1.0)


def gpu_sketch(A, d, dist, seed=1, stream_id=0, plan=None):
    sk = capi.Sketch(A.m, A.n, d, dist, seed=seed, stream_id=stream_id)
    if plan:
        sk.set_plan(**plan)
    dA = capi.DeviceCSC(A)
    out = sk.apply(dA)
    torch.cuda.synchronize()
    st = sk.device_status()
    sk.close()
    assert st == capi.SKETCH_OK
    return out.cpu().numpy().astype(np.float64).T  # d x n


def oracle_sketch(A, d, dist, seed=1, stream_id=0):
    ref, _ = oracle.sketch_jki(A.m, A.n, d, DISTS[dist], seed, stream_id,
                               A.colptr, A.rowidx, A.values)
    return ref


REGEN_PLANS = [dict(mode=capi.SKETCH_MODE_REGEN, q_tiles=q, split=s)
               for q in (1, 2, 3, 4) for s in (1, 2, 4, 8)]
PANEL_PLANS = [dict(mode=capi.SKETCH_MODE_PANEL, n_block=nb, row_groups=g)
               for nb, g in ((37, 1), (16, 3), (5, 7), (37, 64))]
TILE_PLANS = [dict(mode=capi.SKETCH_MODE_TILE, panel_rows=r, row_groups=g,
                   cols_per_warp=c, tile_acc=t)
              for r, g, c, t in ((1024, 1, 4, 0), (768, 3, 16, 0), (100, 7, 64, 0),
                                 (8, 50, 4, 0), (512, 3, 32, 1), (8, 50, 32, 1))]


# ---------------------------------------------------------------- generator
def test_philox_matches_oracle():
    rng = np.random.default_rng(0)
    ctr = rng.integers(0, 2**32, size=(20000, 4), dtype=np.uint64)
    ctr[0] = 0
    ctr[1] = 2**32 - 1
    for seed in (0, 1, 0xFFFFFFFFFFFFFFFF, 0x0123456789ABCDEF):
        run, keyed = capi.debug_philox(
            torch.from_numpy(ctr.astype(np.uint32).view(np.int32)).cuda(), seed, both=True)
        dev = run.cpu().numpy().view(np.uint32)
        # the precomputed-round-key form gives the same blocks everywhere
        assert np.array_equal(dev, keyed.cpu().numpy().view(np.uint32))
        key = np.array([seed & 0xFFFFFFFF, seed >> 32], dtype=np.uint32)
        for t in list(range(50)) + [19999]:
            assert np.array_equal(dev[t], oracle.philox4x32_10(ctr[t].astype(np.uint32), key))


@pytest.mark.parametrize("dist", ["pm1", "uniform", "normal"])
def test_S_entries_match_oracle(dist):
    rng = np.random.default_rng(1)
    i = rng.integers(0, 5000, size=4000)
    j = rng.integers(0, 2**31 - 1, size=4000)
    i[:8] = [0, 1, 2, 3, 127, 128, 4999, 31]
    seed, stream = 0xDEADBEEF12345678, 5
    got = capi.debug_S(DISTS[dist], seed, stream, torch.from_numpy(i).cuda(),
                       torch.from_numpy(j).cuda()).cpu().numpy()
    ref = np.array([oracle.S_entry(DISTS[dist], seed, stream, int(a), int(b))
                    for a, b in zip(i, j)])
    if dist == "normal":
        assert np.all(np.abs(got - ref) <= 4e-7 * np.maximum(1.0, np.abs(ref)))
    else:
        assert np.array_equal(got.astype(np.float64), ref)


def test_normal_transform_matches_oracle_at_the_extremes():
    """The N(0,1) transform on chosen word pairs: radius words at both ends
    of u1 (u1 -> 1 gives a tiny r, u1 = 2^-24 the largest), every octant
    boundary of the angle, and random pairs; each output within 4e-7
    max(1, |z|) of the oracle's FP64 Box-Muller (Sec. 4.2)."""
    rng = np.random.default_rng(11)
    top = np.arange(2**24 - 4096, 2**24, dtype=np.uint64)        # u1 -> 1
    low = np.arange(0, 4096, dtype=np.uint64)                     # u1 -> 0
    ang = np.array([(o * 2**21 + d) % 2**24 for o in range(8) for d in (-2, -1, 0, 1, 2)])
    rad_words = np.concatenate([top, low, np.repeat(rng.integers(0, 2**24, 8), ang.size),
                                rng.integers(0, 2**24, 100_000)]).astype(np.uint64)
    ang_words = np.concatenate([np.full(top.size, 12345), np.full(low.size, 2**22 + 7),
                                np.tile(ang, 8), rng.integers(0, 2**24, 100_000)]).astype(np.uint64)
    low_bits = rng.integers(0, 256, size=(rad_words.size, 2)).astype(np.uint64)
    w = np.stack([(rad_words << 8) | low_bits[:, 0], (ang_words << 8) | low_bits[:, 1]], axis=1)
    got = capi.debug_normal_pair(torch.from_numpy(w.astype(np.uint32).view(np.int32)).cuda())
    got = got.cpu().numpy().astype(np.float64)
    ref = np.array([[oracle.normal_from_words(int(a), int(b), 0),
                     oracle.normal_from_words(int(a), int(b), 1)] for a, b in w])
    err = np.abs(got - ref) / np.maximum(1.0, np.abs(ref))
    assert err.max() <= 4e-7, (err.max(), w[np.unravel_index(err.argmax(), err.shape)[0]])


# ------------------------------------------------------- exactness / tiling
@pytest.mark.parametrize("plan", REGEN_PLANS + PANEL_PLANS + TILE_PLANS)
def test_pm1_integer_bit_exact_every_plan(plan):
    # d = 300 and n = 37 leave ragged tails in every tile shape
    A = inputs.integer_uniform(6000, 37, 0.02, seed=3)
    ref = oracle_sketch(A, 300, "pm1")
    got = gpu_sketch(A, 300, "pm1", plan=plan)
    assert np.array_equal(got, ref)


@pytest.mark.parametrize("dist", ["uniform", "normal"])
@pytest.mark.parametrize("plan", [REGEN_PLANS[0], REGEN_PLANS[-1],
                                  REGEN_PLANS[9]] + PANEL_PLANS + TILE_PLANS)
def test_float_within_tolerance_every_plan(dist, plan):
    A = inputs.float_uniform(6000, 37, 0.02, seed=4)
    ref = oracle_sketch(A, 301, dist)
    got = gpu_sketch(A, 301, dist, plan=plan)
    assert rel_fro(got, ref) <= TOL


@pytest.mark.parametrize("dist", ["pm1", "uniform", "normal"])
def test_tile_tensor_memory_sums_equal_register_sums(dist):
    """TILE keeps a CTA's running sums in registers (16 warps x 64 columns,
    one CTA per row tile and row range) or in tensor memory (32 warps x 32
    columns: one wave of C CTAs per column block, each taking the same share
    of every row range's (tile, panel) blocks).  Per tile both add within a
    range, then the ranges in order, so where each CTA owns whole tiles
    (d = 32 C or 64 C) the bits are the register path's, for 1, 2 or 3 ranges
    of 23 panels.  With d = 100 every tile is shared by many CTAs, whose
    pieces are added in CTA order: within the tolerance.  n = 1100 spreads
    columns over every warp (all four tensor-memory lane quarters) and two
    column blocks, the last one ragged."""
    A = inputs.float_uniform(3000, 1100, 0.01, seed=21)
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    C = max(1, sms // 2)  # CTAs per column block: two column blocks
    for d in (32 * C, 64 * C, 100):
        ref = oracle_sketch(A, d, dist) if d == 100 or dist == "normal" else None
        for g in (1, 2, 3):
            base = gpu_sketch(A, d, dist, plan=dict(
                mode=capi.SKETCH_MODE_TILE, panel_rows=136, row_groups=g, cols_per_warp=64,
                tile_acc=0))
            got = gpu_sketch(A, d, dist, plan=dict(
                mode=capi.SKETCH_MODE_TILE, panel_rows=136, row_groups=g, cols_per_warp=32,
                tile_acc=1))
            if d != 100:
                assert np.array_equal(got, base), (d, g)
            if ref is not None:
                assert rel_fro(got, ref) <= TOL, (d, g)
                assert rel_fro(base, ref) <= TOL, (d, g)


@pytest.mark.parametrize("dist", ["pm1", "uniform", "normal"])
@pytest.mark.parametrize("d,ld", [(100, 100), (98, 100), (61, 64), (300, 304)])
def test_pregenerated_S_gives_the_generated_bits(dist, d, ld):
    """Sec. 3.3's pre-generated S: S written to memory, then the TILE kernel
    reading it, equals the TILE kernel generating it bit for bit; the stored
    S matches the oracle's entries (ragged d, padded leading dimension)."""
    A = inputs.float_uniform(3000, 300, 0.02, seed=23)
    sk = capi.Sketch(A.m, A.n, d, dist, seed=5, stream_id=2)
    sk.set_plan(capi.SKETCH_MODE_TILE, panel_rows=512, row_groups=3, cols_per_warp=32,
                tile_acc=1)
    dA = capi.DeviceCSC(A)
    fly = sk.apply(dA).clone()
    S = sk.generate_S(ld_s=ld)
    mem = sk.apply_pregen(dA, S)
    torch.cuda.synchronize()
    assert sk.device_status() == capi.SKETCH_OK
    assert torch.equal(fly, mem)
    Sh = S.cpu().numpy()
    rng = np.random.default_rng(3)
    for i, j in list(zip(rng.integers(0, d, 300), rng.integers(0, A.m, 300))) + \
            [(0, 0), (d - 1, A.m - 1), (d - 1, 0)]:
        ref = oracle.S_entry(DISTS[dist], 5, 2, int(i), int(j))
        if dist == "normal":
            assert abs(Sh[j, i] - ref) <= 4e-7 * max(1.0, abs(ref))
        else:
            assert Sh[j, i] == ref
    sk.close()


def test_pregenerated_S_default_plan_and_tolerance():
    """Without a forced plan the S-from-memory path picks its own panels;
    result within the FP32 tolerance of the oracle, n > 1024 (two column
    blocks)."""
    A = inputs.float_uniform(2000, 1100, 0.01, seed=24)
    d = 64
    sk = capi.Sketch(A.m, A.n, d, "uniform", seed=1)
    S = sk.generate_S()
    got = sk.apply_pregen(capi.DeviceCSC(A), S)
    torch.cuda.synchronize()
    assert sk.device_status() == capi.SKETCH_OK
    ref = oracle_sketch(A, d, "uniform")
    assert rel_fro(got.cpu().numpy().astype(np.float64).T, ref) <= TOL
    sk.close()


def test_uniform_integer_values_exact_in_integer_scale():
    """U entries are odd multiples of 2^-24; with small integer A every
    partial sum of (2u+1) a is an integer below 2^24 only for tiny sums, so
    instead check the tolerance and the absence of any systematic bias."""
    A = inputs.integer_uniform(4000, 20, 0.01, seed=5)
    ref = oracle_sketch(A, 128, "uniform")
    got = gpu_sketch(A, 128, "uniform")
    assert rel_fro(got, ref) <= TOL


def test_streams_give_different_S_and_match_oracle():
    A = inputs.integer_uniform(3000, 10, 0.02, seed=6)
    g0 = gpu_sketch(A, 200, "pm1", stream_id=0)
    g7 = gpu_sketch(A, 200, "pm1", stream_id=7)
    assert not np.array_equal(g0, g7)
    assert np.array_equal(g7, oracle_sketch(A, 200, "pm1", stream_id=7))


def test_bf16_values():
    A, b, _ = inputs.lsq_mixed(m=20000, n=30, density=0.01)
    ref = oracle_sketch(A, 60, "pm1")
    for plan in (REGEN_PLANS[5], PANEL_PLANS[0], TILE_PLANS[1]):
        got = gpu_sketch(A, 60, "pm1", plan=plan)
        assert rel_fro(got, ref) <= TOL


def test_config_plain_small_bit_exact():
    """m=50,000, n=200, d=400, density 1%, integer values, +-1 S, seed 1."""
    A = inputs.plain_small()
    ref = oracle_sketch(A, inputs.PLAIN_SMALL_D, "pm1")
    got = gpu_sketch(A, inputs.PLAIN_SMALL_D, "pm1")  # tuned plan
    assert np.array_equal(got, ref)


# --------------------------------------------------------------- edge cases
def test_empty_matrix_gives_zero():
    A = inputs.CSC(100, 7, np.zeros(8, np.int32), np.zeros(0, np.int32),
                   np.zeros(0, np.float32))
    got = gpu_sketch(A, 33, "uniform")
    assert np.all(got == 0)


def test_empty_columns_and_tiny_shapes():
    colptr = np.array([0, 0, 2, 2, 3], np.int32)
    rowidx = np.array([1, 4, 0], np.int32)
    vals = np.array([2.0, -1.0, 3.0], np.float32)
    A = inputs.CSC(5, 4, colptr, rowidx, vals)
    for d in (1, 3, 4, 5, 129):
        for dist in ("pm1", "uniform"):
            ref = oracle_sketch(A, d, dist)
            for plan in (None, REGEN_PLANS[0], PANEL_PLANS[2], TILE_PLANS[3]):
                got = gpu_sketch(A, d, dist, plan=plan)
                if dist == "pm1":
                    assert np.array_equal(got, ref), (d, plan)
                else:
                    assert rel_fro(got, ref) <= TOL


def test_long_column_accuracy():
    """One column with 200k nonzeros: FP32 accumulation must stay within the
    1e-6 gate (two-level sums in REGEN, row groups in PANEL and TILE)."""
    m = 400_000
    rng = np.random.default_rng(7)
    rows = np.sort(rng.choice(m, size=200_000, replace=False)).astype(np.int32)
    A = inputs.CSC(m, 1, np.array([0, rows.size], np.int32), rows,
                   rng.uniform(-1, 1, size=rows.size).astype(np.float32))
    ref = oracle_sketch(A, 256, "uniform")
    for plan in (REGEN_PLANS[4 * 1 + 0], REGEN_PLANS[4 * 1 + 3], None,
                 dict(mode=capi.SKETCH_MODE_TILE, panel_rows=1024,
                      row_groups=400, cols_per_warp=4),
                 # tensor-memory sums: 2942 panels in 400 and 100 ranges, the
                 # 8 row tiles shared by the CTAs of one wave
                 dict(mode=capi.SKETCH_MODE_TILE, panel_rows=136, row_groups=400,
                      cols_per_warp=32, tile_acc=1),
                 dict(mode=capi.SKETCH_MODE_TILE, panel_rows=136, row_groups=100,
                      cols_per_warp=32, tile_acc=1)):
        got = gpu_sketch(A, 256, "uniform", plan=plan)
        assert rel_fro(got, ref) <= TOL, plan


def test_generation_counts():
    """Sec. 3.2: Alg. 3 generates d * nnz entries; Alg. 4 generates d per
    nonempty row per column block."""
    A = inputs.integer_uniform(5000, 40, 0.005, seed=8)
    d = 200
    for plan, expect in (
            (REGEN_PLANS[6], d * A.nnz),
            (dict(mode=capi.SKETCH_MODE_PANEL, n_block=40, row_groups=3),
             d * np.unique(A.rowidx).size),
            (dict(mode=capi.SKETCH_MODE_TILE, panel_rows=1000, row_groups=2,
                  cols_per_warp=4), d * A.m),
            (dict(mode=capi.SKETCH_MODE_TILE, panel_rows=1000, row_groups=5,
                  cols_per_warp=32, tile_acc=1), d * A.m)):
        sk = capi.Sketch(A.m, A.n, d, "uniform", seed=1)
        sk.set_plan(**plan)
        sk.set_counting(True)
        sk.apply(capi.DeviceCSC(A))
        assert sk.generated_entries() == expect
        sk.close()


def test_bad_row_index_is_reported_not_faulted():
    A = inputs.integer_uniform(1000, 5, 0.02, seed=9)
    A.rowidx = A.rowidx.copy()
    A.rowidx[3] = 1000 + 17      # out of range
    dA = capi.DeviceCSC(A)
    assert capi.validate_csc(dA) == capi.SKETCH_ERR_CSC
    for plan in (REGEN_PLANS[0], PANEL_PLANS[0], TILE_PLANS[0]):
        sk = capi.Sketch(A.m, A.n, 64, "pm1", seed=1)
        sk.set_plan(**plan)
        sk.apply(dA)
        torch.cuda.synchronize()
        assert sk.device_status() == capi.SKETCH_ERR_CSC
        sk.close()


def _decreasing_colptr(A, k):
    """colptr[k + 1] set one below colptr[k]: column k's range decreases and
    column k + 1's range reaches one entry back into column k - 1.  Every
    index stays inside [0, nnz], so even a kernel without the clamps would
    address only A's own arrays."""
    B = inputs.CSC(A.m, A.n, A.colptr.copy(), A.rowidx, A.values)
    assert B.colptr[k] > 0 and B.colptr[k + 2] > B.colptr[k]
    B.colptr[k + 1] = B.colptr[k] - 1
    return B


def test_decreasing_colptr_is_reported_by_every_plan():
    """A malformed colptr is clamped column by column inside the kernels and
    reported as SKETCH_ERR_CSC through the device status word."""
    A = _decreasing_colptr(inputs.integer_uniform(3000, 12, 0.02, seed=12), 4)
    dA = capi.DeviceCSC(A)
    assert capi.validate_csc(dA) == capi.SKETCH_ERR_CSC
    for plan in (REGEN_PLANS[0], PANEL_PLANS[0], TILE_PLANS[0], TILE_PLANS[4],
                 dict(mode=capi.SKETCH_MODE_REGEN, q_tiles=1, split=1, tc_min_row_nnz=2)):
        sk = capi.Sketch(A.m, A.n, 64, "pm1", seed=1)
        sk.set_plan(**plan)
        sk.apply(dA)
        torch.cuda.synchronize()
        assert sk.device_status() == capi.SKETCH_ERR_CSC, plan
        assert sk.device_status() == capi.SKETCH_OK  # reading clears it
        sk.close()


def test_validator_accepts_good_and_rejects_unsorted():
    A = inputs.integer_uniform(1000, 5, 0.02, seed=10)
    assert capi.validate_csc(capi.DeviceCSC(A)) == capi.SKETCH_OK
    B = inputs.integer_uniform(1000, 5, 0.02, seed=10)
    B.rowidx = B.rowidx.copy()
    B.rowidx[[0, 1]] = B.rowidx[[1, 0]]
    assert capi.validate_csc(capi.DeviceCSC(B)) == capi.SKETCH_ERR_CSC


def test_shape_mismatch_is_an_argument_error():
    A = inputs.integer_uniform(1000, 5, 0.02, seed=10)
    sk = capi.Sketch(999, 5, 10, "pm1")
    with pytest.raises(capi.SketchError) as e:
        sk.apply(capi.DeviceCSC(A))
    assert e.value.code == capi.SKETCH_ERR_ARG


# ------------------------------------------------- full-size skewed workload
@pytest.fixture(scope="module")
def skew_large():
    return inputs.skew_large()


SKEW_TACC = dict(mode=capi.SKETCH_MODE_TILE, panel_rows=1024, row_groups=20,
                 cols_per_warp=32, tile_acc=1)


@pytest.mark.parametrize("dist,plan", [("pm1", None), ("uniform", None), ("normal", None),
                                       ("normal", SKEW_TACC)])
def test_skew_large_sampled_columns(skew_large, dist, plan):
    """m=2e6, n=1000, d=3000, ~1e7 nnz, power-law rows: the tuned launch the
    benchmark times (and TILE with tensor-memory sums), checked on sampled
    columns (columns of A_hat depend only on the matching column of A, so the
    oracle computes them alone)."""
    A = skew_large
    d = inputs.SKEW_LARGE_D
    sk = capi.Sketch(A.m, A.n, d, dist, seed=1)
    if plan:
        sk.set_plan(**plan)
    dA = capi.DeviceCSC(A)
    out = sk.apply(dA)
    torch.cuda.synchronize()
    assert sk.device_status() == capi.SKETCH_OK
    got = out.cpu().numpy().astype(np.float64)  # n x d
    sk.close()
    # 60 columns: the three heaviest, the ends and middle, and random ones
    lens = np.diff(A.colptr)
    cols = set(np.argsort(lens)[-3:].tolist()) | {0, 1, 499, 998, 999}
    rng = np.random.default_rng(13)
    while len(cols) < 60:
        cols.add(int(rng.integers(0, A.n)))
    cols = sorted(cols)
    ref = oracle_sketch(A.columns(cols), d, dist).T  # len(cols) x d
    for t, k in enumerate(cols):
        assert rel_fro(got[k], ref[t]) <= TOL, (dist, k)
    assert rel_fro(got[cols], ref) <= TOL


# ------------------------------------------------ tensor-core dense panels
def _dense_rows_matrix(m, n, every, dens, integer, seed):
    """Every `every`-th row dense (the paper's Abnormal_A pattern) on top of a
    uniformly sparse background."""
    rng = np.random.default_rng(seed)
    bg = inputs.integer_uniform(m, n, dens, seed=seed) if integer else \
        inputs.float_uniform(m, n, dens, seed=seed)
    S = bg.to_scipy().tolil()
    for j in range(0, m, every):
        vals = rng.integers(1, 4, size=n) * rng.choice([-1, 1], size=n) if integer \
            else rng.uniform(-1, 1, size=n)
        S[j, :] = vals
    C = S.tocsc()
    C.sort_indices()
    return inputs.CSC(m, n, C.indptr.astype(np.int32), C.indices.astype(np.int32),
                      C.data.astype(np.float32))


TC_PLANS = [dict(mode=capi.SKETCH_MODE_REGEN, q_tiles=2, split=2, tc_min_row_nnz=64),
            dict(mode=capi.SKETCH_MODE_TILE, panel_rows=512, row_groups=4,
                 cols_per_warp=16, tc_min_row_nnz=40)]


@pytest.mark.parametrize("plan", TC_PLANS)
def test_tensor_core_panel_integer_bit_exact(plan):
    A = _dense_rows_matrix(9000, 300, 97, 0.003, True, seed=31)   # 93 dense rows
    for d in (300, 257):
        ref = oracle_sketch(A, d, "pm1")
        got = gpu_sketch(A, d, "pm1", plan=plan)
        assert np.array_equal(got, ref), d


@pytest.mark.parametrize("plan", TC_PLANS)
@pytest.mark.parametrize("every", [50, 97])
def test_tensor_core_panel_float_tolerance(plan, every):
    """U(-1,1) values: 180 dense rows (two groups of steps, promoted sums) and
    93 (one group: 128 x 256 units, the whole unit in one accumulator)."""
    A = _dense_rows_matrix(9000, 300, every, 0.003, False, seed=32)
    ref = oracle_sketch(A, 301, "pm1")
    got = gpu_sketch(A, 301, "pm1", plan=plan)
    assert rel_fro(got, ref) <= TOL


@pytest.mark.parametrize("plan", TC_PLANS)
def test_tensor_core_panel_only_dense_rows(plan):
    """Every nonzero in the panel (the Abnormal_A pattern): the sparse pass
    has nothing left and the panel's product is stored into A_hat directly;
    integer values keep it bit-exact, at ragged d and n."""
    rng = np.random.default_rng(34)
    m, n = 5000, 301
    rows = np.arange(0, m, 97)
    keys = np.sort((np.arange(n)[:, None] * m + rows[None, :]).ravel())
    colptr = np.searchsorted(keys // m, np.arange(n + 1)).astype(np.int32)
    rowidx = (keys % m).astype(np.int32)
    vals = (rng.integers(1, 4, size=keys.size) * rng.choice([-1, 1], size=keys.size))
    A = inputs.CSC(m, n, colptr, rowidx, vals.astype(np.float32))
    for d in (256, 259):
        ref = oracle_sketch(A, d, "pm1")
        got = gpu_sketch(A, d, "pm1", plan=plan)
        assert np.array_equal(got, ref), d


@pytest.mark.parametrize("d", [256, 300, 611])
def test_tensor_core_long_panel_integer_bit_exact(d):
    """A long panel streams its B operand through the stage ring and is split
    along K: 760 dense rows, ragged d and n = 301 (the last column tile is
    mostly past n), integer values: bit-exact."""
    A = _dense_rows_matrix(30_400, 301, 40, 0.002, True, seed=37)
    plan = dict(mode=capi.SKETCH_MODE_REGEN, q_tiles=2, split=2, tc_min_row_nnz=100)
    got = gpu_sketch(A, d, "pm1", plan=plan)
    assert np.array_equal(got, oracle_sketch(A, d, "pm1"))


def test_tensor_core_resident_panel_many_units_per_cta():
    """A short panel (100 dense rows) over 24 x 24 tiles of 128 x 128: each
    CTA keeps a column tile's B operand in shared memory and walks a run of
    about four units, reloading B where its run crosses into the next
    column tile; ragged d, integer values: bit-exact on sampled columns
    (both ends of each crossing included)."""
    A = _dense_rows_matrix(20_000, 3000, 200, 0.001, True, seed=36)
    d = 3001
    plan = dict(mode=capi.SKETCH_MODE_REGEN, q_tiles=4, split=1, tc_min_row_nnz=1000)
    got = gpu_sketch(A, d, "pm1", plan=plan)
    rng = np.random.default_rng(36)
    cols = sorted({0, 127, 128, 255, 256, 1535, 1536, 2943, 2944, 2999} |
                  set(rng.choice(A.n, size=30, replace=False).tolist()))
    ref = oracle_sketch(A.columns(cols), d, "pm1")
    assert np.array_equal(got[:, cols], ref)


PREPARED_PLANS = [dict(mode=capi.SKETCH_MODE_REGEN, q_tiles=2, split=2, tc_min_row_nnz=40),
                  dict(mode=capi.SKETCH_MODE_TILE, panel_rows=512, row_groups=4,
                       cols_per_warp=32, tile_acc=1),
                  dict(mode=capi.SKETCH_MODE_TILE, panel_rows=512, row_groups=4,
                       cols_per_warp=16, tc_min_row_nnz=100)]


@pytest.mark.parametrize("plan", PREPARED_PLANS)
def test_prepared_data_reused_and_rebuilt_when_A_changes(plan):
    """Plans that derive data from A (a tensor-core panel, TILE's panel-major
    copy) reuse it on the next call with the same A: fewer launches, the same
    bits.  Rewriting A's values or rows in place (same addresses) changes its
    content hash, so the data is rebuilt and the sketch matches the oracle
    for the new A."""
    A = _dense_rows_matrix(30_400, 300, 40, 0.002, True, seed=35)
    d = 300
    sk = capi.Sketch(A.m, A.n, d, "pm1", seed=1)
    sk.set_plan(**plan)
    dA = capi.DeviceCSC(A)
    out = torch.empty((A.n, d), dtype=torch.float32, device="cuda")
    sk.apply(dA, out)
    torch.cuda.synchronize()
    first = out.clone()
    n0 = sk.launch_count()
    sk.apply(dA, out)
    torch.cuda.synchronize()
    reused = sk.launch_count() - n0
    assert torch.equal(out, first)
    assert np.array_equal(first.cpu().numpy().astype(np.float64).T, oracle_sketch(A, d, "pm1"))
    # new values at the same addresses
    rng = np.random.default_rng(36)
    B = inputs.CSC(A.m, A.n, A.colptr, A.rowidx,
                   (rng.integers(1, 4, size=A.nnz) * rng.choice([-1, 1], size=A.nnz))
                   .astype(np.float32))
    dA.values.copy_(torch.from_numpy(B.values))
    n1 = sk.launch_count()
    sk.apply(dA, out)
    torch.cuda.synchronize()
    rebuilt = sk.launch_count() - n1
    assert rebuilt > reused
    assert np.array_equal(out.cpu().numpy().astype(np.float64).T, oracle_sketch(B, d, "pm1"))
    # the last row of a column moved down by one (the column stays sorted and
    # distinct): the pattern changes
    rows = A.rowidx.copy()
    lasts = A.colptr[1:][np.diff(A.colptr) > 0] - 1
    lasts = lasts[rows[lasts] < A.m - 1]
    rows[lasts[0]] += 1
    C = inputs.CSC(A.m, A.n, A.colptr, rows, B.values)
    dA.rowidx.copy_(torch.from_numpy(C.rowidx))
    sk.apply(dA, out)
    torch.cuda.synchronize()
    assert sk.device_status() == capi.SKETCH_OK
    assert np.array_equal(out.cpu().numpy().astype(np.float64).T, oracle_sketch(C, d, "pm1"))
    sk.close()


@pytest.mark.parametrize("every,fp8", [(97, 0), (40, 0), (20, 0), (97, 1), (20, 1)])
def test_tensor_core_repeated_applies_identical(every, fp8):
    """The panel kernel's two MMA threads, S builders and bulk copies meet
    only through their stage rings; repeated applies of one plan give the
    same bits every time and a clean status word (short panels: 128 x 256
    units; 760 and 1520 dense rows: 128 x 128 units, split along K)."""
    A = _dense_rows_matrix(30_400 if every != 97 else 9000, 700, every, 0.002, False,
                           seed=41)
    d = 1000
    sk = capi.Sketch(A.m, A.n, d, "pm1", seed=2)
    sk.set_plan(mode=capi.SKETCH_MODE_REGEN, q_tiles=4, split=2, tc_min_row_nnz=300,
                tc_fp8=fp8)
    dA = capi.DeviceCSC(A)
    out = torch.empty((A.n, d), dtype=torch.float32, device="cuda")
    sk.apply(dA, out)
    torch.cuda.synchronize()
    first = out.clone()
    for _ in range(12):
        out.fill_(float("nan"))
        sk.apply(dA, out)
        torch.cuda.synchronize()
        assert torch.equal(out, first)
    assert sk.device_status() == capi.SKETCH_OK
    sk.close()


def test_tensor_core_long_panel_float_tolerance():
    A = _dense_rows_matrix(30_400, 300, 40, 0.002, False, seed=38)
    plan = dict(mode=capi.SKETCH_MODE_TILE, panel_rows=512, row_groups=4,
                cols_per_warp=16, tc_min_row_nnz=100)
    got = gpu_sketch(A, 513, "pm1", plan=plan)
    assert rel_fro(got, oracle_sketch(A, 513, "pm1")) <= TOL


FP8_PLANS = [dict(mode=capi.SKETCH_MODE_REGEN, q_tiles=2, split=2, tc_min_row_nnz=40, tc_fp8=1),
             dict(mode=capi.SKETCH_MODE_TILE, panel_rows=512, row_groups=4, cols_per_warp=16,
                  tc_min_row_nnz=100, tc_fp8=1)]


@pytest.mark.parametrize("plan", FP8_PLANS)
@pytest.mark.parametrize("every", [97, 40, 20])
def test_fp8_panel_integer_bit_exact(plan, every):
    """FP8 panels: +-1 is exact in E4M3 and integers up to 3 in magnitude
    survive the per-column power-of-two scale and the two-term split, so the
    sketch stays bit-exact (93 and 760 dense rows: B resident in shared
    memory; 1520: streamed and split along K)."""
    A = _dense_rows_matrix(9000 if every == 97 else 30_400, 300, every, 0.002, True, seed=39)
    for d in (256, 301):
        got = gpu_sketch(A, d, "pm1", plan=plan)
        assert np.array_equal(got, oracle_sketch(A, d, "pm1")), d


@pytest.mark.parametrize("plan", FP8_PLANS)
def test_fp8_panel_float_within_2e_2(plan):
    """U(-1,1) values: each value is carried by two E4M3 terms (about 2^-8
    relative), so the sketch meets the FP8 gate of 2e-2 against FP64."""
    A = _dense_rows_matrix(30_400, 300, 40, 0.002, False, seed=40)
    ref = oracle_sketch(A, 513, "pm1")
    err = rel_fro(gpu_sketch(A, 513, "pm1", plan=plan), ref)
    assert err <= 2e-2, err


def test_fp8_panel_needs_a_panel():
    sk = capi.Sketch(1000, 10, 64, "pm1")
    with pytest.raises(capi.SketchError) as e:
        sk.set_plan(mode=capi.SKETCH_MODE_REGEN, q_tiles=1, split=1, tc_fp8=1)
    assert e.value.code == capi.SKETCH_ERR_ARG


def test_tuned_plan_on_dense_rows_is_exact():
    """With tuning on, +-1 S on a matrix with dense rows: whichever plan the
    tuner takes (tensor-core panels are candidates), the sketch is the
    oracle's, bit for bit (integer values)."""
    A = _dense_rows_matrix(9000, 300, 97, 0.003, True, seed=35)
    sk = capi.Sketch(A.m, A.n, 300, "pm1", seed=1)
    sk.set_autotune(True)
    dA = capi.DeviceCSC(A)
    out = sk.apply(dA)
    plan = sk.get_plan(dA)
    got = out.cpu().numpy().T
    sk.close()
    assert plan["mode"] in (capi.SKETCH_MODE_REGEN, capi.SKETCH_MODE_TILE)
    assert np.array_equal(got, oracle_sketch(A, 300, "pm1"))


def test_abnormal_a_full_size_tensor_core_plan_sampled_columns():
    """The benchmark's Abnormal_A case at full size (m = 100,000, n = 10,000,
    every 1000th row dense, d = 30,000): the tensor-core panel plan and the
    tuned plan, 64 sampled columns (including both ends of the column range
    and the CTA tile edges) against the oracle within 1e-6."""
    A = inputs.abnormal("a")
    d = 3 * A.n
    dA = capi.DeviceCSC(A)
    rng = np.random.default_rng(14)
    cols = sorted({0, 1, 127, 128, 255, 256, A.n - 2, A.n - 1} |
                  set(rng.choice(A.n, size=56, replace=False).tolist()))
    ref = oracle_sketch(A.columns(cols), d, "pm1").T
    for plan in (dict(mode=capi.SKETCH_MODE_REGEN, q_tiles=4, split=8,
                      tc_min_row_nnz=A.n // 2), None):
        sk = capi.Sketch(A.m, A.n, d, "pm1", seed=1)
        if plan:
            sk.set_plan(**plan)
        out = sk.apply(dA)
        torch.cuda.synchronize()
        assert sk.device_status() == capi.SKETCH_OK
        if plan is None:
            assert sk.get_plan(dA)["tc_min_row_nnz"] > 0  # the tuner takes a panel
        got = out[cols].cpu().numpy().astype(np.float64)
        sk.close()
        for t, k in enumerate(cols):
            assert rel_fro(got[t], ref[t]) <= TOL, (plan, k)
        del out


def test_bounded_wait_times_out_into_status_and_context_survives():
    """A kernel waits on an mbarrier phase that nothing completes: the wait
    gives up after its iteration limit, the host reads SKETCH_ERR_TIMEOUT
    from the status word (once: reading clears it), and the context still
    sketches correctly afterwards."""
    A = inputs.integer_uniform(3000, 20, 0.01, seed=36)
    sk = capi.Sketch(A.m, A.n, 128, "pm1", seed=1)
    capi.debug_wait_timeout(sk)
    torch.cuda.synchronize()
    assert sk.device_status() == capi.SKETCH_ERR_TIMEOUT
    assert sk.device_status() == capi.SKETCH_OK
    got = sk.apply(capi.DeviceCSC(A)).cpu().numpy().T
    sk.close()
    assert np.array_equal(got, oracle_sketch(A, 128, "pm1"))


def test_tensor_core_panel_without_dense_rows_and_bad_dist():
    A = inputs.integer_uniform(4000, 50, 0.01, seed=33)
    got = gpu_sketch(A, 200, "pm1", plan=TC_PLANS[0])
    assert np.array_equal(got, oracle_sketch(A, 200, "pm1"))
    sk = capi.Sketch(A.m, A.n, 64, "uniform")
    with pytest.raises(capi.SketchError) as e:
        sk.set_plan(**TC_PLANS[0])
    assert e.value.code == capi.SKETCH_ERR_UNSUPPORTED
