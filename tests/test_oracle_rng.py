"""Pins for the oracle's generator and distribution transforms (CPU only).

Philox4x32-10 (Sec. 4.2 names the counter-based family) is pinned to an
independent implementation run as a black box: PyTorch's header-only
``at::philox_engine``.  The transforms of Sec. 3.3 are pinned by closed forms,
exact special cases and distribution tests.
"""
import os
import shutil
import subprocess
import sysconfig

import numpy as np
import pytest

import oracle

HERE = os.path.dirname(os.path.abspath(__file__))


def _torch_include():
    try:
        import torch  # noqa: F401
    except Exception:
        return None
    import torch.utils.cpp_extension as ce
    for p in ce.include_paths():
        if os.path.exists(os.path.join(p, "ATen", "core", "PhiloxRNGEngine.h")):
            return p
    return None


@pytest.fixture(scope="module")
def torch_philox(tmp_path_factory):
    inc = _torch_include()
    gxx = shutil.which("g++")
    if inc is None or gxx is None:
        pytest.skip("torch headers or g++ unavailable")
    exe = str(tmp_path_factory.mktemp("philox") / "philox_ref")
    subprocess.run([gxx, "-O1", "-std=c++17", "-I", inc,
                    os.path.join(HERE, "philox_torch_ref.cpp"), "-o", exe],
                   check=True)

    def run(triples):
        inp = "\n".join("%d %d %d" % t for t in triples) + "\n"
        out = subprocess.run([exe], input=inp, capture_output=True, text=True,
                             check=True).stdout.split()
        return np.array([int(v) for v in out], dtype=np.uint64).reshape(-1, 4)
    return run


def test_philox_matches_torch_engine(torch_philox):
    rng = np.random.default_rng(123)
    ctrs = rng.integers(0, 2**32, size=(10_000, 4), dtype=np.uint64)
    keys = rng.integers(0, 2**32, size=(10_000, 2), dtype=np.uint64)
    # edge counters/keys: all zero and all ones
    ctrs[0] = 0
    keys[0] = 0
    ctrs[1] = 2**32 - 1
    keys[1] = 2**32 - 1
    triples = []
    for c, k in zip(ctrs, keys):
        key64 = int(k[0]) | (int(k[1]) << 32)
        sub = int(c[2]) | (int(c[3]) << 32)
        off = int(c[0]) | (int(c[1]) << 32)
        triples.append((key64, sub, off))
    ref = torch_philox(triples)
    for t in range(len(triples)):
        got = oracle.philox4x32_10(ctrs[t].astype(np.uint32), keys[t].astype(np.uint32))
        assert np.array_equal(got.astype(np.uint64), ref[t]), t


def test_counter_layout_and_pm1_bits_match_torch_engine(torch_philox):
    """S(i, j) for +-1 is bit (i & 127) of block (i >> 7, j, stream, 0)."""
    seed, stream = 0x0123456789ABCDEF, 7
    cases = [(i, j) for i in (0, 1, 31, 32, 127, 128, 1000, 2999)
             for j in (0, 5, 2**20, 2**31 - 1)]
    triples = [(seed, stream, (j << 32) | (i >> 7)) for i, j in cases]
    ref = torch_philox(triples)
    for (i, j), words in zip(cases, ref):
        b = i & 127
        bit = (int(words[b >> 5]) >> (b & 31)) & 1
        assert oracle.S_entry(oracle.PM1, seed, stream, i, j) == (-1.0 if bit else 1.0)


def test_uniform_and_normal_use_block_i_over_4(torch_philox):
    seed, stream = 42, 3
    cases = [(i, j) for i in (0, 1, 2, 3, 4, 401, 2998) for j in (0, 9, 777777)]
    ref = torch_philox([(seed, stream, (j << 32) | (i >> 2)) for i, j in cases])
    for (i, j), w in zip(cases, ref):
        q = i & 3
        assert oracle.S_entry(oracle.UNIFORM, seed, stream, i, j) == \
            oracle.uniform_from_word(int(w[q]))
        p = q >> 1
        assert oracle.S_entry(oracle.NORMAL, seed, stream, i, j) == \
            oracle.normal_from_words(int(w[2 * p]), int(w[2 * p + 1]), q & 1)


def test_uniform_closed_forms():
    e = 2.0 ** -24
    # u = top 24 bits as a signed integer; S = (2u+1) 2^-24
    assert oracle.uniform_from_word(0x00000000) == e
    assert oracle.uniform_from_word(0x000000FF) == e          # low byte ignored
    assert oracle.uniform_from_word(0x00000100) == 3 * e
    assert oracle.uniform_from_word(0xFFFFFFFF) == -e
    assert oracle.uniform_from_word(0x7FFFFF00) == 1.0 - e    # largest
    assert oracle.uniform_from_word(0x80000000) == -1.0 + e   # smallest
    # symmetric: w and ~w map to negatives of each other
    rng = np.random.default_rng(5)
    for w in rng.integers(0, 2**32, size=2000, dtype=np.uint64):
        w = int(w)
        a = oracle.uniform_from_word(w)
        b = oracle.uniform_from_word((~w) & 0xFFFFFFFF)
        assert a == -b and -1.0 < a < 1.0
        # exactly representable in FP32
        assert float(np.float32(a)) == a


def test_normal_closed_forms():
    # u1 = 1 (top 24 bits all ones) -> r = 0 -> both branches exactly 0
    assert oracle.normal_from_words(0xFFFFFF00, 0x12345678, 0) == 0.0
    assert oracle.normal_from_words(0xFFFFFFFF, 0x12345678, 1) == 0.0
    # angle word 0 -> theta = 0: cos branch = r, sin branch = 0
    r = np.sqrt(-2.0 * np.log(2.0 ** -24))                  # u1 = 2^-24 (w = 0)
    assert abs(oracle.normal_from_words(0, 0, 0) - r) < 1e-15 * r
    assert oracle.normal_from_words(0, 0, 1) == 0.0
    # theta = pi/2 (u2 = 1/4): cos ~ 0, sin = r
    assert abs(oracle.normal_from_words(0, 0x40000000, 1) - r) < 1e-14
    assert abs(oracle.normal_from_words(0, 0x40000000, 0)) < 1e-14
    # pair identity z_even^2 + z_odd^2 = -2 ln u1
    rng = np.random.default_rng(6)
    for w0, w1 in rng.integers(0, 2**32, size=(500, 2), dtype=np.uint64):
        z0 = oracle.normal_from_words(int(w0), int(w1), 0)
        z1 = oracle.normal_from_words(int(w0), int(w1), 1)
        u1 = ((int(w0) >> 8) + 1) * 2.0 ** -24
        assert abs(z0 * z0 + z1 * z1 + 2.0 * np.log(u1)) < 1e-12 * max(1.0, -2 * np.log(u1))


@pytest.mark.parametrize("dist", [oracle.PM1, oracle.UNIFORM, oracle.NORMAL])
def test_column_equals_entries(dist):
    """S does not depend on how it is generated (tiling independence)."""
    seed, stream, d = 99, 1, 301
    for j in (0, 1, 12345, 2**31 - 1):
        col = oracle.S_column(dist, seed, stream, d, j)
        ent = np.array([oracle.S_entry(dist, seed, stream, i, j) for i in range(d)])
        assert np.array_equal(col, ent)
    dense = oracle.S_dense(dist, seed, stream, 77, 13)
    for j in range(13):
        assert np.array_equal(dense[:, j], oracle.S_column(dist, seed, stream, 77, j))


def test_streams_and_seeds_differ():
    a = oracle.S_column(oracle.UNIFORM, 1, 0, 64, 5)
    b = oracle.S_column(oracle.UNIFORM, 1, 1, 64, 5)
    c = oracle.S_column(oracle.UNIFORM, 2, 0, 64, 5)
    assert not np.array_equal(a, b) and not np.array_equal(a, c)


@pytest.mark.parametrize("dist,var", [(oracle.PM1, 1.0),
                                      (oracle.UNIFORM, (1 - 2.0**-48) / 3.0),
                                      (oracle.NORMAL, 1.0)])
def test_moments_StS_over_d(dist, var):
    """E[S^T S]/d = var * I (iid entries, mean 0).  m=64 columns, d=2^16."""
    d, m = 1 << 16, 64
    S = oracle.S_dense(dist, 2024, 0, d, m)
    G = S.T @ S / d
    diag = np.diag(G)
    off = G - np.diag(diag)
    if dist == oracle.PM1:
        assert np.all(diag == 1.0)
    else:
        # sd of the diagonal estimate: sqrt(Var(s^2)/d); Var(s^2) = 4/45 (U), 2 (N)
        v2 = 4.0 / 45.0 if dist == oracle.UNIFORM else 2.0
        assert np.all(np.abs(diag - var) < 6 * np.sqrt(v2 / d))
    assert np.max(np.abs(off)) < 6.0 * var / np.sqrt(d)
    assert abs(S.mean()) < 6.0 * np.sqrt(var / S.size)


def test_distribution_shapes_ks():
    from scipy import stats
    d, m = 4096, 16
    U = oracle.S_dense(oracle.UNIFORM, 7, 0, d, m).ravel()
    N = oracle.S_dense(oracle.NORMAL, 7, 0, d, m).ravel()
    P = oracle.S_dense(oracle.PM1, 7, 0, d, m).ravel()
    assert stats.kstest(U, stats.uniform(loc=-1, scale=2).cdf).pvalue > 1e-4
    assert stats.kstest(N, stats.norm.cdf).pvalue > 1e-4
    assert set(np.unique(P)) == {-1.0, 1.0}
    assert abs((P == 1).mean() - 0.5) < 6 * 0.5 / np.sqrt(P.size)
