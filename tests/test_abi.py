"""The C ABI library builds, loads without a GPU, and exports every function
that include/*.h declares (no compute calls here)."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        src = re.sub(r"//[^\n]*", "", src)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(\w+)\s*\(",
                             src, flags=re.M):
            name = m.group(1)
            if name not in ("if", "while", "for", "return", "sizeof"):
                names.add(name)
    return names


def test_header_declares_entry_points():
    names = _declared()
    for n in ("sketch_create", "sketch_apply", "sketch_destroy",
              "sketch_lsq_solve", "sketch_last_error"):
        assert n in names


def test_library_exports_every_declared_symbol():
    from paper_2310_15419_gb300 import capi
    lib = ctypes.CDLL(capi.load().__dict__["_name"])
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    from paper_2310_15419_gb300 import capi
    bound = {n for n, _, _ in capi.SIGNATURES}
    assert _declared() <= bound, _declared() - bound


def test_host_side_argument_errors_need_no_gpu():
    from paper_2310_15419_gb300 import capi
    lib = capi.load()
    h = ctypes.c_void_p()
    assert lib.sketch_create(0, 5, 5, 0, 1, ctypes.byref(h)) == capi.SKETCH_ERR_ARG
    assert lib.sketch_create(10, 5, 5, 7, 1, ctypes.byref(h)) == capi.SKETCH_ERR_ARG
    assert lib.sketch_create(10, 5, 5, 0, 1, None) == capi.SKETCH_ERR_ARG
    assert b"distribution" in lib.sketch_last_error(None) or True
    assert lib.sketch_create(10, 5, 5, 1, 1, ctypes.byref(h)) == capi.SKETCH_OK
    # wrong shape and null pointers are refused before any CUDA call
    A = capi.sketch_csc(11, 5, 0, 0, 0, 0, 0)
    assert lib.sketch_apply(h, ctypes.byref(A), ctypes.c_void_p(8), None) == capi.SKETCH_ERR_ARG
    A = capi.sketch_csc(10, 5, 2**31, 8, 8, 8, 0)
    assert lib.sketch_apply(h, ctypes.byref(A), ctypes.c_void_p(8), None) == capi.SKETCH_ERR_UNSUPPORTED
    A = capi.sketch_csc(10, 5, 3, 8, 8, 8, 5)
    assert lib.sketch_apply(h, ctypes.byref(A), ctypes.c_void_p(8), None) == capi.SKETCH_ERR_ARG
    assert lib.sketch_apply(h, ctypes.byref(A), None, None) == capi.SKETCH_ERR_ARG
    bad = capi.sketch_plan(1, 9, 1, 0, 0)
    assert lib.sketch_set_plan(h, ctypes.byref(bad)) == capi.SKETCH_ERR_ARG
    assert lib.sketch_destroy(h) == capi.SKETCH_OK


def test_tile_plan_checks_need_no_gpu():
    """TILE plans: register sums take 4, 16 or 64 columns per warp, tensor-
    memory sums (tile_acc = 1) exactly 32; both need panel_rows 8..1248."""
    from paper_2310_15419_gb300 import capi
    lib = capi.load()
    h = ctypes.c_void_p()
    assert lib.sketch_create(1000, 100, 64, 1, 1, ctypes.byref(h)) == capi.SKETCH_OK
    T = capi.SKETCH_MODE_TILE
    # mode, q_tiles, split, n_block, row_groups, panel_rows, cols_per_warp, tc, tile_acc
    good = [(T, 0, 0, 0, 1, 1024, 64, 0, 0), (T, 0, 0, 0, 3, 8, 4, 0, 0),
            (T, 0, 0, 0, 20, 1152, 32, 0, 1), (T, 0, 0, 0, 21, 1248, 32, 0, 1),
            (T, 0, 0, 0, 1, 8, 32, 0, 1)]
    bad = [(T, 0, 0, 0, 1, 1024, 64, 0, 1), (T, 0, 0, 0, 1, 512, 16, 0, 1),
           (T, 0, 0, 0, 1, 512, 32, 0, 0), (T, 0, 0, 0, 1, 512, 32, 0, 2),
           (T, 0, 0, 0, 1, 1249, 32, 0, 1), (T, 0, 0, 0, 1, 7, 64, 0, 0),
           (T, 0, 0, 0, 0, 1024, 64, 0, 0)]
    for f in good:
        assert lib.sketch_set_plan(h, ctypes.byref(capi.sketch_plan(*f))) == capi.SKETCH_OK, f
    for f in bad:
        assert lib.sketch_set_plan(h, ctypes.byref(capi.sketch_plan(*f))) == capi.SKETCH_ERR_ARG, f
    assert lib.sketch_destroy(h) == capi.SKETCH_OK


def test_pregenerated_S_argument_errors_need_no_gpu():
    from paper_2310_15419_gb300 import capi
    lib = capi.load()
    h = ctypes.c_void_p()
    assert lib.sketch_create(1000, 10, 30, 1, 1, ctypes.byref(h)) == capi.SKETCH_OK
    E = capi.SKETCH_ERR_ARG
    assert lib.sketch_generate_S(h, None, 32, None) == E           # null S
    assert lib.sketch_generate_S(h, ctypes.c_void_p(4096), 28, None) == E  # ld_s < d
    assert lib.sketch_generate_S(h, ctypes.c_void_p(4096), 34, None) == E  # not a multiple of 4
    assert lib.sketch_generate_S(h, ctypes.c_void_p(4104), 32, None) == E  # not 16-byte aligned
    A = capi.sketch_csc(1000, 10, 3, 8, 8, 8, 0)
    out = ctypes.c_void_p(8192)
    assert lib.sketch_apply_pregen(h, ctypes.byref(A), None, 32, out, None) == E
    assert lib.sketch_apply_pregen(h, ctypes.byref(A), ctypes.c_void_p(4096), 30, out,
                                   None) == E
    assert lib.sketch_apply_pregen(h, ctypes.byref(A), ctypes.c_void_p(4096), 32, None,
                                   None) == E
    B = capi.sketch_csc(999, 10, 3, 8, 8, 8, 0)
    assert lib.sketch_apply_pregen(h, ctypes.byref(B), ctypes.c_void_p(4096), 32, out,
                                   None) == E
    assert lib.sketch_destroy(h) == capi.SKETCH_OK


def test_heuristic_plans_need_no_gpu():
    """With tuning off the plan is the heuristic's, chosen on the host:
    +-1 -> REGEN; U and N -> TILE, with tensor-memory sums (32 warps x 32
    columns, panels of 1248 rows) when n > 256; very sparse input -> REGEN."""
    from paper_2310_15419_gb300 import capi
    lib = capi.load()

    def plan(m, n, d, dist, nnz):
        h = ctypes.c_void_p()
        assert lib.sketch_create(m, n, d, dist, 1, ctypes.byref(h)) == capi.SKETCH_OK
        assert lib.sketch_set_autotune(h, 0) == capi.SKETCH_OK
        A = capi.sketch_csc(m, n, nnz, 8, 8, 8, 0)
        p = capi.sketch_plan()
        assert lib.sketch_get_plan(h, ctypes.byref(A), ctypes.byref(p), None) == capi.SKETCH_OK
        assert lib.sketch_destroy(h) == capi.SKETCH_OK
        return p.as_dict()

    p = plan(2_000_000, 1000, 3000, 0, 10_000_000)
    assert (p["mode"], p["q_tiles"], p["split"]) == (capi.SKETCH_MODE_REGEN, 4, 8)
    for dist in (1, 2):
        p = plan(2_000_000, 1000, 3000, dist, 10_000_000)
        assert (p["mode"], p["panel_rows"], p["cols_per_warp"], p["tile_acc"]) == \
            (capi.SKETCH_MODE_TILE, 1248, 32, 1)
        assert p["row_groups"] >= 20          # <= 512 terms of a column per range
        p = plan(100_000, 200, 400, dist, 1_000_000)
        assert (p["mode"], p["panel_rows"], p["cols_per_warp"], p["tile_acc"]) == \
            (capi.SKETCH_MODE_TILE, 1024, 16, 0)
        p = plan(100_000, 200, 400, dist, 500)
        assert p["mode"] == capi.SKETCH_MODE_REGEN
