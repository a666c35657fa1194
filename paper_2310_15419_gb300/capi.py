"""Thin Python binding of libsketch.so (include/sketch.h).

Argument marshalling only: every step of the sketch, the QR and LSQR runs in
the library's CUDA kernels.  PyTorch supplies device memory and streams.  The
binding fails loudly (ImportError / RuntimeError) when the library cannot be
built or loaded; there is no CPU fallback.

Names match the C ABI: ``sketch_create``, ``sketch_apply``, ... operate on raw
handles; the classes ``DeviceCSC`` and ``Sketch`` wrap them for tensors.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import build as _build

SKETCH_OK = 0
SKETCH_ERR_ARG = -1
SKETCH_ERR_OOM = -2
SKETCH_ERR_CSC = -3
SKETCH_ERR_CUDA = -4
SKETCH_ERR_TIMEOUT = -5
SKETCH_ERR_NO_CONVERGENCE = -6
SKETCH_ERR_UNSUPPORTED = -7

SKETCH_PM1, SKETCH_UNIFORM, SKETCH_NORMAL = 0, 1, 2
SKETCH_F32, SKETCH_BF16 = 0, 1
SKETCH_MODE_AUTO, SKETCH_MODE_REGEN, SKETCH_MODE_PANEL, SKETCH_MODE_TILE = 0, 1, 2, 3
SKETCH_LSQ_SAP_QR, SKETCH_LSQ_SAP_SVD, SKETCH_LSQ_LSQR_D = 0, 1, 2
LSQ_METHODS = {"sap_qr": SKETCH_LSQ_SAP_QR, "sap_svd": SKETCH_LSQ_SAP_SVD,
               "lsqr_d": SKETCH_LSQ_LSQR_D}

DIST_NAMES = {"pm1": SKETCH_PM1, "uniform": SKETCH_UNIFORM,
              "normal": SKETCH_NORMAL}


class SketchError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("sketch error %d: %s" % (code, msg))
        self.code = code


class sketch_csc(ctypes.Structure):
    _fields_ = [("m", ctypes.c_int64), ("n", ctypes.c_int64),
                ("nnz", ctypes.c_int64), ("colptr", ctypes.c_void_p),
                ("rowidx", ctypes.c_void_p), ("values", ctypes.c_void_p),
                ("dtype", ctypes.c_int32)]


class sketch_plan(ctypes.Structure):
    _fields_ = [("mode", ctypes.c_int32), ("q_tiles", ctypes.c_int32),
                ("split", ctypes.c_int32), ("n_block", ctypes.c_int32),
                ("row_groups", ctypes.c_int32), ("panel_rows", ctypes.c_int32),
                ("cols_per_warp", ctypes.c_int32), ("tc_min_row_nnz", ctypes.c_int32),
                ("tile_acc", ctypes.c_int32), ("tc_fp8", ctypes.c_int32)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class sketch_server_result(ctypes.Structure):
    _fields_ = [("id", ctypes.c_int64), ("status", ctypes.c_int32),
                ("iters", ctypes.c_int32), ("error", ctypes.c_double),
                ("t_submit", ctypes.c_double), ("t_start", ctypes.c_double),
                ("t_done", ctypes.c_double)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class sketch_lsq_info(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int32), ("status", ctypes.c_int32),
                ("istop", ctypes.c_int32), ("rank", ctypes.c_int32),
                ("error", ctypes.c_double), ("test2", ctypes.c_double),
                ("ms_sketch", ctypes.c_double), ("ms_qr", ctypes.c_double),
                ("ms_lsqr", ctypes.c_double)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


_lock = threading.Lock()
_lib = None

# (name, restype, argtypes) for every function include/sketch.h declares.
_VP, _I32, _I64, _U32, _U64, _D = (ctypes.c_void_p, ctypes.c_int32,
                                   ctypes.c_int64, ctypes.c_uint32,
                                   ctypes.c_uint64, ctypes.c_double)
_CSCP = ctypes.POINTER(sketch_csc)
SIGNATURES = [
    ("sketch_create", _I32, [_I64, _I64, _I64, _I32, _U64, ctypes.POINTER(_VP)]),
    ("sketch_destroy", _I32, [_VP]),
    ("sketch_set_stream_id", _I32, [_VP, _U32]),
    ("sketch_set_plan", _I32, [_VP, ctypes.POINTER(sketch_plan)]),
    ("sketch_get_plan", _I32, [_VP, _CSCP, ctypes.POINTER(sketch_plan), _VP]),
    ("sketch_apply", _I32, [_VP, _CSCP, _VP, _VP]),
    ("sketch_apply_noalloc", _I32, [_VP, _CSCP, _VP, _VP]),
    ("sketch_generate_S", _I32, [_VP, _VP, _I64, _VP]),
    ("sketch_apply_pregen", _I32, [_VP, _CSCP, _VP, _I64, _VP, _VP]),
    ("sketch_last_error", ctypes.c_char_p, [_VP]),
    ("sketch_device_status", _I32, [_VP, _VP]),
    ("sketch_validate_csc", _I32, [_CSCP, _VP]),
    ("sketch_lsq_solve", _I32, [_VP, _CSCP, _VP, _VP, _D, _I32,
                                ctypes.POINTER(sketch_lsq_info), _VP]),
    ("sketch_lsq_solve_method", _I32, [_VP, _CSCP, _VP, _VP, _D, _I32, _I32,
                                       ctypes.POINTER(sketch_lsq_info), _VP]),
    ("sketch_debug_philox", _I32, [_VP, _U64, _VP, _I64, _VP]),
    ("sketch_debug_S", _I32, [_I32, _U64, _U32, _VP, _VP, _VP, _I64, _VP]),
    ("sketch_debug_normal_pair", _I32, [_VP, _VP, _I64, _VP]),
    ("sketch_debug_wait_timeout", _I32, [_VP, _VP]),
    ("sketch_set_counting", _I32, [_VP, _I32]),
    ("sketch_generated_entries", _I64, [_VP, _VP]),
    ("sketch_launch_count", _I64, [_VP]),
    ("sketch_bench_generator", _I32, [_I32, _U64, _I64, _I64, _VP, _VP]),
    ("sketch_bench_fma", _I32, [_I64, _I64, _VP, _VP]),
    ("sketch_debug_candidates", _I32, [_VP, _CSCP, ctypes.POINTER(sketch_plan), _I32,
                                       ctypes.POINTER(_I32)]),
    ("sketch_debug_qr", _I32, [_I64, _I64, _VP, _VP, _VP, _VP]),
    ("sketch_batch_create", _I32, [_I32, ctypes.POINTER(_VP), _CSCP,
                                   ctypes.POINTER(_VP), _VP, ctypes.POINTER(_VP)]),
    ("sketch_batch_apply", _I32, [_VP, _VP]),
    ("sketch_batch_info", _I32, [_VP, ctypes.POINTER(_I32), ctypes.POINTER(_I64),
                                 ctypes.POINTER(_I64)]),
    ("sketch_batch_status", _I32, [_VP, _VP]),
    ("sketch_batch_destroy", _I32, [_VP]),
    ("sketch_reshape", _I32, [_VP, _I64, _I64, _I64]),
    ("sketch_set_autotune", _I32, [_VP, _I32]),
    ("sketch_server_create", _I32, [_I32, _I64, _I32, _U64, _D, _D, _I32,
                                    ctypes.POINTER(_VP)]),
    ("sketch_server_submit", _I32, [_VP, _CSCP, _VP, _VP, ctypes.POINTER(_I64)]),
    ("sketch_server_poll", _I32, [_VP, ctypes.POINTER(sketch_server_result), _I32,
                                  ctypes.POINTER(_I32), _I32]),
    ("sketch_server_drain", _I32, [_VP]),
    ("sketch_server_now", _D, [_VP]),
    ("sketch_server_destroy", _I32, [_VP]),
]


def library_path() -> str:
    return _build.LIB


def load(build_if_needed: bool = True):
    """Load libsketch.so (building it first if it is missing or stale)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.build() if build_if_needed else _build.LIB
        if not os.path.exists(path):
            raise ImportError("libsketch.so not found at %s" % path)
        lib = ctypes.CDLL(path)
        for name, res, args in SIGNATURES:
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def _check(rc, h=None):
    if rc != SKETCH_OK:
        lib = load()
        msg = lib.sketch_last_error(h)
        raise SketchError(rc, (msg or b"").decode())


def _stream_ptr(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


class DeviceCSC:
    """A CSC matrix resident on the GPU (torch tensors) + its ABI descriptor.

    Built from the host arrays of ``inputs.CSC``; the tensors are owned here
    and stay alive as long as this object."""

    def __init__(self, A, device="cuda"):
        import torch
        self.m, self.n = int(A.m), int(A.n)
        self.colptr = torch.from_numpy(np.ascontiguousarray(A.colptr, np.int32)).to(device)
        self.rowidx = torch.from_numpy(np.ascontiguousarray(A.rowidx, np.int32)).to(device)
        if A.dtype == SKETCH_BF16:
            bits = np.ascontiguousarray(A.values_bf16, np.uint16).view(np.int16)
            self.values = torch.from_numpy(bits).to(device).view(torch.bfloat16)
        else:
            self.values = torch.from_numpy(np.ascontiguousarray(A.values, np.float32)).to(device)
        self.dtype = int(A.dtype)
        self.nnz = int(self.rowidx.numel())
        self.desc = self.descriptor()

    def descriptor(self) -> sketch_csc:
        return sketch_csc(self.m, self.n, self.nnz, self.colptr.data_ptr(),
                          self.rowidx.data_ptr() if self.nnz else 0,
                          self.values.data_ptr() if self.nnz else 0, self.dtype)

    @property
    def nbytes(self):
        return (self.colptr.numel() * 4 + self.rowidx.numel() * 4 +
                self.values.numel() * self.values.element_size())


class Sketch:
    """A_hat = S A with S (d x m) regenerated on the GPU (sketch_create)."""

    def __init__(self, m, n, d, dist="pm1", seed=1, stream_id=0):
        lib = load()
        self.m, self.n, self.d = int(m), int(n), int(d)
        self.dist = DIST_NAMES[dist] if isinstance(dist, str) else int(dist)
        self.seed = int(seed)
        h = ctypes.c_void_p()
        _check(lib.sketch_create(self.m, self.n, self.d, self.dist,
                                 ctypes.c_uint64(self.seed), ctypes.byref(h)))
        self.h = h
        if stream_id:
            _check(lib.sketch_set_stream_id(self.h, stream_id), self.h)

    def close(self):
        if getattr(self, "h", None):
            load().sketch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_autotune(self, on=True):
        _check(load().sketch_set_autotune(self.h, 1 if on else 0), self.h)

    def reshape(self, m, n, d):
        _check(load().sketch_reshape(self.h, m, n, d), self.h)
        self.m, self.n, self.d = int(m), int(n), int(d)

    def set_plan(self, mode=SKETCH_MODE_AUTO, q_tiles=0, split=0, n_block=0,
                 row_groups=0, panel_rows=0, cols_per_warp=0, tc_min_row_nnz=0,
                 tile_acc=0, tc_fp8=0):
        p = sketch_plan(mode, q_tiles, split, n_block, row_groups, panel_rows,
                        cols_per_warp, tc_min_row_nnz, tile_acc, tc_fp8)
        _check(load().sketch_set_plan(self.h, ctypes.byref(p)), self.h)

    def get_plan(self, A: DeviceCSC, stream=None) -> dict:
        p = sketch_plan()
        _check(load().sketch_get_plan(self.h, ctypes.byref(A.desc),
                                      ctypes.byref(p), _stream_ptr(stream)), self.h)
        return p.as_dict()

    def candidates(self, A: DeviceCSC) -> list:
        """The tuner's candidate plans for A (sketch_debug_candidates)."""
        arr = (sketch_plan * 64)()
        cnt = ctypes.c_int32()
        _check(load().sketch_debug_candidates(self.h, ctypes.byref(A.desc), arr, 64,
                                              ctypes.byref(cnt)), self.h)
        return [arr[t].as_dict() for t in range(min(cnt.value, 64))]

    def apply(self, A: DeviceCSC, out=None, stream=None):
        import torch
        if out is None:
            # column-major d x n == row-major n x d
            out = torch.empty((self.n, self.d), dtype=torch.float32,
                              device=A.colptr.device)
        _check(load().sketch_apply(self.h, ctypes.byref(A.desc),
                                   ctypes.c_void_p(out.data_ptr()),
                                   _stream_ptr(stream)), self.h)
        return out

    def apply_noalloc(self, A: DeviceCSC, out, stream=None):
        """sketch_apply_noalloc: same result as apply(); allocates nothing
        (`out` must be a preallocated n x d float32 tensor)."""
        _check(load().sketch_apply_noalloc(self.h, ctypes.byref(A.desc),
                                           ctypes.c_void_p(out.data_ptr()),
                                           _stream_ptr(stream)), self.h)
        return out

    def generate_S(self, ld_s=None, out=None, stream=None):
        """sketch_generate_S: S materialised on the device as an (m, ld_s)
        float32 tensor whose row j holds column j of S (rows 0..d-1 used);
        ld_s defaults to d rounded up to a multiple of 4."""
        import torch
        if ld_s is None:
            ld_s = (self.d + 3) // 4 * 4
        if out is None:
            out = torch.empty((self.m, ld_s), dtype=torch.float32, device="cuda")
        _check(load().sketch_generate_S(self.h, ctypes.c_void_p(out.data_ptr()), int(ld_s),
                                        _stream_ptr(stream)), self.h)
        return out

    def apply_pregen(self, A: DeviceCSC, S, out=None, stream=None):
        """sketch_apply_pregen: A_hat = S A with S read from `S` (as written by
        generate_S, leading dimension S.shape[1])."""
        import torch
        if out is None:
            out = torch.empty((self.n, self.d), dtype=torch.float32,
                              device=A.colptr.device)
        _check(load().sketch_apply_pregen(self.h, ctypes.byref(A.desc),
                                          ctypes.c_void_p(S.data_ptr()), int(S.stride(0)),
                                          ctypes.c_void_p(out.data_ptr()),
                                          _stream_ptr(stream)), self.h)
        return out

    def device_status(self, stream=None):
        return load().sketch_device_status(self.h, _stream_ptr(stream))

    def set_counting(self, on=True):
        _check(load().sketch_set_counting(self.h, 1 if on else 0), self.h)

    def launch_count(self) -> int:
        return int(load().sketch_launch_count(self.h))

    def generated_entries(self, stream=None) -> int:
        return int(load().sketch_generated_entries(self.h, _stream_ptr(stream)))

    def lsq_solve(self, A: DeviceCSC, b, x=None, tol=1e-10, maxit=1000,
                  stream=None, check=True, method=None):
        """sketch_lsq_solve, or sketch_lsq_solve_method when `method` is given
        ("sap_qr", "sap_svd", "lsqr_d" or the enum value)."""
        import torch
        if x is None:
            x = torch.zeros(self.n, dtype=torch.float64, device=b.device)
        info = sketch_lsq_info()
        if method is None:
            rc = load().sketch_lsq_solve(self.h, ctypes.byref(A.desc),
                                         ctypes.c_void_p(b.data_ptr()),
                                         ctypes.c_void_p(x.data_ptr()), float(tol),
                                         int(maxit), ctypes.byref(info),
                                         _stream_ptr(stream))
        else:
            code = LSQ_METHODS[method] if isinstance(method, str) else int(method)
            rc = load().sketch_lsq_solve_method(self.h, ctypes.byref(A.desc),
                                                ctypes.c_void_p(b.data_ptr()),
                                                ctypes.c_void_p(x.data_ptr()), float(tol),
                                                int(maxit), code, ctypes.byref(info),
                                                _stream_ptr(stream))
        if check and rc not in (SKETCH_OK, SKETCH_ERR_NO_CONVERGENCE):
            _check(rc, self.h)
        d = info.as_dict()
        d["rc"] = rc
        return x, d


class Batch:
    """Many uneven sketches in one persistent launch (sketch_batch_*)."""

    def __init__(self, sketches, mats, outs=None, stream=None):
        import torch
        lib = load()
        self.sketches, self.mats = list(sketches), list(mats)
        if outs is None:
            outs = [torch.empty((A.n, sk.d), dtype=torch.float32, device="cuda")
                    for sk, A in zip(self.sketches, self.mats)]
        self.outs = list(outs)
        cnt = len(self.sketches)
        H = (ctypes.c_void_p * cnt)(*[sk.h.value for sk in self.sketches])
        D = (sketch_csc * cnt)(*[A.desc for A in self.mats])
        O = (ctypes.c_void_p * cnt)(*[o.data_ptr() for o in self.outs])
        b = ctypes.c_void_p()
        _check(lib.sketch_batch_create(cnt, H, D, O, _stream_ptr(stream),
                                       ctypes.byref(b)))
        self.b = b

    def apply(self, stream=None):
        _check(load().sketch_batch_apply(self.b, _stream_ptr(stream)))
        return self.outs

    def info(self):
        q, n, l = ctypes.c_int32(), ctypes.c_int64(), ctypes.c_int64()
        _check(load().sketch_batch_info(self.b, ctypes.byref(q), ctypes.byref(n),
                                        ctypes.byref(l)))
        return {"q_tiles": q.value, "items": n.value, "launches": l.value}

    def status(self, stream=None):
        return load().sketch_batch_status(self.b, _stream_ptr(stream))

    def close(self):
        if getattr(self, "b", None):
            load().sketch_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Continuous-batching SAP-QR least-squares server (sketch_server_*).

    submit() takes host arrays (an ``inputs.CSC`` and b); they are kept alive
    here until the request is polled.  poll() returns result dicts with the
    solution under "x"."""

    def __init__(self, slots=4, mem_budget=32 << 30, dist="pm1", seed=1,
                 d_over_n=2.0, tol=1e-10, maxit=1000):
        lib = load()
        self.dist = DIST_NAMES[dist] if isinstance(dist, str) else int(dist)
        s = ctypes.c_void_p()
        _check(lib.sketch_server_create(int(slots), int(mem_budget), self.dist,
                                        ctypes.c_uint64(seed), float(d_over_n),
                                        float(tol), int(maxit), ctypes.byref(s)))
        self.s = s
        self.live = {}

    def submit(self, A, b):
        lib = load()
        colptr = np.ascontiguousarray(A.colptr, np.int32)
        rowidx = np.ascontiguousarray(A.rowidx, np.int32)
        if A.dtype == SKETCH_BF16:
            vals = np.ascontiguousarray(A.values_bf16, np.uint16)
        else:
            vals = np.ascontiguousarray(A.values, np.float32)
        bb = np.ascontiguousarray(b, np.float64)
        x = np.zeros(A.n, dtype=np.float64)
        desc = sketch_csc(A.m, A.n, int(colptr[-1]), colptr.ctypes.data,
                          rowidx.ctypes.data, vals.ctypes.data, int(A.dtype))
        rid = ctypes.c_int64()
        _check(lib.sketch_server_submit(self.s, ctypes.byref(desc),
                                        ctypes.c_void_p(bb.ctypes.data),
                                        ctypes.c_void_p(x.ctypes.data),
                                        ctypes.byref(rid)))
        self.live[rid.value] = (colptr, rowidx, vals, bb, x, desc)
        return rid.value

    def poll(self, max_results=64, wait_ms=0):
        arr = (sketch_server_result * max_results)()
        n = ctypes.c_int32()
        _check(load().sketch_server_poll(self.s, arr, max_results, ctypes.byref(n),
                                         int(wait_ms)))
        out = []
        for t in range(n.value):
            d = arr[t].as_dict()
            keep = self.live.pop(d["id"])
            d["x"] = keep[4]
            out.append(d)
        return out

    def drain(self):
        _check(load().sketch_server_drain(self.s))

    def now(self):
        return load().sketch_server_now(self.s)

    def close(self):
        if getattr(self, "s", None):
            load().sketch_server_destroy(self.s)
            self.s = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def validate_csc(A: DeviceCSC, stream=None) -> int:
    return load().sketch_validate_csc(ctypes.byref(A.desc), _stream_ptr(stream))


def debug_philox(ctr, seed, stream=None, both=False):
    """ctr: int tensor (count, 4) of uint32 values on the GPU (as int32 bits).
    Returns the (count, 4) blocks; with both=True a pair (running-key form,
    round-key form)."""
    import torch
    count = ctr.shape[0]
    out = torch.empty((2 * count, 4), dtype=torch.int32, device=ctr.device)
    _check(load().sketch_debug_philox(ctypes.c_void_p(ctr.data_ptr()),
                                      ctypes.c_uint64(seed),
                                      ctypes.c_void_p(out.data_ptr()), count,
                                      _stream_ptr(stream)))
    return (out[:count], out[count:]) if both else out[:count]


def debug_normal_pair(words, stream=None):
    """words: int tensor (count, 2) of uint32 values on the GPU (as int32
    bits), (radius word, angle word) per row; returns (count, 2) float32."""
    import torch
    count = words.shape[0]
    out = torch.empty((count, 2), dtype=torch.float32, device=words.device)
    _check(load().sketch_debug_normal_pair(ctypes.c_void_p(words.data_ptr()),
                                           ctypes.c_void_p(out.data_ptr()), count,
                                           _stream_ptr(stream)))
    return out


def debug_wait_timeout(sketch, stream=None):
    """Run the bounded-wait timeout path on purpose (see include/sketch.h)."""
    _check(load().sketch_debug_wait_timeout(sketch.h, _stream_ptr(stream)), sketch.h)


def bench_generator(dist, seed, threads, blocks_per_thread, sink, stream=None):
    """Launch the generator throughput probe (see include/sketch.h)."""
    _check(load().sketch_bench_generator(int(dist), ctypes.c_uint64(seed),
                                         int(threads), int(blocks_per_thread),
                                         ctypes.c_void_p(sink.data_ptr()),
                                         _stream_ptr(stream)))


def bench_fma(threads, iters, sink, stream=None):
    """Launch the FP32 FMA throughput probe (see include/sketch.h)."""
    _check(load().sketch_bench_fma(int(threads), int(iters),
                                   ctypes.c_void_p(sink.data_ptr()), _stream_ptr(stream)))


def debug_qr(A, stream=None):
    """R and R^{-1} (row-major n x n) of the device FP64 QR of A (d x n)."""
    import torch
    d, n = A.shape
    a = A.t().contiguous()  # column-major d x n
    R = torch.empty((n, n), dtype=torch.float64, device=A.device)
    Ri = torch.empty((n, n), dtype=torch.float64, device=A.device)
    _check(load().sketch_debug_qr(d, n, ctypes.c_void_p(a.data_ptr()),
                                  ctypes.c_void_p(R.data_ptr()),
                                  ctypes.c_void_p(Ri.data_ptr()),
                                  _stream_ptr(stream)))
    return R, Ri


def debug_S(dist, seed, stream_id, i, j, stream=None):
    import torch
    out = torch.empty(i.numel(), dtype=torch.float32, device=i.device)
    _check(load().sketch_debug_S(int(dist), ctypes.c_uint64(seed), stream_id,
                                 ctypes.c_void_p(i.data_ptr()),
                                 ctypes.c_void_p(j.data_ptr()),
                                 ctypes.c_void_p(out.data_ptr()), i.numel(),
                                 _stream_ptr(stream)))
    return out
