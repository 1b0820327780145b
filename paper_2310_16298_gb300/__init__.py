"""Python binding of the GB300 stencil-matrixization library (``include/stencil.h``).

The functions below carry the C names and only marshal arguments: every step
of a sweep runs in the library's CUDA kernels.  Importing the package does not
load the library; the first call does, and raises if ``libstencil_gb300.so``
has not been built (``python -m paper_2310_16298_gb300.build``).  There is no
CPU fallback.

``Plan`` wraps a plan handle for PyTorch CUDA tensors (device memory and the
current stream come from PyTorch; nothing else does).
"""
from __future__ import annotations

import ctypes
import os
import threading
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libstencil_gb300.so")

# status codes
OK, EINVAL, ENOMEM, ECUDA, EBUSY, ENOTREADY, ETIMEDOUT, EUNSUPPORTED = range(8)
STATUS_NAMES = ["OK", "EINVAL", "ENOMEM", "ECUDA", "EBUSY", "ENOTREADY", "ETIMEDOUT", "EUNSUPPORTED"]
STAR, BOX = 0, 1
F32, F64 = 0, 1
BC_DIRICHLET_ZERO, BC_PERIODIC = 0, 1
PREC_NATIVE, PREC_TF32, PREC_TF32X3, PREC_BF16, PREC_BF16X2, PREC_BF16X3, PREC_BF16_W2 = range(7)
IMPL_AUTO, IMPL_GATHER, IMPL_MATRIXIZED = range(3)

KINDS = {"star": STAR, "box": BOX}
DTYPES = {"f32": F32, "f64": F64}
BCS = {"dirichlet": BC_DIRICHLET_ZERO, "periodic": BC_PERIODIC}
PRECS = {"native": PREC_NATIVE, "tf32": PREC_TF32, "tf32x3": PREC_TF32X3, "bf16": PREC_BF16,
         "bf16x2": PREC_BF16X2, "bf16x3": PREC_BF16X3, "bf16w2": PREC_BF16_W2}
IMPLS = {"auto": IMPL_AUTO, "gather": IMPL_GATHER, "matrixized": IMPL_MATRIXIZED}


class StencilError(RuntimeError):
    def __init__(self, status: int, where: str, message: str):
        self.status = status
        name = STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else str(status)
        super().__init__(f"{where}: {name}: {message}")


class stencil_options(ctypes.Structure):
    _fields_ = [("prec", ctypes.c_int32), ("bc", ctypes.c_int32), ("impl", ctypes.c_int32),
                ("tb", ctypes.c_int32), ("cover", ctypes.c_int32), ("pitch", ctypes.c_int32),
                ("unit_planes", ctypes.c_int32), ("reserved", ctypes.c_int32 * 1)]


class stencil_batch_info_t(ctypes.Structure):
    _fields_ = [("packed", ctypes.c_int32), ("tb", ctypes.c_int32), ("launches", ctypes.c_int32),
                ("tile_shape", ctypes.c_int32), ("tiles", ctypes.c_int64), ("updates", ctypes.c_int64)]


class stencil_request(ctypes.Structure):
    _fields_ = [("ndim", ctypes.c_int32), ("radius", ctypes.c_int32), ("kind", ctypes.c_int32),
                ("dtype", ctypes.c_int32), ("bc", ctypes.c_int32), ("impl", ctypes.c_int32),
                ("shape", ctypes.c_int64 * 3), ("coeffs", ctypes.POINTER(ctypes.c_double)),
                ("h_in", ctypes.c_void_p), ("seed", ctypes.c_uint64), ("lo", ctypes.c_double),
                ("hi", ctypes.c_double), ("steps", ctypes.c_int64)]


class stencil_request_stats(ctypes.Structure):
    _fields_ = [("submit_s", ctypes.c_double), ("admit_s", ctypes.c_double), ("done_s", ctypes.c_double),
                ("impl", ctypes.c_int32), ("status", ctypes.c_int32), ("updates", ctypes.c_int64)]


class stencil_server_stats_t(ctypes.Structure):
    _fields_ = [(f, ctypes.c_int64) for f in ("queued", "resident", "admitted", "completed", "bytes_in_use",
                                              "peak_bytes", "peak_resident", "quanta_issued")]


class stencil_plan_info_t(ctypes.Structure):
    _fields_ = [("impl", ctypes.c_int32), ("prec", ctypes.c_int32), ("tb", ctypes.c_int32),
                ("n_lines", ctypes.c_int32), ("n_scalar", ctypes.c_int32), ("tile_n", ctypes.c_int32),
                ("scratch_bytes", ctypes.c_int64), ("device_error", ctypes.c_int32),
                ("cover", ctypes.c_int32), ("kernels_per_sweep", ctypes.c_int32)]


_P = ctypes.c_void_p
_I64P = ctypes.POINTER(ctypes.c_int64)
_DP = ctypes.POINTER(ctypes.c_double)

# name -> (restype, argtypes); the names are the C ABI's.
_SIGS = {
    "stencil_plan_create": (ctypes.c_int, [ctypes.POINTER(_P), ctypes.c_int, _I64P, ctypes.c_int,
                                           ctypes.c_int, _DP, ctypes.c_int,
                                           ctypes.POINTER(stencil_options)]),
    "stencil_plan_destroy": (ctypes.c_int, [_P]),
    "stencil_plan_info": (ctypes.c_int, [_P, ctypes.POINTER(stencil_plan_info_t)]),
    "stencil_plan_raise_error": (ctypes.c_int, [_P, ctypes.c_uint32]),
    "stencil_apply": (ctypes.c_int, [_P, _P, _P, ctypes.c_int64, _P]),
    "stencil_apply_host": (ctypes.c_int, [_P, _P, _P, ctypes.c_int64]),
    "stencil_apply_noalloc": (ctypes.c_int, [_P, _P, _P, ctypes.c_int64, _P]),
    "stencil_submit": (ctypes.c_int, [_P, _P, _P, ctypes.c_int64, ctypes.POINTER(ctypes.c_uint64)]),
    "stencil_poll": (ctypes.c_int, [ctypes.c_uint64]),
    "stencil_wait": (ctypes.c_int, [ctypes.c_uint64, ctypes.c_int64]),
    "stencil_last_error": (ctypes.c_char_p, []),
    "stencil_batch_run": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(_P), ctypes.POINTER(_P),
                                         ctypes.POINTER(_P), _I64P, _P]),
    "stencil_batch_create": (ctypes.c_int, [ctypes.POINTER(_P), ctypes.c_int, ctypes.POINTER(_P),
                                            ctypes.POINTER(_P), ctypes.POINTER(_P), _I64P, ctypes.c_int32]),
    "stencil_batch_create_ex": (ctypes.c_int, [ctypes.POINTER(_P), ctypes.c_int, ctypes.POINTER(_P),
                                               ctypes.POINTER(_P), ctypes.POINTER(_P), _I64P, ctypes.c_int32,
                                               ctypes.c_int32]),
    "stencil_batch_launch": (ctypes.c_int, [_P, _P]),
    "stencil_batch_info": (ctypes.c_int, [_P, ctypes.POINTER(stencil_batch_info_t)]),
    "stencil_batch_destroy": (ctypes.c_int, [_P]),
    "stencil_server_create": (ctypes.c_int, [ctypes.POINTER(_P), ctypes.c_int64, ctypes.c_int32, ctypes.c_int32,
                                             ctypes.c_int32]),
    "stencil_server_submit": (ctypes.c_int, [_P, ctypes.POINTER(stencil_request), ctypes.POINTER(ctypes.c_uint64)]),
    "stencil_server_poll": (ctypes.c_int, [_P, ctypes.c_uint64]),
    "stencil_server_wait": (ctypes.c_int, [_P, ctypes.c_uint64, ctypes.c_int64]),
    "stencil_server_result": (ctypes.c_int, [_P, ctypes.c_uint64, _P, ctypes.POINTER(stencil_request_stats)]),
    "stencil_server_stats": (ctypes.c_int, [_P, ctypes.POINTER(stencil_server_stats_t)]),
    "stencil_server_destroy": (ctypes.c_int, [_P]),
    "stencil_fill_uniform": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int64, ctypes.c_uint64, ctypes.c_int64,
                                            ctypes.c_double, ctypes.c_double, _P]),
    "stencil_error_norms": (ctypes.c_int, [_P, ctypes.c_int, _P, ctypes.c_int64, _DP, _P]),
    "stencil_band_operand": (ctypes.c_int, [ctypes.c_int, _DP, ctypes.c_int, ctypes.c_int, _DP]),
    "stencil_min_line_cover": (ctypes.c_int, [ctypes.c_int, _P, _P, _P, ctypes.POINTER(ctypes.c_int32)]),
    "stencil_line_cover": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                          ctypes.c_int, ctypes.POINTER(ctypes.c_int32), _I64P]),
    "stencil_version": (ctypes.c_char_p, []),
}

_lock = threading.Lock()
_lib = None


def lib():
    """The loaded C library (raises if it was not built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise ImportError(f"{LIB_PATH} is missing: build the CUDA library first "
                                  "(python -m paper_2310_16298_gb300.build)")
            h = ctypes.CDLL(LIB_PATH)
            for name, (res, args) in _SIGS.items():
                fn = getattr(h, name)
                fn.restype = res
                fn.argtypes = args
            _lib = h
    return _lib


def exported_symbols():
    return list(_SIGS)


def _check(status: int, where: str):
    if status != OK:
        raise StencilError(status, where, stencil_last_error())


def _dp(a: np.ndarray):
    return a.ctypes.data_as(_DP)


# ---------------------------------------------------------------- C names
def stencil_last_error() -> str:
    return lib().stencil_last_error().decode()


def stencil_version() -> str:
    return lib().stencil_version().decode()


COVERS = {"auto": 0, "parallel": 1, "hybrid": 2}


def make_options(prec="native", bc="dirichlet", impl="auto", tb=0, cover="auto", pitch=0,
                 unit_planes=0) -> stencil_options:
    o = stencil_options()
    o.prec = PRECS[prec] if isinstance(prec, str) else int(prec)
    o.bc = BCS[bc] if isinstance(bc, str) else int(bc)
    o.impl = IMPLS[impl] if isinstance(impl, str) else int(impl)
    o.tb = int(tb)
    o.cover = COVERS[cover] if isinstance(cover, str) else int(cover)
    o.pitch = int(pitch)
    o.unit_planes = int(unit_planes)
    return o


def stencil_plan_create(shape: Sequence[int], radius: int, kind, coeffs: np.ndarray, dtype,
                        opt: Optional[stencil_options] = None) -> int:
    """Returns the plan handle (an int).  Raises StencilError on a non-OK status."""
    shp = np.ascontiguousarray(shape, dtype=np.int64)
    c = np.ascontiguousarray(coeffs, dtype=np.float64)
    k = KINDS[kind] if isinstance(kind, str) else int(kind)
    dt = DTYPES[dtype] if isinstance(dtype, str) else int(dtype)
    h = _P()
    st = lib().stencil_plan_create(ctypes.byref(h), len(shp), shp.ctypes.data_as(_I64P), int(radius), k,
                                   _dp(c), dt, ctypes.byref(opt) if opt is not None else None)
    _check(st, "stencil_plan_create")
    return h.value


def stencil_plan_destroy(plan: int):
    _check(lib().stencil_plan_destroy(plan), "stencil_plan_destroy")


def stencil_plan_info(plan: int) -> dict:
    info = stencil_plan_info_t()
    _check(lib().stencil_plan_info(plan, ctypes.byref(info)), "stencil_plan_info")
    return {f: getattr(info, f) for f, _ in info._fields_}


def stencil_plan_raise_error(plan: int, bits: int):
    _check(lib().stencil_plan_raise_error(plan, int(bits)), "stencil_plan_raise_error")


def stencil_apply(plan: int, d_in: int, d_out: int, steps: int, stream: int = 0):
    _check(lib().stencil_apply(plan, d_in, d_out, int(steps), stream), "stencil_apply")


def stencil_apply_noalloc(plan: int, d_in: int, d_out: int, steps: int, stream: int = 0):
    _check(lib().stencil_apply_noalloc(plan, d_in, d_out, int(steps), stream), "stencil_apply_noalloc")


def stencil_apply_host(plan: int, h_in: np.ndarray, h_out: np.ndarray, steps: int):
    _check(lib().stencil_apply_host(plan, h_in.ctypes.data, h_out.ctypes.data, int(steps)),
           "stencil_apply_host")


def stencil_submit(plan: int, d_in: int, d_out: int, steps: int) -> int:
    t = ctypes.c_uint64()
    _check(lib().stencil_submit(plan, d_in, d_out, int(steps), ctypes.byref(t)), "stencil_submit")
    return t.value


def stencil_poll(ticket: int) -> int:
    """Returns the raw status (OK, ENOTREADY, or an error code)."""
    return int(lib().stencil_poll(ticket))


def stencil_wait(ticket: int, timeout_ms: int = -1) -> int:
    """Returns the raw status (OK, ETIMEDOUT, or an error code)."""
    return int(lib().stencil_wait(ticket, int(timeout_ms)))


def stencil_batch_run(plans: Sequence[int], d_in: Sequence[int], d_out: Sequence[int],
                      steps: Sequence[int], stream: int = 0):
    n = len(plans)
    P = (_P * n)(*plans)
    I = (_P * n)(*d_in)
    O = (_P * n)(*d_out)
    S = np.ascontiguousarray(steps, dtype=np.int64)
    _check(lib().stencil_batch_run(n, P, I, O, S.ctypes.data_as(_I64P), stream), "stencil_batch_run")


def stencil_batch_create(plans: Sequence[int], d_in: Sequence[int], d_out: Sequence[int],
                         steps: Sequence[int], tb: int = 0) -> int:
    n = len(plans)
    h = _P()
    P = (_P * n)(*plans)
    I = (_P * n)(*d_in)
    O = (_P * n)(*d_out)
    S = np.ascontiguousarray(steps, dtype=np.int64)
    _check(lib().stencil_batch_create(ctypes.byref(h), n, P, I, O, S.ctypes.data_as(_I64P), int(tb)),
           "stencil_batch_create")
    return h.value


def stencil_batch_create_ex(plans: Sequence[int], d_in: Sequence[int], d_out: Sequence[int],
                            steps: Sequence[int], tb: int = 0, tile_shape: int = -1) -> int:
    n = len(plans)
    h = _P()
    P = (_P * n)(*plans)
    I = (_P * n)(*d_in)
    O = (_P * n)(*d_out)
    S = np.ascontiguousarray(steps, dtype=np.int64)
    _check(lib().stencil_batch_create_ex(ctypes.byref(h), n, P, I, O, S.ctypes.data_as(_I64P), int(tb),
                                         int(tile_shape)), "stencil_batch_create_ex")
    return h.value


def stencil_batch_launch(batch: int, stream: int = 0):
    _check(lib().stencil_batch_launch(batch, stream), "stencil_batch_launch")


def stencil_batch_info(batch: int) -> dict:
    info = stencil_batch_info_t()
    _check(lib().stencil_batch_info(batch, ctypes.byref(info)), "stencil_batch_info")
    return {f: getattr(info, f) for f, _ in info._fields_}


def stencil_batch_destroy(batch: int):
    _check(lib().stencil_batch_destroy(batch), "stencil_batch_destroy")


def stencil_fill_uniform(d_out: int, dtype, count: int, seed: int, offset: int = 0, lo: float = 0.0,
                         hi: float = 1.0, stream: int = 0):
    dt = DTYPES[dtype] if isinstance(dtype, str) else int(dtype)
    _check(lib().stencil_fill_uniform(d_out, dt, int(count), int(seed) & 0xFFFFFFFFFFFFFFFF, int(offset),
                                      float(lo), float(hi), stream), "stencil_fill_uniform")


def stencil_server_create(budget_bytes: int, max_resident: int = 64, quantum_steps: int = 16,
                          nstreams: int = 8) -> int:
    h = _P()
    _check(lib().stencil_server_create(ctypes.byref(h), int(budget_bytes), int(max_resident), int(quantum_steps),
                                       int(nstreams)), "stencil_server_create")
    return h.value


def make_request(shape, radius, kind, coeffs, dtype, steps, bc="dirichlet", impl="auto", h_in=None,
                 seed=0, lo=0.0, hi=1.0):
    """A stencil_request plus the Python objects its pointers refer to (keep both alive)."""
    c = np.ascontiguousarray(coeffs, dtype=np.float64)
    rq = stencil_request()
    rq.ndim = len(shape)
    rq.radius = int(radius)
    rq.kind = KINDS[kind] if isinstance(kind, str) else int(kind)
    rq.dtype = DTYPES[dtype] if isinstance(dtype, str) else int(dtype)
    rq.bc = BCS[bc] if isinstance(bc, str) else int(bc)
    rq.impl = IMPLS[impl] if isinstance(impl, str) else int(impl)
    for d, n in enumerate(shape):
        rq.shape[d] = int(n)
    rq.coeffs = _dp(c)
    rq.h_in = h_in.ctypes.data if h_in is not None else None
    rq.seed = int(seed) & 0xFFFFFFFFFFFFFFFF
    rq.lo = float(lo)
    rq.hi = float(hi)
    rq.steps = int(steps)
    return rq, (c, h_in)


def stencil_server_submit(server: int, rq: stencil_request) -> int:
    i = ctypes.c_uint64()
    _check(lib().stencil_server_submit(server, ctypes.byref(rq), ctypes.byref(i)), "stencil_server_submit")
    return i.value


def stencil_server_poll(server: int, rid: int) -> int:
    return int(lib().stencil_server_poll(server, rid))


def stencil_server_wait(server: int, rid: int, timeout_ms: int = -1) -> int:
    return int(lib().stencil_server_wait(server, rid, int(timeout_ms)))


def stencil_server_result(server: int, rid: int, h_out: Optional[np.ndarray] = None) -> dict:
    st = stencil_request_stats()
    _check(lib().stencil_server_result(server, rid, h_out.ctypes.data if h_out is not None else None,
                                       ctypes.byref(st)), "stencil_server_result")
    return {f: getattr(st, f) for f, _ in st._fields_}


def stencil_server_stats(server: int) -> dict:
    st = stencil_server_stats_t()
    _check(lib().stencil_server_stats(server, ctypes.byref(st)), "stencil_server_stats")
    return {f: getattr(st, f) for f, _ in st._fields_}


def stencil_server_destroy(server: int):
    _check(lib().stencil_server_destroy(server), "stencil_server_destroy")


def stencil_error_norms(d_got: int, got_dtype, d_ref: int, count: int, stream: int = 0) -> np.ndarray:
    out = np.zeros(4)
    dt = DTYPES[got_dtype] if isinstance(got_dtype, str) else int(got_dtype)
    _check(lib().stencil_error_norms(d_got, dt, d_ref, int(count), _dp(out), stream), "stencil_error_norms")
    return out


def stencil_band_operand(radius: int, line: np.ndarray, n: int, pad: int) -> np.ndarray:
    w = np.ascontiguousarray(line, dtype=np.float64)
    out = np.zeros((n + 2 * pad, n))
    _check(lib().stencil_band_operand(int(radius), _dp(w), int(n), int(pad), _dp(out)), "stencil_band_operand")
    return out


def stencil_line_cover(ndim: int, radius: int, kind, option: int, n: int):
    nl = ctypes.c_int32()
    ops = ctypes.c_int64()
    k = KINDS[kind] if isinstance(kind, str) else int(kind)
    _check(lib().stencil_line_cover(ndim, radius, k, option, n, ctypes.byref(nl), ctypes.byref(ops)),
           "stencil_line_cover")
    return nl.value, ops.value


def stencil_min_line_cover(mask):
    """(number of lines, rows, cols) of a minimal axis-parallel line cover of
    the n x n weight pattern ``mask`` (nonzero = weight present)."""
    m = np.ascontiguousarray(np.asarray(mask) != 0, dtype=np.uint8)
    if m.ndim != 2 or m.shape[0] != m.shape[1]:
        raise ValueError("mask must be square")
    n = m.shape[0]
    rows = np.zeros(n, dtype=np.int32)
    cols = np.zeros(n, dtype=np.int32)
    count = ctypes.c_int32()
    _check(lib().stencil_min_line_cover(n, m.ctypes.data, rows.ctypes.data, cols.ctypes.data, ctypes.byref(count)),
           "stencil_min_line_cover")
    return count.value, rows.astype(bool), cols.astype(bool)


# ---------------------------------------------------------------- torch helper
class Plan:
    """A plan for torch CUDA tensors of the plan's dtype and shape."""

    def __init__(self, shape, radius, kind, coeffs, dtype="f32", bc="dirichlet", impl="auto",
                 prec="native", tb=0, cover="auto", pitch=0, unit_planes=0):
        self.shape = tuple(int(s) for s in shape)
        self.dtype = dtype
        self.handle = stencil_plan_create(self.shape, radius, kind, coeffs, dtype,
                                          make_options(prec, bc, impl, tb, cover, pitch, unit_planes))
        self.info = stencil_plan_info(self.handle)

    def apply(self, x, out=None, steps=1, stream=None):
        import torch
        if out is None:
            out = torch.empty_like(x)
        self._check_tensor(x)
        self._check_tensor(out)
        s = stream if stream is not None else torch.cuda.current_stream(x.device)
        stencil_apply(self.handle, x.data_ptr(), out.data_ptr(), steps, s.cuda_stream)
        return out

    def _check_tensor(self, t):
        import torch
        want = torch.float32 if self.dtype == "f32" else torch.float64
        if not t.is_cuda or t.dtype != want or tuple(t.shape) != self.shape or not t.is_contiguous():
            raise ValueError(f"expected a contiguous CUDA {want} tensor of shape {self.shape}")

    def close(self):
        if self.handle:
            stencil_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
