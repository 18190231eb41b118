"""ctypes binding of the C ABI in include/gbfft.h -- argument marshalling only.

Every function keeps its C name. The library is the in-tree
``paper_2601_12209_gb300/lib/libgbfft.so`` built by ``_build.build()``; if it
is missing, loading raises instead of falling back to anything else.
"""
from __future__ import annotations

import ctypes
import os
import threading

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "lib", "libgbfft.so")

# constants mirrored from include/gbfft.h
GBFFT_C2C = 0
GBFFT_R2C = 1
GBFFT_FP32 = 0
GBFFT_FP16_SPLIT_TC5 = 3
GBFFT_BF16_SPLIT_TC5 = 4
GBFFT_FP16_SPLIT = 1
GBFFT_BF16_SPLIT = 2
GBFFT_PENCIL = 0
GBFFT_SLAB = 1
GBFFT_TRANSPOSED_OUT = 2
GBFFT_STAGED = 4
GBFFT_NO_TMA = 8
GBFFT_DEBUG_TIMEOUT = 1 << 16
GBFFT_OP_FORWARD = 0
GBFFT_OP_INVERSE = 1
GBFFT_OP_ADJOINT = 2
GBFFT_OP_INVERSE_ADJOINT = 3
GBFFT_OP_POISSON = 4  # gbfft_exec_host only
GBFFT_OP_POISSON_BOUNDED = 5  # gbfft_exec_host only
GBFFT_R2R_NONE = -1
GBFFT_R2R_DCT = 0
GBFFT_R2R_DST = 1
GBFFT_OK = 0
GBFFT_ERR_INVALID_ARG = -1
GBFFT_ERR_UNSUPPORTED_SIZE = -2
GBFFT_ERR_ALIGNMENT = -3
GBFFT_ERR_INPLACE = -4
GBFFT_ERR_ALLOC = -5
GBFFT_ERR_CUDA = -6
GBFFT_ERR_TIMEOUT = -7
GBFFT_ERR_NO_DEVICE = -8
GBFFT_ERR_STATIC_LIMIT = -9
GBFFT_ERR_SETUP_IN_CAPTURE = -10
GBFFT_NOALLOC_MAX_POINTS = 4194304

# every symbol include/gbfft.h declares
EXPORTED = (
    "gbfft_plan_create", "gbfft_plan_get_cached", "gbfft_plan_cache_clear", "gbfft_exec",
    "gbfft_exec_forward", "gbfft_exec_inverse", "gbfft_exec_adjoint", "gbfft_exec_inverse_adjoint",
    "gbfft_exec_poisson", "gbfft_exec_poisson_bounded", "gbfft_exec_r2r_z", "gbfft_exec_r2r", "gbfft_exec_host", "gbfft_workspace_size", "gbfft_set_workspace",
    "gbfft_get_device_error", "gbfft_debug_run", "gbfft_strerror", "gbfft_plan_destroy",
    "gbfft_supported_length", "gbfft_radix_plan", "gbfft_version", "gbfft_exec_c2c_noalloc",
    "gbfft_plan_autotune", "gbfft_plan_get_tuning", "gbfft_plan_time_stages", "gbfft_plan_stage_times",
    "gbfft_plan_set_tuning", "gbfft_many_create", "gbfft_many_layout", "gbfft_many_exec",
    "gbfft_many_exec_separate", "gbfft_many_get_device_error", "gbfft_many_destroy", "gbfft_many_exec_staged",
    "gbfft_plan_set_host_chunks", "gbfft_many_autotune", "gbfft_many_get_tuning", "gbfft_many_set_tuning", "gbfft_many_get_lag",
    "gbfft_many_set_lag",
)

_lib = None
_lock = threading.Lock()


class GbfftError(RuntimeError):
    def __init__(self, code: int, what: str):
        self.code = code
        super().__init__(f"{what} failed: {strerror(code)} ({code})")


def load() -> ctypes.CDLL:
    """Open libgbfft.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libgbfft.so is not built ({LIB_PATH}); run "
                               "paper_2601_12209_gb300._build.build() or __graft_entry__.build()")
        lib = ctypes.CDLL(LIB_PATH)
        vp, i, u, sz = ctypes.c_void_p, ctypes.c_int, ctypes.c_uint, ctypes.c_size_t
        plan_p = ctypes.POINTER(ctypes.c_void_p)
        sig = {
            "gbfft_plan_create": (i, [plan_p, i, i, i, i, i, i, u]),
            "gbfft_plan_get_cached": (i, [plan_p, i, i, i, i, i, i, u]),
            "gbfft_plan_cache_clear": (None, []),
            "gbfft_exec": (i, [vp, i, vp, vp, vp]),
            "gbfft_exec_forward": (i, [vp, vp, vp, vp]),
            "gbfft_exec_inverse": (i, [vp, vp, vp, vp]),
            "gbfft_exec_adjoint": (i, [vp, vp, vp, vp]),
            "gbfft_exec_inverse_adjoint": (i, [vp, vp, vp, vp]),
            "gbfft_exec_poisson": (i, [vp, vp, vp, vp]),
            "gbfft_exec_poisson_bounded": (i, [vp, vp, vp, vp]),
            "gbfft_exec_r2r_z": (i, [vp, i, i, vp, vp, vp]),
            "gbfft_exec_r2r": (i, [vp, i, i, i, i, vp, vp, vp]),
            "gbfft_exec_host": (i, [vp, i, vp, vp]),
            "gbfft_workspace_size": (i, [vp, ctypes.POINTER(sz)]),
            "gbfft_set_workspace": (i, [vp, vp, sz]),
            "gbfft_get_device_error": (i, [vp, ctypes.POINTER(i)]),
            "gbfft_debug_run": (i, [vp, i, vp, vp, vp]),
            "gbfft_strerror": (ctypes.c_char_p, [i]),
            "gbfft_plan_destroy": (None, [vp]),
            "gbfft_supported_length": (i, [i]),
            "gbfft_radix_plan": (i, [i, ctypes.POINTER(i), i]),
            "gbfft_version": (ctypes.c_char_p, []),
            "gbfft_exec_c2c_noalloc": (i, [i, i, i, i, vp, vp, vp]),
            "gbfft_plan_autotune": (i, [vp, vp]),
            "gbfft_plan_get_tuning": (i, [vp, i, ctypes.POINTER(i), ctypes.POINTER(i), ctypes.POINTER(u),
                                          ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_float)]),
            "gbfft_plan_time_stages": (i, [vp, i]),
            "gbfft_plan_set_tuning": (i, [vp, i, i, u]),
            "gbfft_many_create": (i, [plan_p, i, ctypes.POINTER(i), i, i, u]),
            "gbfft_many_autotune": (i, [vp, vp]),
            "gbfft_plan_set_host_chunks": (i, [vp, i]),
            "gbfft_many_get_tuning": (i, [vp, i, ctypes.POINTER(i), ctypes.POINTER(i), i, ctypes.POINTER(i),
                                          ctypes.POINTER(ctypes.c_float)]),
            "gbfft_many_set_tuning": (i, [vp, i, ctypes.POINTER(i), ctypes.POINTER(i), i]),
            "gbfft_many_get_lag": (i, [vp, i, ctypes.POINTER(i)]),
            "gbfft_many_set_lag": (i, [vp, i, i]),
            "gbfft_many_layout": (i, [vp, i, ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(ctypes.c_longlong)]),
            "gbfft_many_exec": (i, [vp, i, vp, vp, vp]),
            "gbfft_many_exec_separate": (i, [vp, i, vp, vp, vp]),
            "gbfft_many_exec_staged": (i, [vp, i, vp, vp, vp]),
            "gbfft_many_get_device_error": (i, [vp, ctypes.POINTER(i)]),
            "gbfft_many_destroy": (None, [vp]),
            "gbfft_plan_stage_times": (i, [vp, i, ctypes.POINTER(ctypes.c_float), ctypes.POINTER(i),
                                           ctypes.POINTER(i)]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def _call(name: str, *args) -> int:
    rc = getattr(load(), name)(*args)
    if rc != GBFFT_OK:
        raise GbfftError(rc, name)
    return rc


def strerror(code: int) -> str:
    return load().gbfft_strerror(int(code)).decode()


def gbfft_version() -> str:
    return load().gbfft_version().decode()


def gbfft_supported_length(n: int) -> bool:
    return bool(load().gbfft_supported_length(int(n)))


def gbfft_radix_plan(n: int) -> list[int]:
    buf = (ctypes.c_int * 16)()
    k = load().gbfft_radix_plan(int(n), buf, 16)
    if k < 0:
        raise GbfftError(k, "gbfft_radix_plan")
    return [buf[j] for j in range(k)]


def gbfft_plan_create(nx, ny, nz, kind=GBFFT_C2C, dtype=GBFFT_FP32, batch=1, flags=0) -> int:
    h = ctypes.c_void_p()
    _call("gbfft_plan_create", ctypes.byref(h), int(nx), int(ny), int(nz), int(kind), int(dtype), int(batch),
          int(flags))
    return h.value


def gbfft_plan_get_cached(nx, ny, nz, kind=GBFFT_C2C, dtype=GBFFT_FP32, batch=1, flags=0) -> int:
    h = ctypes.c_void_p()
    _call("gbfft_plan_get_cached", ctypes.byref(h), int(nx), int(ny), int(nz), int(kind), int(dtype), int(batch),
          int(flags))
    return h.value


def gbfft_plan_cache_clear() -> None:
    load().gbfft_plan_cache_clear()


def gbfft_plan_destroy(plan: int) -> None:
    load().gbfft_plan_destroy(ctypes.c_void_p(plan))


def gbfft_exec(plan: int, op: int, in_ptr: int, out_ptr: int, stream: int = 0) -> None:
    _call("gbfft_exec", ctypes.c_void_p(plan), int(op), ctypes.c_void_p(in_ptr), ctypes.c_void_p(out_ptr),
          ctypes.c_void_p(stream))


def gbfft_exec_forward(plan, in_ptr, out_ptr, stream=0):
    _call("gbfft_exec_forward", ctypes.c_void_p(plan), ctypes.c_void_p(in_ptr), ctypes.c_void_p(out_ptr),
          ctypes.c_void_p(stream))


def gbfft_exec_inverse(plan, in_ptr, out_ptr, stream=0):
    _call("gbfft_exec_inverse", ctypes.c_void_p(plan), ctypes.c_void_p(in_ptr), ctypes.c_void_p(out_ptr),
          ctypes.c_void_p(stream))


def gbfft_exec_adjoint(plan, in_ptr, out_ptr, stream=0):
    _call("gbfft_exec_adjoint", ctypes.c_void_p(plan), ctypes.c_void_p(in_ptr), ctypes.c_void_p(out_ptr),
          ctypes.c_void_p(stream))


def gbfft_exec_inverse_adjoint(plan, in_ptr, out_ptr, stream=0):
    _call("gbfft_exec_inverse_adjoint", ctypes.c_void_p(plan), ctypes.c_void_p(in_ptr), ctypes.c_void_p(out_ptr),
          ctypes.c_void_p(stream))


def gbfft_exec_poisson(plan, in_ptr, out_ptr, stream=0):
    _call("gbfft_exec_poisson", ctypes.c_void_p(plan), ctypes.c_void_p(in_ptr), ctypes.c_void_p(out_ptr),
          ctypes.c_void_p(stream))


def gbfft_exec_r2r(plan, r2r_x, r2r_y, r2r_z, inverse, in_ptr, out_ptr, stream=0):
    _call("gbfft_exec_r2r", ctypes.c_void_p(plan), int(r2r_x), int(r2r_y), int(r2r_z), int(bool(inverse)),
          ctypes.c_void_p(in_ptr), ctypes.c_void_p(out_ptr), ctypes.c_void_p(stream))


def gbfft_exec_r2r_z(plan, r2r, inverse, in_ptr, out_ptr, stream=0):
    _call("gbfft_exec_r2r_z", ctypes.c_void_p(plan), int(r2r), int(bool(inverse)), ctypes.c_void_p(in_ptr),
          ctypes.c_void_p(out_ptr), ctypes.c_void_p(stream))


def gbfft_exec_poisson_bounded(plan, in_ptr, out_ptr, stream=0):
    _call("gbfft_exec_poisson_bounded", ctypes.c_void_p(plan), ctypes.c_void_p(in_ptr), ctypes.c_void_p(out_ptr),
          ctypes.c_void_p(stream))


def gbfft_exec_host(plan: int, op: int, host_in: int, host_out: int) -> None:
    _call("gbfft_exec_host", ctypes.c_void_p(plan), int(op), ctypes.c_void_p(host_in), ctypes.c_void_p(host_out))


def gbfft_workspace_size(plan: int) -> int:
    n = ctypes.c_size_t()
    _call("gbfft_workspace_size", ctypes.c_void_p(plan), ctypes.byref(n))
    return n.value


def gbfft_set_workspace(plan: int, ptr: int, nbytes: int) -> None:
    _call("gbfft_set_workspace", ctypes.c_void_p(plan), ctypes.c_void_p(ptr), ctypes.c_size_t(nbytes))


def gbfft_get_device_error(plan: int) -> int:
    c = ctypes.c_int()
    _call("gbfft_get_device_error", ctypes.c_void_p(plan), ctypes.byref(c))
    return c.value


def gbfft_debug_run(plan: int, step: int, in_ptr: int, out_ptr: int, stream: int = 0) -> None:
    _call("gbfft_debug_run", ctypes.c_void_p(plan), int(step), ctypes.c_void_p(in_ptr), ctypes.c_void_p(out_ptr),
          ctypes.c_void_p(stream))


def gbfft_exec_c2c_noalloc(nx: int, ny: int, nz: int, op: int, in_ptr: int, out_ptr: int, stream: int = 0) -> None:
    """Allocation-free C2C transform on one grid; see include/gbfft.h."""
    _call("gbfft_exec_c2c_noalloc", int(nx), int(ny), int(nz), int(op), ctypes.c_void_p(in_ptr),
          ctypes.c_void_p(out_ptr), ctypes.c_void_p(stream))


def gbfft_plan_autotune(plan: int, stream: int = 0) -> None:
    _call("gbfft_plan_autotune", ctypes.c_void_p(plan), ctypes.c_void_p(stream))


def gbfft_plan_get_tuning(plan: int, pipeline: int) -> dict:
    tuned, pers = ctypes.c_int(), ctypes.c_int()
    mask = ctypes.c_uint()
    ms = ctypes.c_float()
    stage = (ctypes.c_float * 5)()
    _call("gbfft_plan_get_tuning", ctypes.c_void_p(plan), int(pipeline), ctypes.byref(tuned), ctypes.byref(pers),
          ctypes.byref(mask), ctypes.byref(ms), stage)
    return {"tuned": bool(tuned.value), "persistent": bool(pers.value), "tma_mask": mask.value, "ms": ms.value,
            "stage_ms": [stage[k] for k in range(5)]}


def gbfft_plan_set_tuning(plan: int, pipeline: int, persistent: bool, tma_mask: int) -> None:
    _call("gbfft_plan_set_tuning", ctypes.c_void_p(plan), int(pipeline), int(bool(persistent)), int(tma_mask))


def gbfft_plan_time_stages(plan: int, enable: bool) -> None:
    _call("gbfft_plan_time_stages", ctypes.c_void_p(plan), int(bool(enable)))


def gbfft_plan_stage_times(plan: int, pipeline: int) -> tuple[list[float], int]:
    avg = (ctypes.c_float * 5)()
    nseg, ncalls = ctypes.c_int(), ctypes.c_int()
    _call("gbfft_plan_stage_times", ctypes.c_void_p(plan), int(pipeline), avg, ctypes.byref(nseg),
          ctypes.byref(ncalls))
    return [avg[k] for k in range(nseg.value)], ncalls.value


def gbfft_many_create(shapes, flags: int = 0, kind: int = GBFFT_C2C, dtype: int = GBFFT_FP32) -> int:
    """shapes: list of (nx, ny, nz)."""
    dims = (ctypes.c_int * (3 * len(shapes)))(*[int(v) for sh in shapes for v in sh])
    h = ctypes.c_void_p()
    _call("gbfft_many_create", ctypes.byref(h), len(shapes), dims, int(kind), int(dtype), int(flags))
    return h.value


def gbfft_plan_set_host_chunks(plan: int, chunks: int) -> None:
    _call("gbfft_plan_set_host_chunks", ctypes.c_void_p(plan), int(chunks))


def gbfft_many_autotune(m: int, stream: int = 0) -> None:
    _call("gbfft_many_autotune", ctypes.c_void_p(m), ctypes.c_void_p(stream))


def gbfft_many_get_tuning(m: int, pipeline: int) -> dict:
    """{"teams": {length: tiles per ticket}, "ms": tuned one-launch time (0 if untuned)}."""
    cap = 64
    lens, teams = (ctypes.c_int * cap)(), (ctypes.c_int * cap)()
    n, ms = ctypes.c_int(), ctypes.c_float()
    _call("gbfft_many_get_tuning", ctypes.c_void_p(m), int(pipeline), lens, teams, cap, ctypes.byref(n),
          ctypes.byref(ms))
    return {"teams": {int(lens[i]): int(teams[i]) for i in range(min(n.value, cap))}, "ms": ms.value}


def gbfft_many_get_lag(m: int, pipeline: int) -> int:
    v = ctypes.c_int()
    _call("gbfft_many_get_lag", ctypes.c_void_p(m), int(pipeline), ctypes.byref(v))
    return v.value


def gbfft_many_set_lag(m: int, pipeline: int, lag: int) -> None:
    _call("gbfft_many_set_lag", ctypes.c_void_p(m), int(pipeline), int(lag))


def gbfft_many_set_tuning(m: int, pipeline: int, teams: dict) -> None:
    """teams: {length: tiles per ticket (1, 2 or 4)}."""
    n = len(teams)
    lens = (ctypes.c_int * max(n, 1))(*[int(k) for k in teams])
    ts = (ctypes.c_int * max(n, 1))(*[int(v) for v in teams.values()])
    _call("gbfft_many_set_tuning", ctypes.c_void_p(m), int(pipeline), lens, ts, n)


def gbfft_many_layout(m: int, grid: int) -> tuple[int, int]:
    off, tot = ctypes.c_longlong(), ctypes.c_longlong()
    _call("gbfft_many_layout", ctypes.c_void_p(m), int(grid), ctypes.byref(off), ctypes.byref(tot))
    return off.value, tot.value


def gbfft_many_exec(m: int, op: int, in_ptr: int, out_ptr: int, stream: int = 0) -> None:
    _call("gbfft_many_exec", ctypes.c_void_p(m), int(op), ctypes.c_void_p(in_ptr), ctypes.c_void_p(out_ptr),
          ctypes.c_void_p(stream))


def gbfft_many_exec_staged(m: int, op: int, in_ptr: int, out_ptr: int, stream: int = 0) -> None:
    _call("gbfft_many_exec_staged", ctypes.c_void_p(m), int(op), ctypes.c_void_p(in_ptr), ctypes.c_void_p(out_ptr),
          ctypes.c_void_p(stream))


def gbfft_many_exec_separate(m: int, op: int, in_ptr: int, out_ptr: int, stream: int = 0) -> None:
    _call("gbfft_many_exec_separate", ctypes.c_void_p(m), int(op), ctypes.c_void_p(in_ptr),
          ctypes.c_void_p(out_ptr), ctypes.c_void_p(stream))


def gbfft_many_get_device_error(m: int) -> int:
    c = ctypes.c_int()
    _call("gbfft_many_get_device_error", ctypes.c_void_p(m), ctypes.byref(c))
    return c.value


def gbfft_many_destroy(m: int) -> None:
    load().gbfft_many_destroy(ctypes.c_void_p(m))


def raw_rc(name: str, *args) -> int:
    """Call a C function and return its code without raising (for error-path tests)."""
    return getattr(load(), name)(*args)
