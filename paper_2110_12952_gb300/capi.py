"""ctypes declarations of the C ABI in ``include/fractal.h`` (argument
marshalling only: every computation runs in ``libfractal.so``).

The library must have been built (``paper_2110_12952_gb300.build.build()``);
loading fails loudly otherwise.  PyTorch is imported first so that the
library binds to the CUDA runtime already loaded by PyTorch.
"""
from __future__ import annotations

import ctypes
import os
import re
import threading

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libfractal.so")
HEADER = os.path.join(os.path.dirname(_HERE), "include", "fractal.h")

FR_OK = 0
ERRORS = {-1: "FR_EINVAL", -2: "FR_EOVERFLOW", -3: "FR_ENOMEM", -4: "FR_ECUDA",
          -5: "FR_ETIMEOUT", -6: "FR_EBUSY", -7: "FR_ENOTFOUND"}

_lock = threading.Lock()
_lib = None

c_int, c_i32, c_i64, c_u32, c_u64, c_dbl, c_vp = (ctypes.c_int, ctypes.c_int32, ctypes.c_int64,
                                                   ctypes.c_uint32, ctypes.c_uint64, ctypes.c_double,
                                                   ctypes.c_void_p)
c_i32p = ctypes.POINTER(ctypes.c_int32)
c_i64p = ctypes.POINTER(ctypes.c_int64)
c_u8p = ctypes.POINTER(ctypes.c_uint8)
c_fp = ctypes.c_void_p  # fractal_t*

SIGNATURES = {
    "fractal_last_error": (ctypes.c_char_p, []),
    "fractal_version": (ctypes.c_char_p, []),
    "fractal_create": (c_int, [c_int, c_int, c_int, c_int, c_i32p, ctypes.POINTER(c_fp)]),
    "fractal_create_mixed": (c_int, [c_int, c_int, c_int, c_i32p, c_i32p, ctypes.POINTER(c_fp)]),
    "fractal_destroy": (c_int, [c_fp]),
    "fractal_info": (c_int, [c_fp, c_i64p, c_i64p]),
    "fractal_lambda": (c_int, [c_fp, c_vp, c_i64, c_vp, c_vp]),
    "fractal_nu": (c_int, [c_fp, c_vp, c_i64, c_vp, c_vp]),
    "fractal_nu2d": (c_int, [c_fp, c_vp, c_i64, c_vp, c_vp]),
    "fractal_init_bernoulli": (c_int, [c_fp, c_vp, c_u64, c_dbl, c_vp]),
    "fractal_step": (c_int, [c_fp, c_vp, c_vp, c_i64, c_u32, c_u32, c_vp]),
    "fractal_bb_step": (c_int, [c_fp, c_vp, c_vp, c_i64, c_u32, c_u32, c_vp]),
    "fractal_scatter_to_box": (c_int, [c_fp, c_vp, c_vp, c_vp]),
    "fractal_gather_from_box": (c_int, [c_fp, c_vp, c_vp, c_vp]),
    "fractal_run_host": (c_int, [c_fp, c_vp, c_vp, c_i64, c_u32, c_u32, c_vp]),
    "fractal_set_tile_levels": (c_int, [c_fp, c_int]),
    "fractal_get_tile_levels": (c_int, [c_fp, ctypes.POINTER(c_int)]),
    "fractal_plan_info": (c_int, [c_fp, ctypes.POINTER(ctypes.c_int32), c_int]),
    "fractal_sync": (c_int, [c_vp]),
    "fractal_check": (c_int, [c_fp]),
    "fractal_step_noalloc": (c_int, [c_fp, c_vp, c_vp, c_i64, c_u32, c_u32, c_vp]),
    "fractal_batch_create": (c_int, [ctypes.POINTER(c_vp)]),
    "fractal_batch_destroy": (c_int, [c_vp]),
    "fractal_batch_add": (c_int, [c_vp, c_fp, c_vp, c_vp, c_i64, c_u32, c_u32, c_i64p]),
    "fractal_batch_clear": (c_int, [c_vp]),
    "fractal_batch_run": (c_int, [c_vp, c_vp]),
    "fractal_batch_stats": (c_int, [c_vp, c_i64p, c_i64p]),
    "fractal_server_create": (c_int, [c_i64, c_int, ctypes.POINTER(c_vp)]),
    "fractal_server_destroy": (c_int, [c_vp]),
    "fractal_server_submit": (c_int, [c_vp, c_fp, c_u64, c_dbl, c_i64, c_u32, c_u32, c_vp, c_i64p]),
    "fractal_server_poll": (c_int, [c_vp, c_i64, ctypes.POINTER(c_int), ctypes.POINTER(c_dbl), c_i64p]),
    "fractal_server_wait_all": (c_int, [c_vp]),
    "fractal_server_stats": (c_int, [c_vp, c_i64p, c_i64p, c_i64p, c_i64p, c_i64p, c_i64p]),
    "fractal_autotune": (c_int, [c_fp, c_vp, c_vp, c_u32, c_u32, c_vp, ctypes.POINTER(c_int)]),
    "fractal_test_arm_timeout": (c_int, [c_fp, c_u32, c_u32]),
    "fractal_set_pipeline_stages": (c_int, [c_fp, c_int]),
    "fractal_nu_tc": (c_int, [c_fp, c_vp, c_i64, c_vp, c_vp, c_vp]),
    "fractal_set_temporal_blocking": (c_int, [c_fp, c_int, c_int]),
    "fractal_lambda_box_step": (c_int, [c_fp, c_int, c_vp, c_vp, c_i64, c_u32, c_u32, c_vp]),
    "fractal_blocked_info": (c_int, [c_fp, c_int, c_i64p]),
    "fractal_blocked_pack": (c_int, [c_fp, c_int, c_vp, c_vp, c_vp]),
    "fractal_blocked_unpack": (c_int, [c_fp, c_int, c_vp, c_vp, c_vp]),
    "fractal_blocked_step": (c_int, [c_fp, c_int, c_vp, c_vp, c_i64, c_u32, c_u32, c_vp]),
    "fractal_lambda_tc": (c_int, [c_fp, c_vp, c_i64, c_vp, c_vp]),
    "fractal_shard_plan": (c_int, [c_int, c_int, c_int, c_int, c_i32p, c_int, c_int, c_int, ctypes.POINTER(c_vp)]),
    "fractal_shard_destroy": (c_int, [c_vp]),
    "fractal_shard_info": (c_int, [c_vp, c_i64p, c_i64p, c_i64p]),
    "fractal_shard_sends": (c_int, [c_vp, c_int, c_i64p, c_i64, c_i64p, c_i64p]),
    "fractal_shard_recvs": (c_int, [c_vp, c_int, c_i64p, c_i64, c_i64p, c_i64p]),
    "fractal_shard_neighbours": (c_int, [c_vp, c_i32p, c_i64]),
    "fractal_shard_attach": (c_int, [c_vp, c_fp]),
    "fractal_shard_pack": (c_int, [c_vp, c_int, c_vp, c_vp, c_vp]),
    "fractal_shard_step": (c_int, [c_vp, c_vp, c_vp, c_u32, c_u32, c_vp]),
}


class FractalError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


def header_functions() -> list[str]:
    """Names of the functions declared in include/fractal.h."""
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(fractal_[a-z0-9_]+)\s*\(", text)))


def load(path: str | None = None):
    """Load libfractal.so (raises if it is missing: there is no fallback)."""
    global _lib
    with _lock:
        if _lib is not None and path is None:
            return _lib
        import torch  # noqa: F401  (binds the CUDA runtime PyTorch loaded)
        p = path or LIB_PATH
        if not os.path.exists(p):
            raise RuntimeError(f"{p} is missing: build it with paper_2110_12952_gb300.build.build()")
        lib = ctypes.CDLL(p)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        if path is None:
            _lib = lib
        return lib


def check(rc: int, lib=None):
    if rc != FR_OK:
        lib = lib or load()
        raise FractalError(rc, lib.fractal_last_error().decode())
    return rc
