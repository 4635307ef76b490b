"""ctypes declarations of the C ABI in include/gemm.h.  Loading fails loudly
when the compiled library is missing: there is no fallback path."""
from __future__ import annotations

import ctypes
import os
import threading

from . import build as _build

_lock = threading.Lock()
_lib = None

i64 = ctypes.c_int64
i32 = ctypes.c_int
f32 = ctypes.c_float
vp = ctypes.c_void_p
cp = ctypes.c_char_p
u64 = ctypes.c_uint64

STATUS_NAMES = {
    0: "GEMM_OK", 1: "GEMM_ERR_INVALID_ARG", 2: "GEMM_ERR_ALIGNMENT", 3: "GEMM_ERR_ALLOC",
    4: "GEMM_ERR_CUDA", 5: "GEMM_ERR_UNSUPPORTED_DEVICE", 6: "GEMM_ERR_TIMEOUT", 7: "GEMM_ERR_IO",
}


class GemmConfig(ctypes.Structure):
    _fields_ = [("block_n", i32), ("stages", i32), ("split_k", i32), ("kb", i32), ("group_m", i32),
                ("fused", i32), ("cluster", i32)]


# name -> (restype, argtypes); mirrors include/gemm.h one to one
SIGNATURES = {
    "gemm_f32": (i32, [i64, i64, i64, f32, vp, i64, vp, i64, f32, vp, i64]),
    "gemm_f32_ex": (i32, [i64, i64, i64, f32, vp, i64, vp, i64, f32, vp, i64, i32, i32, vp]),
    "gemm_f32_host": (i32, [i64, i64, i64, f32, vp, i64, vp, i64, f32, vp, i64, i32, vp]),
    "gemm_plan_create": (i32, [i64, i64, i64, i64, i64, i64, i32, i32, ctypes.POINTER(vp)]),
    "gemm_plan_create_config": (i32, [i64, i64, i64, i64, i64, i64, i32, i32, ctypes.POINTER(vp)]),
    "gemm_plan_create_opts": (i32, [i64, i64, i64, i64, i64, i64, i32, i32, i32, ctypes.c_uint,
                                    ctypes.POINTER(vp)]),
    "gemm_conv_plan_create": (i32, [i64, i64, i64, i64, i64, i32, i32, i32, i32, ctypes.POINTER(vp)]),
    "gemm_conv3x3_plan_create": (i32, [i64, i64, i64, i64, i64, i32, i32, ctypes.POINTER(vp)]),
    "gemm_plan_create_t": (i32, [i32, i32, i64, i64, i64, i64, i64, i64, i32, i32, ctypes.POINTER(vp)]),
    "gemm_f32_t": (i32, [i32, i32, i64, i64, i64, f32, vp, i64, vp, i64, f32, vp, i64, i32, i32, vp]),
    "gemm_plan_execute": (i32, [vp, f32, vp, vp, f32, vp, vp]),
    "gemm_plan_info": (i32, [vp, ctypes.POINTER(i32), ctypes.POINTER(i32), ctypes.POINTER(ctypes.c_size_t)]),
    "gemm_plan_destroy": (i32, [vp]),
    "gemm_plan_profile": (i32, [vp, i32]),
    "gemm_plan_profile_read": (i32, [vp, ctypes.POINTER(i32), ctypes.POINTER(f32),
                                     ctypes.POINTER(f32), ctypes.POINTER(f32)]),
    "gemm_config_count": (i32, [i32]),
    "gemm_config_get": (i32, [i32, i32, ctypes.POINTER(GemmConfig)]),
    "gemm_config_default": (i32, [i32, i64, i64, i64]),
    "gemm_last_error": (cp, []),
    "gemm_device_error": (i32, []),
    "gemm_device_sm_count": (i32, []),
    "gemm_selftest_wait_timeout": (i32, []),
    "gemm_split_pack": (i32, [i32, i32, i64, i64, vp, i64, vp, i64, vp, vp]),
    "gemm_f32_bf16x3_noalloc": (i32, [i64, i64, i64, f32, vp, i64, vp, i64, f32, vp, i64, vp]),
    "gemm_grouped_plan_create": (i32, [i32, vp, vp, vp, vp, vp, vp, i32, i32, ctypes.POINTER(vp)]),
    "gemm_grouped_plan_create_config": (i32, [i32, vp, vp, vp, vp, vp, vp, i32, i32, i32,
                                              ctypes.POINTER(vp)]),
    "gemm_grouped_execute": (i32, [vp, vp, vp, vp, vp, vp, vp]),
    "gemm_grouped_execute_eager": (i32, [vp, vp, vp, vp, vp, vp, vp]),
    "gemm_grouped_plan_info": (i32, [vp, ctypes.POINTER(i32), ctypes.POINTER(i32),
                                     ctypes.POINTER(i32), ctypes.POINTER(ctypes.c_size_t)]),
    "gemm_grouped_plan_destroy": (i32, [vp]),
    "gemm_autotune": (i32, [vp, i32, i32, i32, cp]),
    "gemm_autotune_load": (i32, [cp]),
    "gemm_autotune_best": (i32, [i64, i64, i64, i64, i64, i64, i32, ctypes.POINTER(i32),
                                 ctypes.POINTER(f32)]),
    "gemm_select_config": (i32, [i64, i64, i64, i64, i64, i64, i32, i32, ctypes.POINTER(i32)]),
    "gemm_costmodel_feature_count": (i32, []),
    "gemm_costmodel_features": (i32, [i64, i64, i64, i32, i32, i32, vp]),
    "gemm_costmodel_train": (i32, [cp, i32, u64, cp, ctypes.POINTER(f32)]),
    "gemm_costmodel_load": (i32, [cp]),
    "gemm_costmodel_predict": (i32, [i64, i64, i64, i32, ctypes.POINTER(i32), ctypes.POINTER(f32)]),
    "gemm_mlp_loss_grad": (i32, [i32, vp, vp, vp, ctypes.POINTER(f32), vp]),
    "gemm_mlp_adam_step": (i32, [i32, vp, vp, vp, vp, i32, f32, f32, f32, f32]),
}


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load (building first if needed) the CUDA library."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.LIB
        if not os.path.exists(path) or not _build.up_to_date():
            if not build_if_missing:
                raise RuntimeError(f"CUDA library not built: {path}")
            _build.build()
        lib = ctypes.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


class GemmError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


def check(status: int) -> None:
    if status != 0:
        msg = load().gemm_last_error()
        raise GemmError(status, msg.decode() if msg else "")
