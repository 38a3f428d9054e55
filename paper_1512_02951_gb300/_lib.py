"""ctypes declarations of the C ABI in include/fds.h (argument marshalling only)."""
from __future__ import annotations

import ctypes
import os
import threading

from . import build as _build

FDS_OK = 0
FDS_E_INVALID = -1
FDS_E_NO_KEY = -2
FDS_E_NOMEM = -3
FDS_E_CUDA = -4
FDS_E_TIMEOUT = -5
FDS_E_BUSY = -6
FDS_MAX_KEYS = 256
FDS_NOALLOC_MAX_IMAGES = 4096
FDS_TC_BF16 = 0
FDS_TC_TF32 = 1
FDS_TC_F16 = 2
FDS_TC_F16_INVERSE = 3
FDS_PACK_11 = 11
FDS_PACK_8 = 8

_c_u8p = ctypes.POINTER(ctypes.c_uint8)


class FdsImage(ctypes.Structure):
    """struct fds_image of fds.h."""
    _fields_ = [
        ("pixel_offset", ctypes.c_uint64),
        ("public_offset", ctypes.c_uint64),
        ("private_offset", ctypes.c_uint64),
        ("width", ctypes.c_int32),
        ("height", ctypes.c_int32),
        ("k", ctypes.c_int32),
        ("key_slot", ctypes.c_int32),
        ("iv", ctypes.c_uint8 * 16),
    ]


# name -> (restype, argtypes)
SIGNATURES = {
    "fds_init": (ctypes.c_int, [ctypes.c_int]),
    "fds_key_register": (ctypes.c_int, [ctypes.c_char_p, ctypes.POINTER(ctypes.c_int32)]),
    "fds_key_release": (ctypes.c_int, [ctypes.c_int32]),
    "fds_sizes": (ctypes.c_int, [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                 ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_uint64)]),
    "fds_protect_image": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32,
                                         ctypes.c_int32, ctypes.c_char_p, ctypes.c_char_p,
                                         ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "fds_restore_image": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32,
                                         ctypes.c_int32, ctypes.c_int32, ctypes.c_char_p,
                                         ctypes.c_char_p, ctypes.c_void_p, ctypes.c_void_p]),
    "fds_protect": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                   ctypes.POINTER(FdsImage), ctypes.c_int32, ctypes.c_void_p]),
    "fds_restore": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                   ctypes.POINTER(FdsImage), ctypes.c_int32, ctypes.c_void_p]),
    "fds_plan_create": (ctypes.c_int, [ctypes.POINTER(FdsImage), ctypes.c_int32,
                                       ctypes.POINTER(ctypes.c_void_p)]),
    "fds_plan_destroy": (ctypes.c_int, [ctypes.c_void_p]),
    "fds_plan_reserve": (ctypes.c_int, [ctypes.c_int32, ctypes.POINTER(ctypes.c_void_p)]),
    "fds_plan_update": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(FdsImage), ctypes.c_int32,
                                       ctypes.c_void_p]),
    "fds_plan_set_schedule": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32,
                                             ctypes.c_int32]),
    "fds_plan_get_schedule": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int32),
                                             ctypes.POINTER(ctypes.c_int32),
                                             ctypes.POINTER(ctypes.c_int32)]),
    "fds_plan_autotune": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                         ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p]),
    "fds_plan_set_direction_schedule": (ctypes.c_int, [ctypes.c_void_p] + [ctypes.c_int32] * 4),
    "fds_plan_get_direction_schedule": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32]
                                        + [ctypes.POINTER(ctypes.c_int32)] * 3),
    "fds_plan_autotune_directions": (ctypes.c_int, [ctypes.c_void_p] * 5
                                     + [ctypes.c_int32, ctypes.c_void_p]),
    "fds_plan_schedule_json": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_char_p, ctypes.c_int64,
                                              ctypes.POINTER(ctypes.c_int64)]),
    "fds_plan_protect": (ctypes.c_int, [ctypes.c_void_p] * 5),
    "fds_plan_restore": (ctypes.c_int, [ctypes.c_void_p] * 5),
    "fds_plan_protect_graph": (ctypes.c_int, [ctypes.c_void_p] * 5),
    "fds_plan_restore_graph": (ctypes.c_int, [ctypes.c_void_p] * 5),
    "fds_protect_batch_noalloc": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                                 ctypes.POINTER(FdsImage), ctypes.c_int32,
                                                 ctypes.c_void_p]),
    "fds_debug_dct_f32": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32,
                                         ctypes.c_void_p, ctypes.c_void_p]),
    "fds_protect_image_tc": (ctypes.c_int, [ctypes.c_int32, ctypes.c_void_p, ctypes.c_int32,
                                            ctypes.c_int32, ctypes.c_int32, ctypes.c_char_p,
                                            ctypes.c_char_p, ctypes.c_void_p, ctypes.c_void_p,
                                            ctypes.c_void_p]),
    "fds_restore_image_tc": (ctypes.c_int, [ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32,
                                            ctypes.c_int32, ctypes.c_int32, ctypes.c_char_p, ctypes.c_char_p,
                                            ctypes.c_void_p, ctypes.c_void_p]),
    "fds_sizes_packed": (ctypes.c_int, [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                        ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_uint64),
                                        ctypes.POINTER(ctypes.c_uint64)]),
    "fds_protect_image_packed": (ctypes.c_int, [ctypes.c_int32, ctypes.c_void_p, ctypes.c_int32,
                                                ctypes.c_int32, ctypes.c_int32, ctypes.c_char_p,
                                                ctypes.c_char_p, ctypes.c_void_p, ctypes.c_void_p,
                                                ctypes.c_void_p, ctypes.c_void_p]),
    "fds_restore_image_packed": (ctypes.c_int, [ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p,
                                                ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                                ctypes.c_char_p, ctypes.c_char_p, ctypes.c_void_p,
                                                ctypes.c_void_p, ctypes.c_void_p]),
    "fds_encrypt_full": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint64,
                                        ctypes.c_char_p, ctypes.c_char_p, ctypes.c_void_p]),
    "fds_protect_image_host": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32,
                                              ctypes.c_int32, ctypes.c_char_p, ctypes.c_char_p, ctypes.c_void_p,
                                              ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32,
                                              ctypes.c_void_p]),
    "fds_restore_image_host": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                              ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_char_p,
                                              ctypes.c_char_p, ctypes.c_int32, ctypes.c_void_p]),
    "fds_public_image": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                        ctypes.c_void_p, ctypes.c_void_p]),
    "fds_image_stats": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p,
                                       ctypes.c_void_p, ctypes.c_void_p]),
    "fds_sizes_strong": (ctypes.c_int, [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                        ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_uint64),
                                        ctypes.POINTER(ctypes.c_uint64)]),
    "fds_protect_image_strong": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32,
                                                ctypes.c_int32, ctypes.c_char_p, ctypes.c_char_p,
                                                ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                                ctypes.c_void_p]),
    "fds_restore_image_strong": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32,
                                                ctypes.c_int32, ctypes.c_int32, ctypes.c_char_p,
                                                ctypes.c_char_p, ctypes.c_void_p, ctypes.c_void_p,
                                                ctypes.c_void_p]),
    "fds_sha512_constants": (ctypes.c_int, [ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_uint64)]),
    "fds_dwt_sizes": (ctypes.c_int, [ctypes.c_int32, ctypes.c_int32, ctypes.POINTER(ctypes.c_uint64),
                                     ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_uint64)]),
    "fds_dwt_protect": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32, ctypes.c_char_p,
                                       ctypes.c_char_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                       ctypes.c_void_p]),
    "fds_dwt_restore": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32,
                                       ctypes.c_int32, ctypes.c_char_p, ctypes.c_char_p, ctypes.c_void_p,
                                       ctypes.c_void_p]),
    "fds_tc_basis": (ctypes.c_int, [ctypes.c_int32, ctypes.c_void_p, ctypes.c_uint64,
                                    ctypes.POINTER(ctypes.c_double)]),
    "fds_debug_dct_tc": (ctypes.c_int, [ctypes.c_int32, ctypes.c_void_p, ctypes.c_int32,
                                        ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p]),
    "fds_debug_exact_round": (ctypes.c_int, [ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32),
                                             ctypes.c_int32]),
    "fds_counters": (ctypes.c_int, [ctypes.POINTER(ctypes.c_uint64), ctypes.c_int]),
    "fds_sync": (ctypes.c_int, [ctypes.c_void_p]),
    "fds_status_of_failures": (ctypes.c_int, [ctypes.c_uint64, ctypes.c_uint64]),
    "fds_debug_set_counters": (ctypes.c_int, [ctypes.POINTER(ctypes.c_uint64)]),
    "fds_last_error": (ctypes.c_char_p, []),
    "fds_copy_many": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32,
                                     ctypes.c_void_p]),
}

_lock = threading.Lock()
_lib = None


class FdsError(RuntimeError):
    def __init__(self, code: int, where: str, msg: str):
        super().__init__(f"{where} failed ({code}): {msg}")
        self.code = code


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = False) -> ctypes.CDLL:
    """Load libfds.so (the CUDA library).  Raises if it is not built: there is no fallback."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.LIB
        if not os.path.exists(path):
            if not build_if_missing:
                raise RuntimeError(f"{path} is missing: build it with "
                                   "paper_1512_02951_gb300.build.build() (needs nvcc)")
            _build.build()
        lib = ctypes.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def check(rc: int, where: str) -> None:
    if rc != FDS_OK:
        msg = load().fds_last_error()
        raise FdsError(rc, where, msg.decode() if msg else "")
