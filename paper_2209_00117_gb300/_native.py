"""ctypes loader for ``_build/libvd.so`` (the C ABI of ``include/vd.h``).

Argument marshalling only.  There is no fallback: if the library has not been
built, :func:`lib` raises, so nothing can silently run on the CPU.
"""
from __future__ import annotations

import ctypes
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libvd.so")

VD_OK = 0
VD_EINVAL = -1
VD_ENOMEM = -2
VD_ECUDA = -3
VD_ETIMEOUT = -4
VD_EBUSY = -5
VD_ENOTFOUND = -6

_ERRNAMES = {VD_EINVAL: "VD_EINVAL", VD_ENOMEM: "VD_ENOMEM", VD_ECUDA: "VD_ECUDA",
             VD_ETIMEOUT: "VD_ETIMEOUT", VD_EBUSY: "VD_EBUSY", VD_ENOTFOUND: "VD_ENOTFOUND"}

_i32, _i64, _u64, _p, _int = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, ctypes.c_void_p, ctypes.c_int
_P32 = ctypes.POINTER(ctypes.c_int32)
_PU64 = ctypes.POINTER(ctypes.c_uint64)

# name -> (restype, argtypes); every symbol the header declares.
SIGNATURES = {
    "vd_last_error": (ctypes.c_char_p, []),
    "vd_abi_version": (_int, []),
    "vd_jfa_schedule": (_int, [_i32, _i32, _i32, _p, _p, _i32]),
    "vd_djfa_schedule": (_int, [_i32, _i32, _i64, _i32, _i32, _i32, _p, _p, _i32]),
    "vd_create": (_p, [_i32, _i32, _i32]),
    "vd_destroy": (_int, [_p]),
    "vd_set_stream": (_int, [_p, _p]),
    "vd_synchronize": (_int, [_p]),
    "vd_get_shape": (_int, [_p, _P32, _P32, _P32, _P32]),
    "vd_set_seeds": (_int, [_p, _p, _int]),
    "vd_get_seeds": (_int, [_p, _p, _int]),
    "vd_move_seeds": (_int, [_p, _p, _int, _i32, _u64, _u64, _i64]),
    "vd_update_seeds": (_int, [_p, _p, _i32, _p, _i32, _int]),
    "vd_jfa": (_int, [_p, _i32, _i32]),
    "vd_djfa_step": (_int, [_p, _i32, _i32, _i32, _i32]),
    "vd_step": (_int, [_p, _p, _int, _i32, _u64, _u64, _i64, _i32, _i32, _i32, _i32]),
    "vd_stamp": (_int, [_p]),
    "vd_pass": (_int, [_p, _i32, _i32, _i32]),
    "vd_pass_rows": (_int, [_p, _i32, _i32, _i32, _i32, _i32, _i32]),
    "vd_clear_labels": (_int, [_p]),
    "vd_set_labels": (_int, [_p, _p, _int]),
    "vd_get_labels": (_int, [_p, _p, _int]),
    "vd_labels_device_ptr": (_int, [_p, ctypes.POINTER(_p)]),
    "vd_get_labels_async": (_int, [_p, _p]),
    "vd_get_labels16_async": (_int, [_p, _p]),
    "vd_get_labels24_async": (_int, [_p, _p]),
    "vd_get_labels_packed_async": (_int, [_p, _p, _i32]),
    "vd_wait_labels": (_int, [_p]),
    "vd_similarity": (_int, [_p, _p, _p, _int, _i32, _PU64, _PU64]),
    "vd_similarity_ctx": (_int, [_p, _p, _PU64]),
    "vd_exact": (_int, [_p, _p, _p, _int, _i32]),
    "vd_set_option": (_int, [_p, _i32, _i64]),
    "vd_autotune": (_int, [_p, _i32, _i32, _i32, _i32, _u64, _i32, _P32, _p, _i32]),
    "vd_get_option": (_int, [_p, _i32, ctypes.POINTER(_i64)]),
    "vd_launch_count": (_i64, [_p]),
    "vd_profile_read": (_int, [_p, _p, _p, _p]),
    "vd_profile_reset": (_int, [_p]),
    "vd_exact_noalloc": (_int, [_p, _i32, _i32, _i32, _i32, _p, _p, _p]),
    "vd_batch_create": (_p, [_i32, _p, _p, _p]),
    "vd_batch_destroy": (_int, [_p]),
    "vd_batch_set_stream": (_int, [_p, _p]),
    "vd_batch_synchronize": (_int, [_p]),
    "vd_batch_get_shape": (_int, [_p, _i32, _P32, _P32, _P32, _P32]),
    "vd_batch_set_seeds": (_int, [_p, _p, _int]),
    "vd_batch_get_seeds": (_int, [_p, _i32, _p, _int]),
    "vd_batch_get_labels": (_int, [_p, _i32, _p, _int]),
    "vd_batch_configure": (_int, [_p, _i32, _i32, _i32, _i32]),
    "vd_batch_jfa": (_int, [_p, _i32]),
    "vd_batch_step": (_int, [_p, _p, _int, _i32, _u64]),
    "vd_batch_step_subset": (_int, [_p, _p, _i32, _i32, _u64]),
    "vd_batch_set_option": (_int, [_p, _i32, _i64]),
    "vd_batch_get_option": (_int, [_p, _i32, ctypes.POINTER(_i64)]),
    "vd_batch_autotune": (_int, [_p, _i32, _i32, _u64, _P32, _p, _i32]),
    "vd_batch_work": (_int, [_p, ctypes.POINTER(_i64), ctypes.POINTER(_i64), ctypes.POINTER(_i64)]),
    "vd_batch_launch_count": (_i64, [_p]),
    "vd_server_create": (_p, [_i32, _i64, _i32, _i32, _i32, _i32, _u64]),
    "vd_server_destroy": (_int, [_p]),
    "vd_server_add_sim": (_i32, [_p, _i32, _i32, _i32, _p]),
    "vd_server_remove_sim": (_int, [_p, _i32]),
    "vd_server_submit": (_i64, [_p, _i32, ctypes.c_double]),
    "vd_server_progress": (_int, [_p]),
    "vd_server_drain": (_int, [_p]),
    "vd_server_completions": (_i32, [_p, _p, _p, _p, _i32]),
    "vd_server_now": (ctypes.c_double, [_p]),
    "vd_server_run_trace": (_int, [_p, _p, _p, _i64, _p]),
    "vd_server_get_labels": (_int, [_p, _i32, _p, _int]),
    "vd_server_stats": (_int, [_p, ctypes.POINTER(_i64), ctypes.POINTER(_i64), _P32, ctypes.POINTER(_i64),
                                ctypes.POINTER(_i64), ctypes.POINTER(_i64)]),
    "vd_server_set_max_batch": (_int, [_p, _i32]),
}

_lib = None
_lock = threading.Lock()


class VDError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{_ERRNAMES.get(code, code)}: {msg}")
        self.code = code


def lib() -> ctypes.CDLL:
    """The loaded library; raises if it was not built (no CPU fallback exists)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(
                f"CUDA library {LIB_PATH} is missing: build it with "
                "`python -c 'import __graft_entry__ as g; g.build()'` (nvcc, sm_103a)")
        handle = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(handle, name)
            fn.restype = res
            fn.argtypes = args
        _lib = handle
        return handle


def last_error() -> str:
    return lib().vd_last_error().decode()


def check(rc: int) -> int:
    if rc < 0:
        raise VDError(rc, last_error())
    return rc
