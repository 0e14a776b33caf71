"""ctypes binding of liblgf.so (include/lgf.h): the same entry points under the
same names, argument marshalling only.  Every step of gauge fixing runs in the
library's CUDA kernels; there is no Python or CPU fallback, and loading fails
with an error if the compiled library is missing.
"""
from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "liblgf.so")

LGF_F64, LGF_F32, LGF_F32_R12, LGF_F64_R12 = 0, 1, 2, 3
DTYPES = {"f64": LGF_F64, "f32": LGF_F32, "f32_r12": LGF_F32_R12, "f64_r12": LGF_F64_R12}

LGF_OK = 0
LGF_ERR_ARG = -1
LGF_ERR_CUDA = -2
LGF_ERR_OOM = -3
LGF_ERR_NOT_CONVERGED = -4
LGF_ERR_NONFINITE = -5
LGF_ERR_TIMEOUT = -6
STATUS_NAMES = {0: "LGF_OK", -1: "LGF_ERR_ARG", -2: "LGF_ERR_CUDA", -3: "LGF_ERR_OOM",
                -4: "LGF_ERR_NOT_CONVERGED", -5: "LGF_ERR_NONFINITE", -6: "LGF_ERR_TIMEOUT"}

LGF_ALPHA, LGF_CHECK_EVERY, LGF_TAIL_THETA, LGF_TAIL_MAX_FP32 = 0, 1, 2, 3
LGF_REUNIT_FP64, LGF_FFT_PIPELINE, LGF_LINK_UPDATE, LGF_TAIL_MODE = 4, 5, 6, 7
LGF_EXP_ORDER, LGF_TRACK_G = 8, 9

# every symbol include/lgf.h declares: name -> (restype, argtypes)
_P = ctypes.c_void_p
_DP = ctypes.POINTER(ctypes.c_double)
_IP = ctypes.POINTER(ctypes.c_int)
ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p)
SIGNATURES = {
    "lgf_set_allocator": (ctypes.c_int, [ALLOC_FN, FREE_FN, _P]),
    "lgf_create": (ctypes.c_int, [ctypes.c_int] * 5 + [ctypes.POINTER(_P)]),
    "lgf_destroy": (ctypes.c_int, [_P]),
    "lgf_set_stream": (ctypes.c_int, [_P, _P]),
    "lgf_set_param": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_double]),
    "lgf_load_links": (ctypes.c_int, [_P, _P]),
    "lgf_load_links_device": (ctypes.c_int, [_P, _P]),
    "lgf_store_links": (ctypes.c_int, [_P, _P]),
    "lgf_store_gauge": (ctypes.c_int, [_P, _P]),
    "lgf_iterate": (ctypes.c_int, [_P, ctypes.c_int]),
    "lgf_fix": (ctypes.c_int, [_P, ctypes.c_double, ctypes.c_int, _IP]),
    "lgf_fix_stream": (ctypes.c_int, [_P, _P, ctypes.c_int, _P, _P, ctypes.c_double, ctypes.c_int, _IP]),
    "lgf_functional": (ctypes.c_int, [_P, _DP, _DP]),
    "lgf_probe": (ctypes.c_int, [_P, _P, _P, _P]),
    "lgf_history": (ctypes.c_int, [_P, _P, ctypes.c_int, _IP]),
    "lgf_fix_split": (ctypes.c_int, [_P, _IP, _IP]),
    "lgf_last_error": (ctypes.c_char_p, [_P]),
    "lgf_launch_count": (ctypes.c_longlong, [_P]),
    "lgf_profile": (ctypes.c_int, [_P, ctypes.c_int]),
    "lgf_profile_read": (ctypes.c_int, [_P, _P, _P, ctypes.c_int]),
    "lgf_kernel_name": (ctypes.c_char_p, [ctypes.c_int]),
    "lgf_functional_noalloc": (ctypes.c_int, [_P] + [ctypes.c_int] * 5 + [_P, _P]),
    "lgf_batch_create": (ctypes.c_int, [_P, ctypes.c_int, ctypes.POINTER(_P)]),
    "lgf_batch_destroy": (ctypes.c_int, [_P]),
    "lgf_batch_iterate": (ctypes.c_int, [_P, ctypes.c_int]),
    "lgf_batch_fix": (ctypes.c_int, [_P, ctypes.c_double, ctypes.c_int, _P, _P]),
    "lgf_batch_last_error": (ctypes.c_char_p, [_P]),
    "lgf_batch_set_lanes": (ctypes.c_int, [_P, ctypes.c_int]),
    "lgf_batch_autotune": (ctypes.c_int, [_P, ctypes.c_int, _P]),
    "lgf_autotune": (ctypes.c_int, [_P, ctypes.c_int, _IP]),
    "lgf_tune_schedule": (ctypes.c_int, [_P, ctypes.c_int, _IP, _IP, _IP]),
    "lgf_set_schedule": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int]),
    "lgf_tune_load": (ctypes.c_int, [ctypes.c_char_p, _IP]),
    "lgf_tune_save": (ctypes.c_int, [ctypes.c_char_p]),
    "lgf_tune_lookup": (ctypes.c_int, [ctypes.c_int] * 5 + [_IP, _IP, _IP]),
    "lgf_tune_clear": (ctypes.c_int, []),
    "lgf_net_param_count": (ctypes.c_int, []),
    "lgf_net_create": (ctypes.c_int, [ctypes.c_ulonglong, ctypes.POINTER(_P)]),
    "lgf_net_destroy": (ctypes.c_int, [_P]),
    "lgf_net_get_params": (ctypes.c_int, [_P, _P]),
    "lgf_net_set_params": (ctypes.c_int, [_P, _P]),
    "lgf_net_forward": (ctypes.c_int, [_P, _P, _P]),
    "lgf_net_train_step": (ctypes.c_int, [_P, _P, ctypes.c_double, _DP, _P]),
    "lgf_net_warm_start": (ctypes.c_int, [_P, _P]),
    "lgf_net_last_error": (ctypes.c_char_p, [_P]),
    "lgf_net_conv": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int, _P, _P, _P, _P] + [ctypes.c_int] * 4 + [_P]),
    "lgf_net_set_wait_budget": (ctypes.c_int, [_P, ctypes.c_longlong]),
}
LGF_NUM_KERNELS = 10

_lib = None


def load(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load liblgf.so and attach the signatures (raises if it is missing)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(
            f"liblgf.so not found at {path}: build it with "
            "`python -c 'import __graft_entry__ as g; g.build()'` (needs nvcc)")
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


class LgfError(RuntimeError):
    def __init__(self, status: int, where: str, detail: str):
        super().__init__(f"{where}: {STATUS_NAMES.get(status, status)}: {detail}")
        self.status = status


def check(status: int, where: str, handle=None) -> int:
    if status == LGF_OK:
        return status
    detail = load().lgf_last_error(handle)
    raise LgfError(status, where, detail.decode() if detail else "")


# --- torch's caching allocator behind the library's allocator hooks ---------
_torch_hooks = None


def use_torch_allocator() -> None:
    """Route the library's device allocations through torch's caching allocator."""
    global _torch_hooks
    if _torch_hooks is not None:
        return
    import torch

    def _alloc(nbytes, device, stream, user):
        try:
            return torch.cuda.caching_allocator_alloc(int(nbytes), int(device), int(stream or 0))
        except Exception:  # out of memory -> the library reports LGF_ERR_OOM
            return None

    def _free(ptr, nbytes, device, stream, user):
        torch.cuda.caching_allocator_delete(int(ptr))

    hooks = (ALLOC_FN(_alloc), FREE_FN(_free))
    check(load().lgf_set_allocator(hooks[0], hooks[1], None), "lgf_set_allocator")
    _torch_hooks = hooks
