"""ctypes declarations of librick's C ABI (include/rick.h).

Argument marshalling only: every step of the imaging path runs in the CUDA
kernels of librick.so.  Loading fails loudly when the library has not been
built -- there is no fallback.
"""
import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "librick.so")

RICK_OK = 0
STATUS_NAMES = {0: "RICK_OK", 1: "RICK_ERR_ARG", 2: "RICK_ERR_OOM", 3: "RICK_ERR_CUDA",
                4: "RICK_ERR_CUFFT", 5: "RICK_ERR_TIMEOUT", 6: "RICK_ERR_STATE"}

KERNEL_GAUSS = 0
KERNEL_KB = 1
GRID_CORRECT = 1
REAL_IMAGE = 2
APPLY_N = 4
UNIFORM_WEIGHT = 8
HERMITIAN_FOLD = 32
FFT_2D = 64
FFT_SPLIT = 128


class RickParams(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("nw", ctypes.c_int32), ("pixel_rad", ctypes.c_double),
                ("w_min", ctypes.c_double), ("w_max", ctypes.c_double), ("kernel", ctypes.c_int32),
                ("support", ctypes.c_int32), ("kernel_param", ctypes.c_double),
                ("plane_group", ctypes.c_int32), ("tile", ctypes.c_int32), ("flags", ctypes.c_uint32),
                ("w_support", ctypes.c_int32)]


class RickStats(ctypes.Structure):
    _fields_ = [("n_gridded", ctypes.c_int64), ("n_dropped", ctypes.c_int64), ("n_entries", ctypes.c_int64),
                ("sum_weights", ctypes.c_double), ("plane_group", ctypes.c_int32), ("tile", ctypes.c_int32),
                ("workspace_bytes", ctypes.c_int64)]


class RickTiming(ctypes.Structure):
    _fields_ = [("prep_ms", ctypes.c_double), ("grid_ms", ctypes.c_double), ("fft_ms", ctypes.c_double),
                ("stack_ms", ctypes.c_double), ("degrid_ms", ctypes.c_double),
                ("prep_calls", ctypes.c_int64), ("grid_calls", ctypes.c_int64), ("fft_calls", ctypes.c_int64),
                ("stack_calls", ctypes.c_int64), ("degrid_calls", ctypes.c_int64),
                ("kernel_launches", ctypes.c_int64), ("colfft_ms", ctypes.c_double), ("colfft_calls", ctypes.c_int64)]


# exported symbol -> (restype, argtypes); kept in the order of include/rick.h
_H = ctypes.c_void_p
_P = ctypes.c_void_p
_S = ctypes.c_int32
SIGNATURES = {
    "rick_params_default": (_S, [ctypes.POINTER(RickParams)]),
    "rick_create": (_S, [ctypes.POINTER(RickParams), ctypes.POINTER(ctypes.c_void_p)]),
    "rick_destroy": (_S, [_H]),
    "rick_set_stream": (_S, [_H, _P]),
    "rick_workspace_size": (_S, [ctypes.POINTER(RickParams), ctypes.c_int64, ctypes.POINTER(ctypes.c_size_t)]),
    "rick_reset": (_S, [_H]),
    "rick_grid": (_S, [_H, _P, _P, _P, _P, _P, ctypes.c_int64]),
    "rick_add_density": (_S, [_H, _P, _P, _P, _P, _P, ctypes.c_int64]),
    "rick_fft_and_stack": (_S, [_H, _P]),
    "rick_grid_planes": (_S, [_H, ctypes.c_int32, ctypes.c_int32, _P]),
    "rick_degrid": (_S, [_H, _P, _P, _P, _P, _P, ctypes.c_int64, _P]),
    "rick_predict": (_S, [_H, _P, _P, _P, _P, ctypes.c_int64, _P]),
    "rick_image_host_async": (_S, [_H, _P, _P, _P, _P, _P, ctypes.c_int64, _P]),
    "rick_synchronize": (_S, [_H]),
    "rick_image_host": (_S, [_H, _P, _P, _P, _P, _P, ctypes.c_int64, _P]),
    "rick_create_batch": (_S, [ctypes.POINTER(RickParams), ctypes.c_int32, _P, _P,
                               ctypes.POINTER(ctypes.c_void_p)]),
    "rick_image_batch": (_S, [_H, _P, _P, _P, _P, _P, _P, _P, ctypes.c_int32]),
    "rick_autotune_batch": (_S, [ctypes.POINTER(RickParams), ctypes.c_int32, _P, _P, _P, _P, _P, _P, _P, _P,
                                 ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32),
                                 ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_double)]),
    "rick_set_prep_blocks": (_S, [_H, ctypes.c_int32]),
    "rick_grid_planes_static": (_S, [ctypes.POINTER(RickParams), _P, _P, _P, _P, _P, ctypes.c_int64, _P, _P,
                                     ctypes.c_char_p, ctypes.c_size_t]),
    "rick_set_plane_range": (_S, [_H, ctypes.c_int32, ctypes.c_int32]),
    "rick_set_weight_sum": (_S, [_H, ctypes.c_double]),
    "rick_debug_colstack": (_S, [_H, ctypes.c_int32, ctypes.c_int64]),
    "rick_get_stats": (_S, [_H, ctypes.POINTER(RickStats)]),
    "rick_set_timing": (_S, [_H, ctypes.c_int32]),
    "rick_get_timing": (_S, [_H, ctypes.POINTER(RickTiming)]),
    "rick_last_error": (ctypes.c_char_p, [_H]),
    "rick_status_string": (ctypes.c_char_p, [_S]),
}

_lib = None


def load(path=LIB_PATH):
    """Load librick.so and declare its signatures.  Raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"librick.so is not built ({path}); run __graft_entry__.build() or "
                           "python paper_2504_00959_gb300/build.py")
    L = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


class RickError(RuntimeError):
    def __init__(self, status, message):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


def check(status, handle=None):
    if status != RICK_OK:
        msg = ""
        if _lib is not None:
            # handle None: the message of the last failed creation on this thread
            raw = _lib.rick_last_error(handle)
            msg = raw.decode() if raw else ""
        raise RickError(status, msg)
