"""ctypes binding of libtsm (argument marshalling only).

Every function here forwards to the C ABI declared in ``include/tsm*.h``
with the same name.  There is no fallback: if ``libtsm.so`` is missing or
cannot be loaded, ``load()`` raises.
"""

import ctypes
import os
import threading

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libtsm.so")
DEFAULT_TABLE = os.path.join(_HERE, "tuning", "gb300_sm103.txt")

TSM_OK = 0
STATUS_NAMES = {0: "TSM_OK", 1: "TSM_ERR_INVALID_VALUE", 2: "TSM_ERR_NOT_SUPPORTED", 3: "TSM_ERR_ALLOC",
                4: "TSM_ERR_LAUNCH", 5: "TSM_ERR_TIMEOUT", 6: "TSM_ERR_INTERNAL", 7: "TSM_ERR_NO_DEVICE"}
R64, C64 = 0, 1
OP_N, OP_T, OP_C = 0, 1, 2
KIND_TSMTTSM, KIND_TSMM, KIND_TSMM_BETA = 0, 1, 2


class TsmError(RuntimeError):
    def __init__(self, status, where):
        self.status = status
        super().__init__("%s failed: %s (%s)" % (where, STATUS_NAMES.get(status, status),
                                                  _status_text(status)))


class VariantInfo(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 64), ("kind", ctypes.c_int), ("dtype", ctypes.c_int),
                ("fixed_m", ctypes.c_int), ("fixed_n", ctypes.c_int), ("tile_m", ctypes.c_int),
                ("tile_n", ctypes.c_int), ("threads_per_row", ctypes.c_int), ("unroll", ctypes.c_int),
                ("block", ctypes.c_int), ("generated", ctypes.c_int), ("runtime_tile", ctypes.c_int)]


class TuneSample(ctypes.Structure):
    _fields_ = [("variant", ctypes.c_int), ("grid", ctypes.c_int), ("ms", ctypes.c_float)]


_lock = threading.Lock()
_lib = None

i32, i64, u64, vp, dp = ctypes.c_int, ctypes.c_int64, ctypes.c_uint64, ctypes.c_void_p, \
    ctypes.POINTER(ctypes.c_double)

# name -> (restype, argtypes); the single source of the binding's signatures
SIGNATURES = {
    "tsm_tsmttsm": (i32, [i32, i32, i32, i32, i64, dp, vp, i64, vp, i64, dp, vp, i64, vp]),
    "tsm_tsmm": (i32, [i32, i32, i32, i32, i64, dp, vp, i64, vp, i64, dp, vp, i64, vp]),
    "tsm_tsmttsm_ex": (i32, [i32, i32, i32, i32, i64, dp, vp, i64, vp, i64, dp, vp, i64, i32, i32, vp]),
    "tsm_tsmm_ex": (i32, [i32, i32, i32, i32, i64, dp, vp, i64, vp, i64, dp, vp, i64, i32, i32, vp]),
    "tsm_gs_step": (i32, [i32, i32, i32, i64, vp, i64, vp, i64, vp, i64, vp]),
    "tsm_gs_step_ex": (i32, [i32, i32, i32, i64, vp, i64, vp, i64, vp, i64, i32, vp]),
    "tsm_gs_status": (i32, [vp]),
    "tsm_gs_set_timeout": (i32, [i64]),
    "tsm_variant_shape": (i32, [i32, i32, i32, i32, i32, ctypes.POINTER(VariantInfo)]),
    "tsm_status_string": (ctypes.c_char_p, [i32]),
    "tsm_version": (ctypes.c_char_p, []),
    "tsm_release": (i32, []),
    "tsm_variant_count": (i32, [i32]),
    "tsm_variant_get": (i32, [i32, i32, ctypes.POINTER(VariantInfo)]),
    "tsm_variant_supports": (i32, [i32, i32, i32, i32, i32]),
    "tsm_tsmttsm_kernels_per_call": (i32, [i32, i32, i32, i32]),
    "tsm_choose": (i32, [i32, i32, i32, i32, i64, ctypes.POINTER(i32), ctypes.POINTER(i32)]),
    "tsm_fill_random": (i32, [vp, i32, i64, i64, i64, u64, i32, vp]),
    "tsm_tune": (i32, [i32, i32, i32, i32, i64, vp, i64, vp, i64, vp, i64, i32,
                       ctypes.POINTER(TuneSample), i32, ctypes.POINTER(i32), vp]),
    "tsm_time_variant": (i32, [i32, i32, i32, i32, i64, vp, i64, vp, i64, vp, i64, i32, i32, i32,
                               ctypes.POINTER(ctypes.c_float), vp]),
    "tsm_set_tuning": (i32, [i32, i32, i32, i32, i64, i32, i32]),
    "tsm_set_tuning_timed": (i32, [i32, i32, i32, i32, i64, i32, i32, ctypes.c_float]),
    "tsm_tune_grids": (i32, [i32, i32, i32, i32, i32, ctypes.POINTER(i32), i32, ctypes.POINTER(i32)]),
    "tsm_load_tuning": (i32, [ctypes.c_char_p]),
    "tsm_save_tuning": (i32, [ctypes.c_char_p]),
    "tsm_clear_tuning": (i32, []),
}


def extend_signatures(extra):
    """Adds signatures declared by other headers (called by sibling modules
    before the first load)."""
    SIGNATURES.update(extra)
    with _lock:
        if _lib is not None:
            for name, (res, args) in extra.items():
                fn = getattr(_lib, name)
                fn.restype = res
                fn.argtypes = args


def load():
    """Loads libtsm.so (raises if it is missing: there is no fallback)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError("libtsm.so not built (%s); run paper_1905_03136_gb300.build" % LIB_PATH)
            lib = ctypes.CDLL(LIB_PATH)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            # The autotuned table for this GPU ships with the package; an
            # explicit TSM_TUNE_FILE replaces it (loaded here, so that the
            # table is complete before anything reads or saves it).
            env = os.environ.get("TSM_TUNE_FILE")
            if env:
                lib.tsm_load_tuning(env.encode())
            elif os.path.exists(DEFAULT_TABLE):
                lib.tsm_load_tuning(DEFAULT_TABLE.encode())
            _lib = lib
    return _lib


def _status_text(status):
    try:
        return load().tsm_status_string(status).decode()
    except Exception:
        return "?"


def check(status, where):
    if status != TSM_OK:
        raise TsmError(status, where)
    return status


def scalar(x, cplx):
    z = complex(x)
    arr = (ctypes.c_double * 2)(z.real, z.imag if cplx else 0.0)
    return arr


def call(name, *args):
    """Calls C function `name` and raises TsmError on a non-zero status."""
    return check(getattr(load(), name)(*args), name)


def raw(name):
    """The ctypes function object for `name` (status not checked)."""
    return getattr(load(), name)
