"""ctypes declarations of the C ABI in include/fgmm.h (libfgmm.so).

Argument marshalling only: every computation happens in the CUDA library.
Loading fails loudly if the library has not been built; there is no
fallback implementation.
"""
from __future__ import annotations

import ctypes
import os

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libfgmm.so")

FGMM_OK = 0
FGMM_ERR_INVALID_ARG = 1
FGMM_ERR_BAD_PARAMS = 2
FGMM_ERR_CAPACITY = 3
FGMM_ERR_CORRUPT = 4
FGMM_ERR_TIMEOUT = 5
FGMM_ERR_CUDA = 6
FGMM_ERR_NO_MEMORY = 7
FGMM_ERR_TOO_LARGE = 8
FGMM_NOALLOC_SCRATCH_BYTES = 16 << 20
FGMM_DTYPE_F32 = 0
FGMM_DTYPE_BF16 = 1
FGMM_MAX_K = 4
FGMM_OPT_DECODE_LANES = 1
FGMM_OPT_DECODE_CLUSTER = 2
FGMM_OPT_DECODE_ROUND0 = 3
FGMM_OPT_TEST_SILENT_STREAM = 4
FGMM_OPT_PHI = 5
FGMM_PHI_AS, FGMM_PHI_LOGISTIC, FGMM_PHI_POLYA = 0, 1, 2
FGMM_PEAK_FMA, FGMM_PEAK_RCP = 0, 1
FGMM_OPT_MLP_ACT = 6
FGMM_OPT_TEST_SILENT_ARRIVALS = 7
FGMM_MLP_ACT_PL, FGMM_MLP_ACT_SIGMOID = 0, 1
FGMM_DEC_LANE, FGMM_DEC_COOP, FGMM_DEC_WIDE, FGMM_DEC_WS = 0, 1, 2, 3
DECODE_KERNELS = {FGMM_DEC_LANE: "fgmm_dec_kernel", FGMM_DEC_COOP: "fgmm_dec_coop_kernel",
                  FGMM_DEC_WIDE: "fgmm_dec_wide_kernel", FGMM_DEC_WS: "fgmm_dec_ws_kernel"}
FGMM_MLP_PARAMS = 4929
FGMM_MLP_PACKED_BYTES = 11024


class fgmm_latent(ctypes.Structure):
    _fields_ = [("K", ctypes.c_int32), ("dtype", ctypes.c_int32), ("N", ctypes.c_int64),
                ("params", ctypes.c_void_p)]


P = ctypes.c_void_p
I32 = ctypes.c_int32
I64 = ctypes.c_int64
LATP = ctypes.POINTER(fgmm_latent)


class fgmm_batch_latent(ctypes.Structure):
    _fields_ = [("K", ctypes.c_int32), ("dtype", ctypes.c_int32), ("N", ctypes.c_int64),
                ("params", ctypes.c_void_p), ("symbols", ctypes.c_void_p), ("decoded", ctypes.c_void_p)]

# name -> (restype, argtypes); every function include/fgmm.h declares.
SIGNATURES = {
    "fgmm_create": (I32, [ctypes.POINTER(P)]),
    "fgmm_destroy": (None, [P]),
    "fgmm_status_string": (ctypes.c_char_p, [I32]),
    "fgmm_last_error": (ctypes.c_char_p, [P]),
    "fgmm_sync_status": (I32, [P, P]),
    "fgmm_self_check": (I32, [P, P]),
    "fgmm_fast_phi_bound": (I32, [P, P]),
    "fgmm_phi": (I32, [P, P, P, I64, P]),
    "fgmm_phi_grid": (I32, [P, I64, P, I64, P]),
    "fgmm_freqs": (I32, [P, LATP, P, P, P]),
    "fgmm_encode_bound_words": (I64, [I64, I32]),
    "fgmm_encode": (I32, [P, LATP, P, I32, P, I64, P, P, P]),
    "fgmm_decode": (I32, [P, LATP, P, I64, P, I32, P, P]),
    "fgmm_stats_enable": (I32, [P, I32]),
    "fgmm_stats_read": (I32, [P, P, P]),
    "fgmm_set_option": (I32, [P, I32, I64]),
    "fgmm_decode_plan": (I32, [P, I32, P]),
    "fgmm_table_bytes": (I64, [I64]),
    "fgmm_table_build": (I32, [P, LATP, P, P]),
    "fgmm_table_encode": (I32, [P, LATP, P, I32, P, P, I64, P, P, P]),
    "fgmm_table_decode": (I32, [P, LATP, P, P, I64, P, I32, P, P]),
    "fgmm_rate_audit": (I32, [P, LATP, P, P, P]),
    "fgmm_ckbd_anchors": (I64, [I64, I64, I64]),
    "fgmm_ckbd_split": (I32, [P, LATP, I64, I64, I64, P, P, P, P, P, P]),
    "fgmm_ckbd_merge": (I32, [P, I64, I64, I64, P, P, P, P]),
    "fgmm_ckbd_context": (I32, [P, LATP, I64, I64, I64, P, P, P]),
    "fgmm_ckbd_encode": (I32, [P, LATP, I64, I64, I64, P, I32, P, I64, P, P, I32, P, I64, P, P, P]),
    "fgmm_ckbd_decode": (I32, [P, LATP, I64, I64, I64, P, I64, P, I32, P, I64, P, I32, P, P]),
    "fgmm_ckbd_decode_plan": (I32, [P, I32, I32, I64, I64, I64, I32, I32, P]),
    "fgmm_gsm_tables_bytes": (I64, []),
    "fgmm_gsm_default_levels": (None, [P]),
    "fgmm_gsm_build": (I32, [P, P, I32, P, P]),
    "fgmm_gsm_freqs": (I32, [P, I32, I64, P, P, P, P, P]),
    "fgmm_gsm_encode": (I32, [P, I32, I64, P, P, I32, P, P, I64, P, P, P]),
    "fgmm_gsm_decode": (I32, [P, I32, I64, P, P, P, I64, P, I32, P, P]),
    "fgmm_autotune": (I32, [P, P, I32, ctypes.c_double, ctypes.c_double, P]),
    "fgmm_batch_create": (I32, [P, P, I32, P, P, I64, P, P, ctypes.POINTER(P)]),
    "fgmm_batch_destroy": (None, [P]),
    "fgmm_batch_segments": (I64, [P]),
    "fgmm_batch_streams": (I32, [P, P]),
    "fgmm_batch_capture": (I32, [P]),
    "fgmm_batch_encode": (I32, [P, P]),
    "fgmm_batch_decode": (I32, [P, P]),
    "fgmm_batch_decode_proposal": (I32, [P, P, P]),
    "fgmm_mlp_data": (I32, [P, LATP, P, P, P, P, P, P]),
    "fgmm_mlp_loss_grad": (I32, [P, P, P, I64, P, P, P, P]),
    "fgmm_mlp_train": (I32, [P, P, P, I64, P, P, P, I64, I64, I64, ctypes.c_float, P, P]),
    "fgmm_mlp_pack": (I32, [P, P, P, P]),
    "fgmm_mlp_forward": (I32, [P, P, I64, P, P, P]),
    "fgmm_decode_proposal": (I32, [P, LATP, P, P, I64, P, I32, P, P]),
    "fgmm_encode_noalloc": (I32, [LATP, P, I32, P, I64, P, P, P, P]),
    "fgmm_peak_probe": (I32, [P, I32, I64, P, P, P]),
}

_lib = None


class FgmmError(RuntimeError):
    def __init__(self, status: int, msg: str = ""):
        self.status = status
        super().__init__(f"fgmm status {status}: {msg}")


def lib():
    """The loaded libfgmm.so (raises if it is missing)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"libfgmm.so not built at {LIB_PATH}; run __graft_entry__.build()")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _bind(name):
    def call(*args):
        return getattr(lib(), name)(*args)
    call.__name__ = name
    call.__doc__ = f"C ABI entry point {name} (include/fgmm.h)."
    return call


for _name in SIGNATURES:
    globals()[_name] = _bind(_name)
