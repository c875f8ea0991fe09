"""CPU oracle for table-free Gaussian-mixture rANS coding (test infrastructure).

Only the test suite, the smoke check and the benchmark's CPU-baseline leg may
import this package. The product (the CUDA library and its binding) never
does, and shares no code with it.

The arithmetic lives in oracle.c (plain C, one symbol at a time); this module
only compiles it with gcc and marshals numpy arrays through ctypes.
"""
from __future__ import annotations

import contextlib
import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

OK, INVALID, BAD_PARAMS, CAPACITY, CORRUPT = 0, 1, 2, 3, 4
PHI_AS, PHI_LOGISTIC, PHI_POLYA = 0, 1, 2


def build(force: bool = False) -> str:
    """Compile oracle.c into oracle/_build/liboracle.so (IEEE FP32: no
    contraction, no fast-math)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
           "-fno-fast-math", "-fno-finite-math-only", "-Wall", "-pthread", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        I64 = ctypes.c_int64
        I32 = ctypes.c_int32
        lib.or_exp.restype = ctypes.c_float
        lib.or_exp.argtypes = [ctypes.c_float]
        lib.or_phi.restype = ctypes.c_float
        lib.or_phi.argtypes = [ctypes.c_float]
        lib.or_phi_many.argtypes = [P, P, I64]
        lib.or_exp_many.argtypes = [P, P, I64]
        lib.or_phi_grid_sweep.argtypes = [I64, I64, I64, P]
        lib.or_phi_grid.argtypes = [I64, I64, P]
        lib.or_mixcdf.restype = ctypes.c_float
        lib.or_mixcdf.argtypes = [P, ctypes.c_int, I64, I64, ctypes.c_float]
        lib.or_window.argtypes = [P, ctypes.c_int, I64, P, P]
        lib.or_freqs.restype = ctypes.c_int
        lib.or_freqs.argtypes = [P, ctypes.c_int, I64, P, P]
        lib.or_table.restype = ctypes.c_int
        lib.or_table.argtypes = [P, ctypes.c_int, I64, P]
        lib.or_encode.restype = I64
        lib.or_encode.argtypes = [P, ctypes.c_int, I64, P, I32, P, I64, P]
        lib.or_decode.restype = ctypes.c_int
        lib.or_decode.argtypes = [P, ctypes.c_int, I64, P, P, I32, P]
        lib.or_encode_mt.restype = I64
        lib.or_encode_mt.argtypes = [P, ctypes.c_int, I64, P, I32, P, I64, P, ctypes.c_int]
        lib.or_decode_mt.restype = ctypes.c_int
        lib.or_decode_mt.argtypes = [P, ctypes.c_int, I64, P, P, I32, P, ctypes.c_int]
        lib.or_p64.restype = ctypes.c_double
        lib.or_p64.argtypes = [P, ctypes.c_int, I64, I64, I32]
        lib.or_rate_audit.restype = ctypes.c_int
        lib.or_rate_audit.argtypes = [P, ctypes.c_int, I64, P, P]
        lib.or_phi_v.restype = ctypes.c_float
        lib.or_phi_v.argtypes = [ctypes.c_float, ctypes.c_int]
        lib.or_phi_v_many.argtypes = [P, P, I64, ctypes.c_int]
        lib.or_phi_v_grid_sweep.argtypes = [I64, I64, I64, ctypes.c_int, P]
        lib.or_set_phi.restype = ctypes.c_int
        lib.or_set_phi.argtypes = [ctypes.c_int]
        lib.or_gsm_levels.argtypes = [P]
        lib.or_gsm_params.restype = ctypes.c_int
        lib.or_gsm_params.argtypes = [P, ctypes.c_int, P, I64, P, P]
        lib.or_ckbd_split.argtypes = [ctypes.c_int, I64, I64, I64, P, P, P, P, P, P]
        lib.or_ckbd_merge.argtypes = [I64, I64, I64, P, P, P]
        lib.or_ckbd_context.argtypes = [ctypes.c_int, I64, I64, I64, P, P, P]
        _lib = lib
        return lib


def _p(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data)


def _params(params: np.ndarray) -> np.ndarray:
    a = np.ascontiguousarray(params, dtype=np.float32)
    assert a.ndim == 3 and a.shape[0] == 3, "params must be [3, K, N]"
    return a


def exp(a) -> np.ndarray:
    a = np.ascontiguousarray(a, dtype=np.float32)
    out = np.empty_like(a)
    _load().or_exp_many(_p(a), _p(out), a.size)
    return out


def phi(z) -> np.ndarray:
    z = np.ascontiguousarray(z, dtype=np.float32)
    out = np.empty_like(z)
    _load().or_phi_many(_p(z), _p(out), z.size)
    return out


def phi_grid(i0: int, n: int) -> np.ndarray:
    out = np.empty(n, dtype=np.float32)
    _load().or_phi_grid(i0, n, _p(out))
    return out


def phi_grid_sweep(i0: int, i1: int, err_stride: int = 1):
    out = np.zeros(3, dtype=np.float64)
    _load().or_phi_grid_sweep(i0, i1, err_stride, _p(out))
    return int(out[0]), float(out[1]), float(out[2])


def phi_v(z, v: int) -> np.ndarray:
    """Phi-hat of approximation v (PHI_AS, PHI_LOGISTIC, PHI_POLYA)."""
    z = np.ascontiguousarray(z, dtype=np.float32)
    out = np.empty_like(z)
    _load().or_phi_v_many(_p(z), _p(out), z.size, v)
    return out


def phi_v_grid_sweep(i0: int, i1: int, err_stride: int, v: int):
    """(decreases on the grid, max error vs v's formula in FP64, its z,
    max error vs Phi, its z) over grid points i0 .. i1."""
    out = np.zeros(5, dtype=np.float64)
    _load().or_phi_v_grid_sweep(i0, i1, err_stride, v, _p(out))
    return int(out[0]), float(out[1]), float(out[2]), float(out[3]), float(out[4])


@contextlib.contextmanager
def approximation(v: int):
    """Codes (freqs, table, encode, decode, rate audit) with approximation v
    inside the block; A&S again afterwards."""
    if _load().or_set_phi(v) != OK:
        raise ValueError(f"unknown approximation {v}")
    try:
        yield
    finally:
        _load().or_set_phi(PHI_AS)


def gsm_levels() -> np.ndarray:
    """The 64 scale levels of the Gaussian single model (fp32)."""
    out = np.empty(64, np.float32)
    _load().or_gsm_levels(_p(out))
    return out


def gsm_params(scales, levels=None):
    """Scales [N] -> (K = 1 parameters [3, 1, N] = (1, 0, level of the
    scale), level indices). The GSM coder codes the residual symbols with
    the K = 1 coder on these parameters. levels default to gsm_levels()."""
    sg = np.ascontiguousarray(scales, dtype=np.float32).ravel()
    lv = gsm_levels() if levels is None else np.ascontiguousarray(levels, dtype=np.float32)
    assert 1 <= lv.size <= 64
    N = sg.size
    po = np.empty((3, 1, N), np.float32)
    li = np.empty(N, np.int32)
    st = _load().or_gsm_params(_p(lv), lv.size, _p(sg), N, _p(po), _p(li))
    if st != OK:
        raise ValueError(f"oracle gsm status {st}")
    return po, li


def mixcdf(params, n: int, b: float) -> float:
    p = _params(params)
    return float(_load().or_mixcdf(_p(p), p.shape[1], p.shape[2], n, b))


def window(params):
    p = _params(params)
    N = p.shape[2]
    lo = np.empty(N, np.int32)
    hi = np.empty(N, np.int32)
    _load().or_window(_p(p), p.shape[1], N, _p(lo), _p(hi))
    return lo, hi


def freqs(params, symbols):
    """Packed intervals start | freq << 16 per symbol (uint32)."""
    p = _params(params)
    s = np.ascontiguousarray(symbols, dtype=np.int32)
    sf = np.empty(s.shape[0], np.uint32)
    st = _load().or_freqs(_p(p), p.shape[1], p.shape[2], _p(s), _p(sf))
    if st != OK:
        raise ValueError(f"oracle freqs status {st}")
    return sf


def table(params):
    """Full quantised-CDF table [N, 512] over j in [-255, 256]."""
    p = _params(params)
    N = p.shape[2]
    tab = np.empty((N, 512), np.uint16)
    st = _load().or_table(_p(p), p.shape[1], N, _p(tab))
    if st != OK:
        raise ValueError(f"oracle table status {st}")
    return tab


def encode_bound_words(N: int, S: int) -> int:
    T = -(-N // S) if N > 0 else 0
    return (S // 32) * (3 * 32 * T + 64)


def encode(params, symbols, S: int, threads: int = 1):
    """Returns (words uint16, offsets int64[S/32 + 1]). threads > 1 codes
    the segments on that many host threads (identical output)."""
    p = _params(params)
    s = np.ascontiguousarray(symbols, dtype=np.int32)
    N = p.shape[2]
    assert s.shape[0] == N
    cap = encode_bound_words(N, S)
    words = np.empty(max(cap, 1), np.uint16)
    offsets = np.empty(S // 32 + 1, np.int64)
    if threads > 1:
        n = _load().or_encode_mt(_p(p), p.shape[1], N, _p(s), S, _p(words), cap, _p(offsets), threads)
    else:
        n = _load().or_encode(_p(p), p.shape[1], N, _p(s), S, _p(words), cap, _p(offsets))
    if n < 0:
        raise ValueError(f"oracle encode status {-n}")
    return words[:n].copy(), offsets


def decode(params, words, offsets, S: int, threads: int = 1):
    """Returns (symbols int32[N], status). threads > 1 decodes the segments
    on that many host threads (identical output)."""
    p = _params(params)
    w = np.ascontiguousarray(words, dtype=np.uint16)
    if w.size == 0:
        w = np.zeros(1, np.uint16)
    o = np.ascontiguousarray(offsets, dtype=np.int64)
    N = p.shape[2]
    out = np.zeros(N, np.int32)
    if threads > 1:
        st = _load().or_decode_mt(_p(p), p.shape[1], N, _p(w), _p(o), S, _p(out), threads)
    else:
        st = _load().or_decode(_p(p), p.shape[1], N, _p(w), _p(o), S, _p(out))
    return out, st


def p64(params, n: int, s: int) -> float:
    p = _params(params)
    return float(_load().or_p64(_p(p), p.shape[1], p.shape[2], n, s))


def rate_audit(params, symbols):
    """(ideal_bits, coded_bits, max_cdf_err, n_escape) in FP64."""
    p = _params(params)
    s = np.ascontiguousarray(symbols, dtype=np.int32)
    out = np.zeros(4, np.float64)
    st = _load().or_rate_audit(_p(p), p.shape[1], p.shape[2], _p(s), _p(out))
    if st != OK:
        raise ValueError(f"oracle audit status {st}")
    return float(out[0]), float(out[1]), float(out[2]), int(out[3])


# ---- checkerboard two-pass coding (anchors h + w even, then the rest) ----

def ckbd_counts(shape):
    """(anchors, non-anchors) of a C x H x W latent."""
    C, H, W = shape
    na = C * ((H * W + 1) // 2)
    return na, C * H * W - na


def ckbd_split(params, y, shape):
    """-> (anchor params [3, K, Na], anchor symbols, non-anchor params,
    non-anchor symbols), each list channel by channel in raster order."""
    p = _params(params)
    K = p.shape[1]
    C, H, W = shape
    assert p.shape[2] == C * H * W
    na, nn = ckbd_counts(shape)
    yy = None if y is None else np.ascontiguousarray(y, dtype=np.int32)
    pa, pn = np.empty((3, K, na), np.float32), np.empty((3, K, nn), np.float32)
    ya, yn = np.zeros(na, np.int32), np.zeros(nn, np.int32)
    _load().or_ckbd_split(K, C, H, W, _p(p), None if yy is None else _p(yy), _p(pa), _p(ya), _p(pn), _p(yn))
    return pa, ya, pn, yn


def ckbd_merge(ya, yn, shape):
    C, H, W = shape
    y = np.zeros(C * H * W, np.int32)
    a = np.ascontiguousarray(ya, dtype=np.int32)
    b = None if yn is None else np.ascontiguousarray(yn, dtype=np.int32)
    _load().or_ckbd_merge(C, H, W, _p(a), None if b is None else _p(b), _p(y))
    return y


def ckbd_context(params, y, shape):
    """The fixed stand-in context model: non-anchor parameters [3, K, Nn]
    from the hyperprior parameters and the anchors of y."""
    p = _params(params)
    C, H, W = shape
    _, nn = ckbd_counts(shape)
    yy = np.ascontiguousarray(y, dtype=np.int32)
    pn = np.empty((3, p.shape[1], nn), np.float32)
    _load().or_ckbd_context(p.shape[1], C, H, W, _p(p), _p(yy), _p(pn))
    return pn


def ckbd_encode(params, y, shape, Sa: int, Sn: int):
    """Two-pass encode: anchors with the hyperprior's parameters, then the
    non-anchors with the context's. -> ((words, offsets) anchors, (words,
    offsets) non-anchors)."""
    pa, ya, _, yn = ckbd_split(params, y, shape)
    pn = ckbd_context(params, y, shape)
    return encode(pa, ya, Sa), encode(pn, yn, Sn)


def ckbd_decode(params, first, second, shape, Sa: int, Sn: int):
    """Two-pass decode: the anchors, then the context from them, then the
    non-anchors. -> (y, status)."""
    pa, _, _, _ = ckbd_split(params, None, shape)
    ya, st = decode(pa, first[0], first[1], Sa)
    if st != OK:
        return None, st
    y = ckbd_merge(ya, None, shape)
    pn = ckbd_context(params, y, shape)
    yn, st = decode(pn, second[0], second[1], Sn)
    if st != OK:
        return None, st
    return ckbd_merge(ya, yn, shape), OK
