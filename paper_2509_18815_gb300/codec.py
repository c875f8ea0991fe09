"""Torch-facing wrappers over the C ABI (include/fgmm.h).

PyTorch supplies device memory and the current CUDA stream; each function
marshals tensors into the C call of the same purpose and checks the status.
All arithmetic runs in libfgmm.so.
"""
from __future__ import annotations

import ctypes
import threading

import numpy as np

import torch

from . import _abi
from ._abi import FgmmError

_handles = {}
_hlock = threading.Lock()


class Handle:
    """Owns an fgmm_handle (workspace + device error word) on one device."""

    def __init__(self, device=None):
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else
                                   torch.device(device).index or 0)
        h = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            st = _abi.fgmm_create(ctypes.byref(h))
        if st != 0:
            raise FgmmError(st, "fgmm_create failed")
        self.ptr = h

    def close(self):
        if self.ptr:
            _abi.fgmm_destroy(self.ptr)
            self.ptr = None

    def last_error(self) -> str:
        return (_abi.fgmm_last_error(self.ptr) or b"").decode()

    def check(self, st: int):
        if st != 0:
            raise FgmmError(st, self.last_error())

    def sync(self, stream=None):
        """Synchronise the stream and raise on any device-recorded error."""
        self.check(_abi.fgmm_sync_status(self.ptr, _stream(stream)))


def handle(device=None) -> Handle:
    """Per-device default handle."""
    idx = torch.cuda.current_device() if device is None else (torch.device(device).index or 0)
    with _hlock:
        h = _handles.get(idx)
        if h is None:
            h = Handle(idx)
            _handles[idx] = h
        return h


def _stream(stream=None):
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


def _ptr(t: torch.Tensor):
    """Device pointer of a CUDA tensor (every pointer the C ABI takes from
    here is a device pointer; a host tensor is refused, not passed on)."""
    if t.numel() > 0 and not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    return ctypes.c_void_p(t.data_ptr() if t.numel() > 0 else 0)


def _tables(tables: torch.Tensor) -> torch.Tensor:
    """A GSM tables blob: a contiguous CUDA tensor of at least
    fgmm_gsm_tables_bytes() bytes, 16-byte aligned."""
    if not tables.is_cuda or not tables.is_contiguous():
        raise ValueError("tables must be a contiguous CUDA tensor")
    if tables.numel() * tables.element_size() < int(_abi.fgmm_gsm_tables_bytes()):
        raise ValueError("tables is smaller than fgmm_gsm_tables_bytes()")
    if tables.data_ptr() % 16:
        raise ValueError("tables must be 16-byte aligned")
    return tables


def latent(params: torch.Tensor) -> _abi.fgmm_latent:
    """Descriptor of a latent whose parameters are a CUDA tensor [3, K, N]
    (fp32 or bf16, contiguous)."""
    if params.dim() != 3 or params.shape[0] != 3:
        raise ValueError("params must have shape [3, K, N]")
    if not params.is_cuda or not params.is_contiguous():
        raise ValueError("params must be a contiguous CUDA tensor")
    if params.dtype == torch.float32:
        dt = _abi.FGMM_DTYPE_F32
    elif params.dtype == torch.bfloat16:
        dt = _abi.FGMM_DTYPE_BF16
    else:
        raise ValueError("params dtype must be float32 or bfloat16")
    return _abi.fgmm_latent(int(params.shape[1]), dt, int(params.shape[2]), params.data_ptr())


def phi(z: torch.Tensor, h: Handle | None = None) -> torch.Tensor:
    h = h or handle(z.device)
    z = z.contiguous()
    out = torch.empty_like(z)
    h.check(_abi.fgmm_phi(h.ptr, _ptr(z), _ptr(out), z.numel(), _stream()))
    h.sync()
    return out


def phi_grid(i0: int, n: int, device="cuda", h: Handle | None = None) -> torch.Tensor:
    h = h or handle(device)
    out = torch.empty(n, dtype=torch.float32, device=device)
    h.check(_abi.fgmm_phi_grid(h.ptr, i0, _ptr(out), n, _stream()))
    h.sync()
    return out


def freqs(params: torch.Tensor, symbols: torch.Tensor, h: Handle | None = None) -> torch.Tensor:
    """Per-symbol intervals start | freq << 16 (int32 tensor holding uint32 bits)."""
    h = h or handle(params.device)
    lat = latent(params)
    sym = symbols.to(torch.int32).contiguous()
    sf = torch.empty(lat.N, dtype=torch.int32, device=params.device)
    h.check(_abi.fgmm_freqs(h.ptr, ctypes.byref(lat), _ptr(sym), _ptr(sf), _stream()))
    h.sync()
    return sf


def encode_bound_words(N: int, S: int) -> int:
    return int(_abi.fgmm_encode_bound_words(N, S))


def encode(params: torch.Tensor, symbols: torch.Tensor, S: int | None = None, h: Handle | None = None,
           words_cap: int | None = None, sync: bool = True):
    """Encode one latent into S interleaved rANS streams (S = None: the
    autotuner's choice for this latent; S = 32 * (len(offsets) - 1)).

    Returns (words uint16-as-int16 tensor trimmed to its length, offsets int64
    [S/32 + 1]). With sync=False returns the untrimmed buffer, offsets and the
    device total, without synchronising."""
    h = h or handle(params.device)
    lat = latent(params)
    if S is None:
        S = autotune([lat.N], h=h)[0]
    sym = symbols.to(torch.int32).contiguous()
    cap = encode_bound_words(lat.N, S) if words_cap is None else words_cap
    if cap < 0:
        raise ValueError("S must be a positive multiple of 32")
    words = torch.empty(max(cap, 1), dtype=torch.int16, device=params.device)
    offsets = torch.empty(S // 32 + 1, dtype=torch.int64, device=params.device)
    total = torch.empty(1, dtype=torch.int64, device=params.device)
    h.check(_abi.fgmm_encode(h.ptr, ctypes.byref(lat), _ptr(sym), S, _ptr(words), cap, _ptr(offsets),
                             _ptr(total), _stream()))
    if not sync:
        return words, offsets, total
    h.sync()
    return words[: int(total.item())], offsets


def decode(params: torch.Tensor, words: torch.Tensor, offsets: torch.Tensor, S: int | None = None,
           h: Handle | None = None, out: torch.Tensor | None = None, sync: bool = True) -> torch.Tensor:
    """Decode one latent; returns int32 symbols [N]. S = None takes
    32 * (len(offsets) - 1)."""
    h = h or handle(params.device)
    lat = latent(params)
    words = words.contiguous()
    offsets = offsets.to(torch.int64).contiguous()
    if S is None:
        S = 32 * (offsets.numel() - 1)
    elif offsets.numel() != S // 32 + 1:
        raise ValueError("offsets must hold S/32 + 1 entries")
    if out is None:
        out = torch.empty(lat.N, dtype=torch.int32, device=params.device)
    h.check(_abi.fgmm_decode(h.ptr, ctypes.byref(lat), _ptr(words), words.numel(), _ptr(offsets), S, _ptr(out),
                             _stream()))
    if sync:
        h.sync()
    return out


def decode_plan(S: int, h: Handle | None = None) -> dict:
    """Decoder that decode() runs for S streams under the handle's options:
    lanes per stream, CTAs per segment, first-round points and the kernel's
    name."""
    h = h or handle()
    out = (ctypes.c_int32 * 4)()
    h.check(_abi.fgmm_decode_plan(h.ptr, S, out))
    return {"lanes": int(out[0]), "cluster": int(out[1]), "round0": int(out[3]),
            "kernel": _abi.DECODE_KERNELS[int(out[2])]}


def stats_enable(on: bool = True, h: Handle | None = None):
    h = h or handle()
    h.check(_abi.fgmm_stats_enable(h.ptr, 1 if on else 0))


def peak_probe(kind: int, iters: int, sink: torch.Tensor, h: Handle | None = None, stream=None) -> float:
    """Launches the library's throughput probe (fgmm_peak_probe: chains of
    FP32 FMAs for kind FGMM_PEAK_FMA, XU reciprocals for FGMM_PEAK_RCP) on
    the stream and returns the per-lane operations it performs; the caller
    times it. sink: a CUDA float tensor of at least one element."""
    h = h or handle()
    ops = ctypes.c_double(0.0)
    h.check(_abi.fgmm_peak_probe(h.ptr, kind, iters, _ptr(sink), ctypes.addressof(ops), _stream(stream)))
    return ops.value


def stats_read(h: Handle | None = None, with_hits: bool = False, with_fallbacks: bool = False):
    """(cdf_evals, symbols_decoded[, proposal_hits][, guide_fallbacks]) since
    the last read."""
    h = h or handle()
    out = (ctypes.c_uint64 * 4)()
    h.check(_abi.fgmm_stats_read(h.ptr, out, _stream()))
    r = (int(out[0]), int(out[1]))
    if with_hits:
        r += (int(out[2]),)
    if with_fallbacks:
        r += (int(out[3]),)
    return r


def table_build(params: torch.Tensor, h: Handle | None = None) -> torch.Tensor:
    """Quantised-CDF table [N, 512] (uint16 bits in int16) of the comparison coder."""
    h = h or handle(params.device)
    lat = latent(params)
    table = torch.empty((lat.N, 512), dtype=torch.int16, device=params.device)
    h.check(_abi.fgmm_table_build(h.ptr, ctypes.byref(lat), _ptr(table), _stream()))
    h.sync()
    return table


def table_encode(params, symbols, S, table=None, h: Handle | None = None, sync: bool = True):
    """Table-based encode (same stream as encode()). Returns (words, offsets)."""
    h = h or handle(params.device)
    lat = latent(params)
    sym = symbols.to(torch.int32).contiguous()
    if table is None:
        table = torch.empty((lat.N, 512), dtype=torch.int16, device=params.device)
    cap = encode_bound_words(lat.N, S)
    words = torch.empty(max(cap, 1), dtype=torch.int16, device=params.device)
    offsets = torch.empty(S // 32 + 1, dtype=torch.int64, device=params.device)
    total = torch.empty(1, dtype=torch.int64, device=params.device)
    h.check(_abi.fgmm_table_encode(h.ptr, ctypes.byref(lat), _ptr(sym), S, _ptr(table), _ptr(words), cap,
                                   _ptr(offsets), _ptr(total), _stream()))
    if not sync:
        return words, offsets, total
    h.sync()
    return words[: int(total.item())], offsets


def table_decode(params, words, offsets, S, table=None, h: Handle | None = None, out=None, sync: bool = True):
    """Table-based decode (builds the table, then searches it)."""
    h = h or handle(params.device)
    lat = latent(params)
    if table is None:
        table = torch.empty((lat.N, 512), dtype=torch.int16, device=params.device)
    if out is None:
        out = torch.empty(lat.N, dtype=torch.int32, device=params.device)
    words = words.contiguous()
    offsets = offsets.to(torch.int64).contiguous()
    h.check(_abi.fgmm_table_decode(h.ptr, ctypes.byref(lat), _ptr(table), _ptr(words), words.numel(), _ptr(offsets),
                                   S, _ptr(out), _stream()))
    if sync:
        h.sync()
    return out


# ---- Gaussian single model with pre-built tables (Sec. II-C) ----

def gsm_default_levels() -> np.ndarray:
    """The 64 default scale levels (log-even in [0.11, 256]), float32."""
    out = np.empty(64, np.float32)
    _abi.fgmm_gsm_default_levels(out.ctypes.data_as(ctypes.c_void_p))
    return out


def gsm_build(levels=None, device="cuda", h: Handle | None = None) -> torch.Tensor:
    """Tables blob (uint8 device tensor) for the given increasing levels
    (default: the 64 default levels)."""
    h = h or handle(device)
    lv = gsm_default_levels() if levels is None else np.ascontiguousarray(levels, dtype=np.float32)
    blob = torch.empty(int(_abi.fgmm_gsm_tables_bytes()), dtype=torch.uint8, device=device)
    h.check(_abi.fgmm_gsm_build(h.ptr, lv.ctypes.data_as(ctypes.c_void_p), int(lv.size), _ptr(blob), _stream()))
    h.sync()
    return blob


def _scales(scales: torch.Tensor):
    if scales.dim() != 1 or not scales.is_cuda or not scales.is_contiguous():
        raise ValueError("scales must be a contiguous 1-D CUDA tensor")
    if scales.dtype == torch.float32:
        return _abi.FGMM_DTYPE_F32
    if scales.dtype == torch.bfloat16:
        return _abi.FGMM_DTYPE_BF16
    raise ValueError("scales dtype must be float32 or bfloat16")


def gsm_freqs(scales, symbols, tables, h: Handle | None = None) -> torch.Tensor:
    h = h or handle(scales.device)
    dt = _scales(scales)
    sym = symbols.to(torch.int32).contiguous()
    sf = torch.empty(scales.numel(), dtype=torch.int32, device=scales.device)
    h.check(_abi.fgmm_gsm_freqs(h.ptr, dt, scales.numel(), _ptr(scales), _ptr(sym), _ptr(_tables(tables)), _ptr(sf),
                                _stream()))
    h.sync()
    return sf


def gsm_encode(scales, symbols, S: int, tables, h: Handle | None = None, sync: bool = True):
    """Encode residuals with their scales. Returns (words, offsets) as encode()."""
    h = h or handle(scales.device)
    dt = _scales(scales)
    N = scales.numel()
    sym = symbols.to(torch.int32).contiguous()
    cap = encode_bound_words(N, S)
    if cap < 0:
        raise ValueError("S must be a positive multiple of 32")
    words = torch.empty(max(cap, 1), dtype=torch.int16, device=scales.device)
    offsets = torch.empty(S // 32 + 1, dtype=torch.int64, device=scales.device)
    total = torch.empty(1, dtype=torch.int64, device=scales.device)
    h.check(_abi.fgmm_gsm_encode(h.ptr, dt, N, _ptr(scales), _ptr(sym), S, _ptr(_tables(tables)), _ptr(words), cap,
                                 _ptr(offsets), _ptr(total), _stream()))
    if not sync:
        return words, offsets, total
    h.sync()
    return words[: int(total.item())], offsets


def gsm_decode(scales, words, offsets, S: int, tables, h: Handle | None = None, out=None, sync: bool = True):
    """Decode residuals; returns int32 [N]."""
    h = h or handle(scales.device)
    dt = _scales(scales)
    N = scales.numel()
    words = words.contiguous()
    offsets = offsets.to(torch.int64).contiguous()
    if out is None:
        out = torch.empty(N, dtype=torch.int32, device=scales.device)
    h.check(_abi.fgmm_gsm_decode(h.ptr, dt, N, _ptr(scales), _ptr(_tables(tables)), _ptr(words), words.numel(),
                                 _ptr(offsets), S, _ptr(out), _stream()))
    if sync:
        h.sync()
    return out


# ---- checkerboard two-pass coding (anchors h + w even, then the rest) ----

def ckbd_split(params, y, shape, h: Handle | None = None):
    """-> (anchor params, anchor symbols, non-anchor params, non-anchor
    symbols); y may be None (parameters only, symbols returned as None)."""
    h = h or handle(params.device)
    lat = latent(params)
    C, H, W = shape
    na = int(_abi.fgmm_ckbd_anchors(C, H, W))
    nn = C * H * W - na
    K = params.shape[1]
    pa = torch.empty((3, K, na), dtype=params.dtype, device=params.device)
    pn = torch.empty((3, K, nn), dtype=params.dtype, device=params.device)
    ya = yn = None
    if y is not None:
        y = y.to(torch.int32).contiguous()
        ya = torch.empty(na, dtype=torch.int32, device=params.device)
        yn = torch.empty(nn, dtype=torch.int32, device=params.device)
    h.check(_abi.fgmm_ckbd_split(h.ptr, ctypes.byref(lat), C, H, W, None if y is None else _ptr(y), _ptr(pa),
                                 None if ya is None else _ptr(ya), _ptr(pn), None if yn is None else _ptr(yn),
                                 _stream()))
    return pa, ya, pn, yn


def ckbd_merge(ya, yn, shape, y=None, h: Handle | None = None):
    h = h or handle(ya.device)
    C, H, W = shape
    if y is None:
        y = torch.zeros(C * H * W, dtype=torch.int32, device=ya.device)
    h.check(_abi.fgmm_ckbd_merge(h.ptr, C, H, W, _ptr(ya), None if yn is None else _ptr(yn), _ptr(y), _stream()))
    return y


def ckbd_context(params, y, shape, out=None, h: Handle | None = None):
    """The fixed stand-in context model: fp32 non-anchor parameters."""
    h = h or handle(params.device)
    lat = latent(params)
    C, H, W = shape
    nn = C * H * W - int(_abi.fgmm_ckbd_anchors(C, H, W))
    if out is None:
        out = torch.empty((3, params.shape[1], nn), dtype=torch.float32, device=params.device)
    h.check(_abi.fgmm_ckbd_context(h.ptr, ctypes.byref(lat), C, H, W, _ptr(y), _ptr(out), _stream()))
    return out


def ckbd_encode(params, y, shape, Sa: int, Sn: int, h: Handle | None = None, sync: bool = True):
    """Two-pass encode (fgmm_ckbd_encode): anchors with the hyperprior's
    parameters, then the non-anchors with the context's.
    -> ((words, offsets), (words, offsets)); with sync=False the untrimmed
    buffers, offsets and device totals of each pass, unsynchronised."""
    h = h or handle(params.device)
    lat = latent(params)
    C, H, W = shape
    na = int(_abi.fgmm_ckbd_anchors(C, H, W))
    nn = C * H * W - na
    yv = y.to(torch.int32).contiguous()
    out = []
    for n, S in ((na, Sa), (nn, Sn)):
        cap = encode_bound_words(n, S)
        if cap < 0:
            raise ValueError("S must be a positive multiple of 32")
        out.append((torch.empty(max(cap, 1), dtype=torch.int16, device=params.device),
                    torch.empty(S // 32 + 1, dtype=torch.int64, device=params.device),
                    torch.empty(1, dtype=torch.int64, device=params.device), cap))
    (wa, oa, ta, ca), (wn, on, tn, cn) = out
    h.check(_abi.fgmm_ckbd_encode(h.ptr, ctypes.byref(lat), C, H, W, _ptr(yv), Sa, _ptr(wa), ca, _ptr(oa), _ptr(ta),
                                  Sn, _ptr(wn), cn, _ptr(on), _ptr(tn), _stream()))
    if not sync:
        return (wa, oa, ta), (wn, on, tn)
    h.sync()
    return (wa[: int(ta.item())], oa), (wn[: int(tn.item())], on)


def ckbd_encode_steps(params, y, shape, Sa: int, Sn: int, h: Handle | None = None, sync: bool = True):
    """The two-pass encode as its separate library calls: split, context,
    two encodes (the same bytes as ckbd_encode)."""
    h = h or handle(params.device)
    pa, ya, _, yn = ckbd_split(params, y, shape, h)
    pn = ckbd_context(params, y.to(torch.int32).contiguous(), shape, h=h)
    return encode(pa, ya, Sa, h, sync=sync), encode(pn, yn, Sn, h, sync=sync)


def ckbd_decode(params, first, second, shape, Sa: int, Sn: int, h: Handle | None = None, sync: bool = True,
                out=None):
    """Two-pass decode (fgmm_ckbd_decode): the anchors, the context from
    them, the non-anchors; one fused launch where the library can."""
    h = h or handle(params.device)
    lat = latent(params)
    C, H, W = shape
    (wa, oa), (wn, on) = first, second
    oa, on = oa.to(torch.int64).contiguous(), on.to(torch.int64).contiguous()
    if out is None:
        out = torch.empty(C * H * W, dtype=torch.int32, device=params.device)
    h.check(_abi.fgmm_ckbd_decode(h.ptr, ctypes.byref(lat), C, H, W, _ptr(wa), wa.numel(), _ptr(oa), Sa,
                                  _ptr(wn), wn.numel(), _ptr(on), Sn, _ptr(out), _stream()))
    if sync:
        h.sync()
    return out


def ckbd_decode_steps(params, first, second, shape, Sa: int, Sn: int, h: Handle | None = None,
                      sync: bool = True):
    """The two-pass decode as its separate library calls, one after the
    other: split, pass-1 decode, anchor merge, context, pass-2 decode,
    merge (the same symbols as ckbd_decode)."""
    h = h or handle(params.device)
    pa, _, _, _ = ckbd_split(params, None, shape, h)
    ya = decode(pa, first[0], first[1], Sa, h, sync=False)
    y = ckbd_merge(ya, None, shape, h=h)
    pn = ckbd_context(params, y, shape, h=h)
    yn = decode(pn, second[0], second[1], Sn, h, sync=False)
    ckbd_merge(ya, yn, shape, y=y, h=h)
    if sync:
        h.sync()
    return y


def ckbd_decode_fused(K: int, dtype, shape, Sa: int, Sn: int, h: Handle | None = None) -> bool:
    """Whether ckbd_decode decodes both passes in one launch for this case."""
    h = h or handle()
    C, H, W = shape
    dt = _abi.FGMM_DTYPE_BF16 if dtype == torch.bfloat16 else _abi.FGMM_DTYPE_F32
    out = ctypes.c_int32(-1)
    h.check(_abi.fgmm_ckbd_decode_plan(h.ptr, K, dt, C, H, W, Sa, Sn, ctypes.byref(out)))
    return bool(out.value)


class CkbdGraphs:
    """Checkerboard two-pass coding of one latent shape replayed from CUDA
    graphs. The encode sequence (fgmm_ckbd_encode) and the decode sequence
    (fgmm_ckbd_decode) are each captured once with fixed buffers; every node
    of a replay is a library kernel, and the graphs remove the host's
    per-launch work and the gaps between kernels. params: [3, K, C H W] on
    the GPU; shape (C, H, W); Sa, Sn: the passes' stream counts.
    capture_encode(y) / encode() fill enc_first and enc_second ((words,
    offsets, total) of each pass, untrimmed); capture_decode(first, second)
    / decode() decode the given (words, offsets) pairs into `y`. The graphs
    hold the handle's workspace, so the class uses a handle of its own
    unless one is given (a call that grows a given handle's workspace after
    a capture invalidates the graphs); every capture first runs each
    sequence it holds once, so that both graphs see the final workspace."""

    def __init__(self, params, shape, Sa: int, Sn: int, h: Handle | None = None):
        self.h = h or Handle(params.device)
        self.params = params.contiguous()
        self.shape = tuple(shape)
        self.Sa, self.Sn = Sa, Sn
        self.g_enc = self.g_dec = None
        self._y_in = self._first = None

    def _encode_seq(self, y):
        return ckbd_encode(self.params, y, self.shape, self.Sa, self.Sn, self.h, sync=False)

    def _decode_seq(self):
        return ckbd_decode(self.params, self._first, self._second, self.shape, self.Sa, self.Sn, self.h, sync=False)

    def _capture(self):
        # every sequence once outside the captures (grows the workspace), then
        # every graph again, so that none holds a workspace that was freed
        if self._y_in is not None:
            self._encode_seq(self._y_in)
        if self._first is not None:
            self._decode_seq()
        self.h.sync()
        if self._y_in is not None:
            self.g_enc = torch.cuda.CUDAGraph()
            with torch.cuda.graph(self.g_enc, capture_error_mode="thread_local"):
                self.enc_first, self.enc_second = self._encode_seq(self._y_in)
        if self._first is not None:
            self.g_dec = torch.cuda.CUDAGraph()
            with torch.cuda.graph(self.g_dec, capture_error_mode="thread_local"):
                self.y = self._decode_seq()

    def capture_encode(self, y):
        self._y_in = y.to(torch.int32).contiguous()
        self._capture()

    def encode(self, sync: bool = True):
        self.g_enc.replay()
        if sync:
            self.h.sync()
        return self.enc_first, self.enc_second

    def capture_decode(self, first, second):
        self._first = (first[0].contiguous(), first[1].to(torch.int64).contiguous())
        self._second = (second[0].contiguous(), second[1].to(torch.int64).contiguous())
        self._capture()

    def decode(self, sync: bool = True):
        self.g_dec.replay()
        if sync:
            self.h.sync()
        return self.y


def rate_audit(params, symbols, h: Handle | None = None):
    """(ideal_bits, coded_bits, max_cdf_err, n_escape) computed in FP64 on the GPU."""
    h = h or handle(params.device)
    lat = latent(params)
    sym = symbols.to(torch.int32).contiguous()
    out = torch.empty(4, dtype=torch.float64, device=params.device)
    h.check(_abi.fgmm_rate_audit(h.ptr, ctypes.byref(lat), _ptr(sym), _ptr(out), _stream()))
    h.sync()
    v = out.cpu().tolist()
    return v[0], v[1], v[2], int(v[3])


def autotune(Ns, max_overhead: float = 0.01, bits_per_symbol: float = 3.5, h: Handle | None = None):
    """Stream counts for a batch of latents with N symbols each (see
    fgmm_autotune in include/fgmm.h)."""
    h = h or handle()
    n = len(Ns)
    arr = (ctypes.c_int64 * max(n, 1))(*[int(x) for x in Ns])
    out = (ctypes.c_int32 * max(n, 1))()
    h.check(_abi.fgmm_autotune(h.ptr, arr, n, max_overhead, bits_per_symbol, out))
    return [int(out[i]) for i in range(n)]


class Batch:
    """A batch plan (fgmm_batch): n latents coded by one persistent launch per
    direction, optionally replayed from captured CUDA graphs.

    params: list of CUDA tensors [3, K, N]; symbols: list of int32 CUDA
    tensors [N]. After encode(), `words`, `offsets`, `n_words` hold the batch
    stream; decode() writes `decoded` (list of int32 tensors)."""

    def __init__(self, params, symbols, S=None, h: Handle | None = None, words_cap: int | None = None):
        self.h = h or handle(params[0].device if params else None)
        dev = params[0].device
        n = len(params)
        self.params = [p.contiguous() for p in params]
        self.symbols = [s.to(torch.int32).contiguous() for s in symbols]
        self.decoded = [torch.empty(int(p.shape[2]), dtype=torch.int32, device=dev) for p in self.params]
        lats = (_abi.fgmm_batch_latent * max(n, 1))()
        for i, (p, s, d) in enumerate(zip(self.params, self.symbols, self.decoded)):
            base = latent(p)
            lats[i] = _abi.fgmm_batch_latent(base.K, base.dtype, base.N, base.params, _ptr(s).value or 0,
                                             _ptr(d).value or 0)
        s_arr = None
        if S is not None:
            s_arr = (ctypes.c_int32 * max(n, 1))(*[int(x) for x in S])
        total_bound = 0
        Ss = S if S is not None else autotune([int(p.shape[2]) for p in self.params], h=self.h)
        for p, si in zip(self.params, Ss):
            total_bound += encode_bound_words(int(p.shape[2]), si)
        cap = total_bound if words_cap is None else words_cap
        self.words = torch.empty(max(cap, 1), dtype=torch.int16, device=dev)
        nseg = sum(si // 32 for si in Ss)
        self.offsets = torch.empty(nseg + 1, dtype=torch.int64, device=dev)
        self.total = torch.empty(1, dtype=torch.int64, device=dev)
        ptr = ctypes.c_void_p()
        self.h.check(_abi.fgmm_batch_create(self.h.ptr, lats, n, s_arr if s_arr is not None else None,
                                            _ptr(self.words), cap, _ptr(self.offsets), _ptr(self.total),
                                            ctypes.byref(ptr)))
        self.ptr = ptr
        out = (ctypes.c_int32 * max(n, 1))()
        self.h.check(_abi.fgmm_batch_streams(self.ptr, out))
        self.S = [int(out[i]) for i in range(n)]
        assert self.S == list(Ss)
        self.seg_base = [0]
        for si in self.S:
            self.seg_base.append(self.seg_base[-1] + si // 32)

    def capture(self):
        self.h.check(_abi.fgmm_batch_capture(self.ptr))

    def encode(self, sync: bool = True):
        self.h.check(_abi.fgmm_batch_encode(self.ptr, _stream()))
        if sync:
            self.h.sync()

    def decode(self, sync: bool = True):
        self.h.check(_abi.fgmm_batch_decode(self.ptr, _stream()))
        if sync:
            self.h.sync()

    def decode_proposal(self, packed=None, sync: bool = True):
        """The whole batch decoded with the proposal (packed network, or the
        analytic proposal for None) in one persistent launch."""
        self.h.check(_abi.fgmm_batch_decode_proposal(self.ptr, _ptr(packed) if packed is not None else None,
                                                     _stream()))
        if sync:
            self.h.sync()

    def latent_stream(self, i: int):
        """(words, offsets) of latent i, in the single-latent format."""
        off = self.offsets[self.seg_base[i]: self.seg_base[i + 1] + 1]
        a, b = int(off[0].item()), int(off[-1].item())
        return self.words[a:b], off - a

    def close(self):
        if self.ptr:
            _abi.fgmm_batch_destroy(self.ptr)
            self.ptr = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------------------------
# Learned decode proposal
# ---------------------------------------------------------------------------

def mlp_data(params, symbols, uniforms, h: Handle | None = None, with_slots: bool = False):
    """Training triples (features X [N, 10], target [N][, slots [N]])."""
    h = h or handle(params.device)
    lat = latent(params)
    dev = params.device
    X = torch.empty((lat.N, 10), dtype=torch.float32, device=dev)
    t = torch.empty(lat.N, dtype=torch.float32, device=dev)
    sl = torch.empty(lat.N, dtype=torch.int32, device=dev) if with_slots else None
    u = uniforms.to(torch.float32).contiguous()
    sym = symbols.to(torch.int32).contiguous()
    h.check(_abi.fgmm_mlp_data(h.ptr, ctypes.byref(lat), _ptr(sym), _ptr(u), _ptr(X), _ptr(t),
                               _ptr(sl) if sl is not None else None, _stream()))
    h.sync()
    return (X, t, sl) if with_slots else (X, t)


def mlp_loss_grad(X, target, theta, h: Handle | None = None):
    h = h or handle(X.device)
    g = torch.empty(_abi.FGMM_MLP_PARAMS, dtype=torch.float32, device=X.device)
    loss = torch.empty(1, dtype=torch.float32, device=X.device)
    h.check(_abi.fgmm_mlp_loss_grad(h.ptr, _ptr(X.contiguous()), _ptr(target.contiguous()), X.shape[0],
                                    _ptr(theta), _ptr(g), _ptr(loss), _stream()))
    h.sync()
    return float(loss.item()), g


class MlpTrainer:
    """FP32 master weights and Adam state of the proposal network on the GPU.
    state_dict()/load_state_dict() checkpoint and resume training exactly."""

    def __init__(self, theta0, device="cuda", h: Handle | None = None):
        self.h = h or handle(device)
        self.theta = torch.as_tensor(theta0, dtype=torch.float32).to(device).contiguous()
        self.m = torch.zeros_like(self.theta)
        self.v = torch.zeros_like(self.theta)
        self.step = 0

    def train(self, X, target, steps: int, batch: int, lr: float):
        trace = torch.empty(max(steps, 1), dtype=torch.float32, device=self.theta.device)
        self.h.check(_abi.fgmm_mlp_train(self.h.ptr, _ptr(X), _ptr(target), X.shape[0], _ptr(self.theta),
                                         _ptr(self.m), _ptr(self.v), self.step, steps, batch, lr, _ptr(trace),
                                         _stream()))
        self.h.sync()
        self.step += steps
        return trace[:steps]

    def state_dict(self):
        return {"theta": self.theta.cpu().clone(), "m": self.m.cpu().clone(), "v": self.v.cpu().clone(),
                "step": self.step}

    def load_state_dict(self, st):
        dev = self.theta.device
        self.theta = st["theta"].to(dev).contiguous()
        self.m = st["m"].to(dev).contiguous()
        self.v = st["v"].to(dev).contiguous()
        self.step = int(st["step"])

    def packed(self):
        P = torch.empty(_abi.FGMM_MLP_PACKED_BYTES // 4, dtype=torch.int32, device=self.theta.device)
        self.h.check(_abi.fgmm_mlp_pack(self.h.ptr, _ptr(self.theta), _ptr(P), _stream()))
        self.h.sync()
        return P


def set_mlp_act(act: int, h: Handle | None = None):
    """Activation of the proposal network on this handle (training,
    inference and the proposal decoders): _abi.FGMM_MLP_ACT_PL or
    _abi.FGMM_MLP_ACT_SIGMOID."""
    h = h or handle()
    h.check(_abi.fgmm_set_option(h.ptr, _abi.FGMM_OPT_MLP_ACT, act))


def mlp_pack(theta, h: Handle | None = None):
    h = h or handle(theta.device)
    P = torch.empty(_abi.FGMM_MLP_PACKED_BYTES // 4, dtype=torch.int32, device=theta.device)
    h.check(_abi.fgmm_mlp_pack(h.ptr, _ptr(theta.contiguous()), _ptr(P), _stream()))
    h.sync()
    return P


def mlp_forward(X, packed, h: Handle | None = None):
    h = h or handle(X.device)
    y = torch.empty(X.shape[0], dtype=torch.float32, device=X.device)
    h.check(_abi.fgmm_mlp_forward(h.ptr, _ptr(X.contiguous()), X.shape[0], _ptr(packed), _ptr(y), _stream()))
    h.sync()
    return y


def decode_proposal(params, words, offsets, S, packed, h: Handle | None = None, out=None, sync: bool = True):
    """Proposal-bracketed decode; packed=None uses the analytic proposal (the
    logistic inverse on the dominant component) instead of the network."""
    h = h or handle(params.device)
    lat = latent(params)
    if out is None:
        out = torch.empty(lat.N, dtype=torch.int32, device=params.device)
    words = words.contiguous()
    offsets = offsets.to(torch.int64).contiguous()
    h.check(_abi.fgmm_decode_proposal(h.ptr, ctypes.byref(lat), _ptr(packed) if packed is not None else None,
                                      _ptr(words), words.numel(),
                                      _ptr(offsets), S, _ptr(out), _stream()))
    if sync:
        h.sync()
    return out
