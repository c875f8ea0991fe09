"""Torch-facing wrappers over the C ABI (include/fgmm.h).

PyTorch supplies device memory and the current CUDA stream; each function
marshals tensors into the C call of the same purpose and checks the status.
All arithmetic runs in libfgmm.so.
"""
from __future__ import annotations

import ctypes
import threading

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
    return ctypes.c_void_p(t.data_ptr() if t.numel() > 0 else 0)


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


def encode(params: torch.Tensor, symbols: torch.Tensor, S: int, h: Handle | None = None,
           words_cap: int | None = None, sync: bool = True):
    """Encode one latent into S interleaved rANS streams.

    Returns (words uint16-as-int16 tensor trimmed to its length, offsets int64
    [S/32 + 1]). With sync=False returns the untrimmed buffer, offsets and the
    device total, without synchronising."""
    h = h or handle(params.device)
    lat = latent(params)
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


def decode(params: torch.Tensor, words: torch.Tensor, offsets: torch.Tensor, S: int,
           h: Handle | None = None, out: torch.Tensor | None = None, sync: bool = True) -> torch.Tensor:
    """Decode one latent; returns int32 symbols [N]."""
    h = h or handle(params.device)
    lat = latent(params)
    words = words.contiguous()
    offsets = offsets.to(torch.int64).contiguous()
    if out is None:
        out = torch.empty(lat.N, dtype=torch.int32, device=params.device)
    h.check(_abi.fgmm_decode(h.ptr, ctypes.byref(lat), _ptr(words), words.numel(), _ptr(offsets), S, _ptr(out),
                             _stream()))
    if sync:
        h.sync()
    return out


def stats_enable(on: bool = True, h: Handle | None = None):
    h = h or handle()
    h.check(_abi.fgmm_stats_enable(h.ptr, 1 if on else 0))


def stats_read(h: Handle | None = None):
    """(cdf_evals, symbols_decoded) since the last read."""
    h = h or handle()
    out = (ctypes.c_uint64 * 2)()
    h.check(_abi.fgmm_stats_read(h.ptr, out, _stream()))
    return int(out[0]), int(out[1])
