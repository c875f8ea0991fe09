"""A self-describing byte container for one coded latent.

The coder's output is the words of S/32 segments plus their offsets, and
decoding needs S, N and K besides the parameters. This module writes them
into one little-endian byte string and reads them back, so a stream can be
stored or sent without side information:

    offset  size  field
    0       4     magic b"FGMM"
    4       2     version (1)
    6       1     coder: 0 = Gaussian mixture, 1 = Gaussian single model
    7       1     window half-width R in scales (8)
    8       8     N, symbols (uint64)
    16      4     S, streams (uint32, a positive multiple of 32)
    20      1     K, mixture components (1..4)
    21      3     reserved, zero
    24      4     number of segments S/32 (uint32)
    28      4*G   segment lengths in words (uint32 each)
    ...     2*W   the words (uint16), W = sum of the lengths

Host-side marshalling only: it neither codes nor decodes.
"""
from __future__ import annotations

import struct

import numpy as np

MAGIC = b"FGMM"
VERSION = 1
CODER_GMM, CODER_GSM = 0, 1
WINDOW_R = 8
_HEAD = struct.Struct("<4sHBBQIB3xI")   # 28 bytes


def pack(words, offsets, S: int, N: int, K: int, coder: int = CODER_GMM) -> bytes:
    """Container bytes for words (uint16 or int16 array / tensor, at least
    offsets[-1] long) and offsets (int64 [S/32 + 1]) of one latent."""
    w = _host(words).view(np.uint16)
    off = _host(offsets).astype(np.int64)
    if S <= 0 or S % 32 != 0:
        raise ValueError("S must be a positive multiple of 32")
    if not 1 <= K <= 4 or N < 0 or coder not in (CODER_GMM, CODER_GSM):
        raise ValueError("bad N, K or coder")
    G = S // 32
    if off.shape != (G + 1,) or off[0] != 0 or np.any(np.diff(off) < 64) or off[-1] > w.size:
        raise ValueError("offsets do not describe S/32 segments of the words")
    lengths = np.diff(off)
    if lengths.max(initial=0) >= 2**32:
        raise ValueError("segment too long for the container")
    head = _HEAD.pack(MAGIC, VERSION, coder, WINDOW_R, N, S, K, G)
    return head + lengths.astype("<u4").tobytes() + w[: off[-1]].astype("<u2").tobytes()


def unpack(blob: bytes):
    """-> dict(words=uint16 array, offsets=int64 array [S/32 + 1], S, N, K,
    coder). Raises ValueError for anything that is not a whole container."""
    if len(blob) < _HEAD.size:
        raise ValueError("container too short")
    magic, ver, coder, R, N, S, K, G = _HEAD.unpack_from(blob, 0)
    if magic != MAGIC or ver != VERSION:
        raise ValueError("not an fgmm container of this version")
    if R != WINDOW_R or coder not in (CODER_GMM, CODER_GSM) or not 1 <= K <= 4:
        raise ValueError("unsupported container parameters")
    if S <= 0 or S % 32 != 0 or G != S // 32:
        raise ValueError("inconsistent stream count")
    end_len = _HEAD.size + 4 * G
    if len(blob) < end_len:
        raise ValueError("container truncated")
    lengths = np.frombuffer(blob, dtype="<u4", count=G, offset=_HEAD.size).astype(np.int64)
    if np.any(lengths < 64):
        raise ValueError("segment shorter than its final states")
    offsets = np.zeros(G + 1, np.int64)
    np.cumsum(lengths, out=offsets[1:])
    if len(blob) != end_len + 2 * int(offsets[-1]):
        raise ValueError("container length does not match its segments")
    words = np.frombuffer(blob, dtype="<u2", offset=end_len).astype(np.uint16)
    return {"words": words, "offsets": offsets, "S": S, "N": N, "K": K, "coder": coder}


def _host(a) -> np.ndarray:
    if hasattr(a, "detach"):   # a torch tensor
        return a.detach().cpu().numpy()
    return np.asarray(a)
