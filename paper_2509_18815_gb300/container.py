"""A self-describing byte container for one coded latent.

The coder's output is the words of S/32 segments plus their offsets, and
decoding needs S, N and K besides the parameters, and the same coded CDF:
the approximation of Phi (Sec. III-B) the stream was coded with, the
parameter type the encoder read (bf16 parameters expand exactly to fp32, so
a decoder given the fp32 originals of bf16-coded parameters would see other
values), and, for the Gaussian single model, the scale levels its tables were
built from (Sec. II-C). This module writes all of it into one little-endian
byte string and reads it back, so a stream can be stored or sent with
everything a decoder must match:

    offset  size  field
    0       4     magic b"FGMM"
    4       2     version (2)
    6       1     coder: 0 = Gaussian mixture, 1 = Gaussian single model
    7       1     window half-width R in scales (8)
    8       8     N, symbols (uint64)
    16      4     S, streams (uint32, a positive multiple of 32)
    20      1     K, mixture components (1..4)
    21      1     Phi approximation: 0 = A&S, 1 = logistic, 2 = Polya
    22      1     parameter type: 0 = fp32, 1 = bf16
    23      1     L, GSM scale levels (1..64; 0 for the mixture coder)
    24      8     GSM levels digest: the first 8 bytes of SHA-256 of the L
                  levels as little-endian float32 (zero for the mixture coder)
    32      4     number of segments S/32 (uint32)
    36      4*G   segment lengths in words (uint32 each)
    ...     2*W   the words (uint16), W = sum of the lengths

Host-side marshalling only: it neither codes nor decodes. expect() checks a
decoder's settings against an unpacked container before it decodes.
"""
from __future__ import annotations

import hashlib
import struct

import numpy as np

MAGIC = b"FGMM"
VERSION = 2
CODER_GMM, CODER_GSM = 0, 1
PHI_AS, PHI_LOGISTIC, PHI_POLYA = 0, 1, 2
DTYPE_F32, DTYPE_BF16 = 0, 1
WINDOW_R = 8
_HEAD = struct.Struct("<4sHBBQIBBBB8sI")   # 36 bytes


def levels_digest(levels) -> bytes:
    """8-byte digest of GSM scale levels (float32, little-endian)."""
    lv = np.ascontiguousarray(_host(levels), dtype="<f4")
    return hashlib.sha256(lv.tobytes()).digest()[:8]


def pack(words, offsets, S: int, N: int, K: int, coder: int = CODER_GMM, phi: int = PHI_AS,
         dtype: int = DTYPE_F32, levels=None) -> bytes:
    """Container bytes for words (uint16 or int16 array / tensor, at least
    offsets[-1] long) and offsets (int64 [S/32 + 1]) of one latent. levels:
    the GSM scale levels (required for CODER_GSM, refused otherwise)."""
    w = _host(words).view(np.uint16)
    off = _host(offsets).astype(np.int64)
    if S <= 0 or S % 32 != 0:
        raise ValueError("S must be a positive multiple of 32")
    if not 1 <= K <= 4 or N < 0 or coder not in (CODER_GMM, CODER_GSM):
        raise ValueError("bad N, K or coder")
    if phi not in (PHI_AS, PHI_LOGISTIC, PHI_POLYA) or dtype not in (DTYPE_F32, DTYPE_BF16):
        raise ValueError("bad Phi approximation or parameter type")
    if coder == CODER_GSM:
        if levels is None or not 1 <= len(_host(levels)) <= 64:
            raise ValueError("the GSM coder needs its 1..64 scale levels")
        L, dig = len(_host(levels)), levels_digest(levels)
    else:
        if levels is not None:
            raise ValueError("scale levels belong to the GSM coder only")
        L, dig = 0, bytes(8)
    G = S // 32
    if off.shape != (G + 1,) or off[0] != 0 or np.any(np.diff(off) < 64) or off[-1] > w.size:
        raise ValueError("offsets do not describe S/32 segments of the words")
    lengths = np.diff(off)
    if lengths.max(initial=0) >= 2**32:
        raise ValueError("segment too long for the container")
    head = _HEAD.pack(MAGIC, VERSION, coder, WINDOW_R, N, S, K, phi, dtype, L, dig, G)
    return head + lengths.astype("<u4").tobytes() + w[: off[-1]].astype("<u2").tobytes()


def unpack(blob: bytes):
    """-> dict(words=uint16 array, offsets=int64 array [S/32 + 1], S, N, K,
    coder, phi, dtype, levels (L), levels_digest). Raises ValueError for
    anything that is not a whole container of this version."""
    if len(blob) < _HEAD.size:
        raise ValueError("container too short")
    magic, ver, coder, R, N, S, K, phi, dtype, L, dig, G = _HEAD.unpack_from(blob, 0)
    if magic != MAGIC or ver != VERSION:
        raise ValueError("not an fgmm container of this version")
    if R != WINDOW_R or coder not in (CODER_GMM, CODER_GSM) or not 1 <= K <= 4:
        raise ValueError("unsupported container parameters")
    if phi not in (PHI_AS, PHI_LOGISTIC, PHI_POLYA) or dtype not in (DTYPE_F32, DTYPE_BF16):
        raise ValueError("unknown Phi approximation or parameter type")
    if (coder == CODER_GSM and not 1 <= L <= 64) or (coder == CODER_GMM and (L != 0 or dig != bytes(8))):
        raise ValueError("scale levels do not match the coder")
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
    return {"words": words, "offsets": offsets, "S": S, "N": N, "K": K, "coder": coder, "phi": phi,
            "dtype": dtype, "levels": L, "levels_digest": dig}


def expect(c: dict, phi: int, dtype: int, levels=None):
    """Raises ValueError unless an unpacked container was coded with the
    Phi approximation, parameter type and (GSM) scale levels that a decoder
    is about to use: decoding with any other would not reproduce the
    encoder's CDF."""
    if c["phi"] != phi:
        raise ValueError(f"stream coded with Phi approximation {c['phi']}, decoder set to {phi}")
    if c["dtype"] != dtype:
        raise ValueError(f"stream coded from parameter type {c['dtype']}, decoder given {dtype}")
    if c["coder"] == CODER_GSM:
        if levels is None or len(_host(levels)) != c["levels"] or levels_digest(levels) != c["levels_digest"]:
            raise ValueError("GSM scale levels differ from the ones the stream was coded with")


def _host(a) -> np.ndarray:
    if hasattr(a, "detach"):   # a torch tensor
        return a.detach().cpu().numpy()
    return np.asarray(a)
