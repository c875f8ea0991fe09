"""fgmm_encode_noalloc: the allocation-free encoder for callers that cannot
allocate device memory while they encode (host callbacks, real-time loops,
plugins whose host application owns every device allocation).

Called through the C ABI, it must give exactly the words, offsets and word
count of fgmm_encode (integer output: the tolerance is equality), on two
calls in a row with different inputs, and again after that, whatever the
shared scratch array holds from earlier calls. Requests that do not fit its
fixed scratch are rejected before anything is launched. This file is
collected last so that a run stopping at the first failure has already run
every other test; it also passes alone in a fresh process.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_2509_18815_gb300 import synth
from tests.gpu_util import dev_i32, dev_params, need_gpu

pytestmark = pytest.mark.gpu


def _encode_noalloc(dp, ds, S):
    from paper_2509_18815_gb300 import _abi, codec
    lat = codec.latent(dp)
    cap = codec.encode_bound_words(lat.N, S)
    words = torch.full((cap,), -1, dtype=torch.int16, device="cuda")
    offsets = torch.full((S // 32 + 1,), -1, dtype=torch.int64, device="cuda")
    total = torch.full((1,), -1, dtype=torch.int64, device="cuda")
    status = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    st = _abi.fgmm_encode_noalloc(ctypes.byref(lat), ds.data_ptr(), S, words.data_ptr(), cap, offsets.data_ptr(),
                                  total.data_ptr(), status.data_ptr(), stream)
    assert st == _abi.FGMM_OK
    torch.cuda.current_stream().synchronize()
    assert int(status.item()) == _abi.FGMM_OK
    n = int(total.item())
    return words[:n].cpu().numpy(), offsets.cpu().numpy(), n


def _encode_reference(dp, ds, S):
    from paper_2509_18815_gb300 import codec
    words, offsets = codec.encode(dp, ds, S)
    return words.cpu().numpy(), offsets.cpu().numpy(), int(words.numel())


def test_noalloc_matches_encode_on_consecutive_calls():
    need_gpu()
    a = synth.make_latent(192, 16, 16, 3, seed=1001)
    b = synth.make_latent(64, 16, 24, 4, seed=77, escape_stress=0.01)
    cases = [(dev_params(a.params), dev_i32(a.symbols), 32),
             (dev_params(b.params, bf16=True), dev_i32(b.symbols), 256),
             (dev_params(a.params), dev_i32(a.symbols), 32)]
    for dp, ds, S in cases:
        w1, o1, n1 = _encode_noalloc(dp, ds, S)
        w0, o0, n0 = _encode_reference(dp, ds, S)
        assert n1 == n0
        np.testing.assert_array_equal(o1, o0)
        np.testing.assert_array_equal(w1, w0)


def test_noalloc_rejects_requests_beyond_its_scratch():
    need_gpu()
    from paper_2509_18815_gb300 import _abi, codec
    N = 4 << 20
    dp = torch.zeros((3, 3, N), dtype=torch.float32, device="cuda")
    ds = torch.zeros(N, dtype=torch.int32, device="cuda")
    lat = codec.latent(dp)
    out = torch.zeros(16, dtype=torch.int64, device="cuda")
    st = _abi.fgmm_encode_noalloc(ctypes.byref(lat), ds.data_ptr(), 1024, out.data_ptr(), 0, out.data_ptr(),
                                  out.data_ptr(), out.data_ptr(), None)
    assert st == _abi.FGMM_ERR_TOO_LARGE
    assert b"scratch" in _abi.fgmm_status_string(st)


def _scratch_bytes(N, S):
    """The scratch a request needs, by the size rule the header states:
    align256(4 N) + align256(2 (S/32) align8(96 ceil(N/S) + 64)) + 8 (S/32)."""
    def a(x, m):
        return (x + m - 1) // m * m
    T = -(-N // S)
    return a(4 * N, 256) + a(2 * (S // 32) * a(96 * T + 64, 8), 256) + 8 * (S // 32)


def test_noalloc_at_the_largest_request_that_fits():
    """At S = 1024 the largest N whose scratch fits the fixed array (found
    from the header's size rule) encodes exactly as fgmm_encode does, and
    N + S symbols are rejected as too large without any launch."""
    need_gpu()
    from paper_2509_18815_gb300 import _abi, codec
    S, limit = 1024, _abi.FGMM_NOALLOC_SCRATCH_BYTES
    lo, hi = 0, 1 << 24
    while hi - lo > 1:
        mid = (lo + hi) // 2
        if _scratch_bytes(mid, S) <= limit:
            lo = mid
        else:
            hi = mid
    N = lo
    assert _scratch_bytes(N, S) <= limit < _scratch_bytes(N + S, S)
    lat = synth.make_latent(1, 1, N, 3, seed=78)
    dp, ds = dev_params(lat.params), dev_i32(lat.symbols)
    w1, o1, n1 = _encode_noalloc(dp, ds, S)
    w0, o0, n0 = _encode_reference(dp, ds, S)
    assert n1 == n0
    np.testing.assert_array_equal(o1, o0)
    np.testing.assert_array_equal(w1, w0)
    big = synth.make_latent(1, 1, N + S, 3, seed=79)
    dpb, dsb = dev_params(big.params), dev_i32(big.symbols)
    lat_b = codec.latent(dpb)
    out = torch.zeros(16, dtype=torch.int64, device="cuda")
    st = _abi.fgmm_encode_noalloc(ctypes.byref(lat_b), dsb.data_ptr(), S, out.data_ptr(), 0, out.data_ptr(),
                                  out.data_ptr(), out.data_ptr(), None)
    assert st == _abi.FGMM_ERR_TOO_LARGE
