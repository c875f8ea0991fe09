"""The C-ABI library builds for sm_103a, loads without a GPU, and exports
every function include/*.h declares; the binding declares the same set."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for hdr in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(hdr).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"\b(fgmm_[a-z0-9_]+)\s*\(", text):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def lib_path():
    from paper_2509_18815_gb300 import build
    return build.build()


def test_header_declares_entry_points():
    d = _declared()
    for name in ["fgmm_create", "fgmm_encode", "fgmm_decode", "fgmm_freqs", "fgmm_sync_status"]:
        assert name in d


def test_library_exports_every_declared_symbol(lib_path):
    lib = ctypes.CDLL(lib_path)
    missing = [n for n in sorted(_declared()) if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_header(lib_path):
    from paper_2509_18815_gb300 import _abi
    assert set(_abi.SIGNATURES) == _declared()


def test_host_only_entry_points(lib_path):
    from paper_2509_18815_gb300 import _abi
    assert _abi.fgmm_encode_bound_words(0, 32) == 64
    assert _abi.fgmm_encode_bound_words(33, 32) == 3 * 32 * 2 + 64
    assert _abi.fgmm_encode_bound_words(10, 48) == -1
    assert _abi.fgmm_status_string(4) == b"corrupt or truncated stream"


def test_host_only_gsm_and_checkerboard_entry_points(lib_path):
    import numpy as np

    import oracle
    from paper_2509_18815_gb300 import _abi
    assert _abi.fgmm_gsm_tables_bytes() == 198144
    lv = np.empty(64, np.float32)
    _abi.fgmm_gsm_default_levels(lv.ctypes.data_as(ctypes.c_void_p))
    np.testing.assert_array_equal(lv.view(np.uint32), oracle.gsm_levels().view(np.uint32))
    for shape in [(3, 5, 5), (2, 4, 6), (1, 1, 1), (0, 3, 3), (4, 7, 1)]:
        assert _abi.fgmm_ckbd_anchors(*shape) == oracle.ckbd_counts(shape)[0]
    assert _abi.fgmm_ckbd_anchors(-1, 2, 2) == -1


def test_binding_refuses_host_tensors_before_any_launch():
    """Every pointer the binding hands to the C ABI is a device pointer: a
    host tensor is refused in Python, so it never reaches a kernel."""
    import torch

    from paper_2509_18815_gb300 import codec
    with pytest.raises(ValueError):
        codec._ptr(torch.zeros(4, dtype=torch.int32))
    assert codec._ptr(torch.zeros(0, dtype=torch.int32)).value is None
    with pytest.raises(ValueError):
        codec._tables(torch.zeros(198144, dtype=torch.uint8))
