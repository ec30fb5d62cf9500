"""The C-ABI library builds, loads and exports every symbol include/crom.h declares (CPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    with open(os.path.join(ROOT, "include", "crom.h")) as f:
        text = f.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(crom_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_2206_02607_gb300 import build
    build()
    from paper_2206_02607_gb300 import crom
    return crom


def test_every_declared_symbol_is_exported(lib):
    names = declared_symbols()
    assert set(names) == set(lib.EXPORTED)
    raw = ctypes.CDLL(lib.LIB_PATH)
    for n in names:
        assert hasattr(raw, n), n


def test_version_and_error_string(lib):
    assert lib.crom_version() == 10000
    assert isinstance(lib.last_error(), str)


def test_create_rejects_bad_shapes_without_touching_the_device(lib):
    h = ctypes.c_void_p()
    for bad in [(0, 8, 128, 5), (2, 0, 128, 5), (2, 8, 100, 5), (2, 8, 128, 0), (4, 8, 128, 5)]:
        d = lib.crom_decoder_desc(*bad)
        code = lib.raw_call("crom_create", ctypes.byref(h), ctypes.byref(d), 0)
        assert code == lib.CROM_ERR_INVALID_ARG
    assert lib.raw_call("crom_create", None, None, 0) == lib.CROM_ERR_INVALID_ARG


def test_null_context_calls_fail_cleanly(lib):
    sd = lib.crom_step_desc(0, 1, 1e-5)
    assert lib.raw_call("crom_step", None, ctypes.byref(sd), 0, 1, None, None, None, None, None, 0, 1,
                        None, None) == lib.CROM_ERR_INVALID_ARG
    assert lib.raw_call("crom_decode", None, 1, None, None, None, 1, 1, None, None) == lib.CROM_ERR_INVALID_ARG
    assert lib.raw_call("crom_reconstruct", None, 0, 1, None, 1, None, None, None) == lib.CROM_ERR_INVALID_ARG
    assert lib.raw_call("crom_destroy", None) == lib.CROM_OK


def test_no_device_is_a_cuda_error_not_a_fallback(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = ctypes.c_void_p()
    d = lib.crom_decoder_desc(2, 8, 128, 5)
    assert lib.raw_call("crom_create", ctypes.byref(h), ctypes.byref(d), 0) == lib.CROM_ERR_CUDA


def test_missing_library_fails_loudly(tmp_path):
    """Without the built library the binding raises instead of computing anything."""
    from paper_2206_02607_gb300 import crom
    with pytest.raises(ImportError):
        crom.load_library(str(tmp_path / "libcrom.so"))


def test_checkpoint_checksum_is_crc32(lib):
    """The checkpoint checksum is CRC-32 (IEEE): the standard check value of the
    ASCII digits 1..9 is 0xCBF43926, and random buffers agree with zlib's
    independent implementation (host code only, no device)."""
    import zlib
    import numpy as np
    assert lib.crom_crc32(b"123456789") == 0xCBF43926
    assert lib.crom_crc32(b"") == 0
    rng = np.random.default_rng(0)
    for n in (1, 7, 64, 1000, 65537):
        data = rng.integers(0, 256, size=n, dtype=np.uint8).tobytes()
        assert lib.crom_crc32(data) == zlib.crc32(data)
