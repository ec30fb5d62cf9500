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


def test_every_entry_point_rejects_null_handles_on_the_host(lib):
    """Each context / trainer entry point checks its handle (and the arguments it
    validates before any device work) on the host: INVALID_ARG with a message that
    names the call, no CUDA call made (this runs without a GPU)."""
    sd = lib.crom_step_desc(0, 1, 1e-5)
    sdp = ctypes.byref(sd)
    calls = {
        "crom_set_weights": (None, None, 0, 0, None),
        "crom_decode_tc": (None, 1, 1, None, None, None, 1, 1, None, None),
        "crom_device_flags": (None, None, None),
        "crom_rollout": (None, sdp, 1, 1, 1, None, None, None, None, None, 1, 1, None, None),
        "crom_step_host": (None, sdp, 1, 1, None, None, None, None, None, 1, 1, None, None),
        "crom_step_noalloc": (None, sdp, 1, None, None, None, None, None, 1, 1, None, None),
        "crom_set_step_tiles": (None, 8, 16),
        "crom_get_step_tiles": (None, None, None, None),
        "crom_autotune": (None, sdp, 1, None, None, None, None, None, 1, 1, None, None),
        "crom_tangent_velocity": (None, 1, None, None, 1e-3, None, None, 1, None, None),
        "crom_robust_samples": (None, sdp, 1, 1, None, None, 1, 1, None, None, 1, None, 1, 0.0, 8, None, None,
                                None, None),
        "crom_trainer_param_count": (None, None),
        "crom_trainer_set_precision": (None, 0),
        "crom_trainer_set_params": (None, None, 0, 0, None),
        "crom_trainer_get_params": (None, None, 0, 0, None),
        "crom_trainer_get_grads": (None, None, 0, 0, None),
        "crom_train_step": (None, None, None, None, 1e-3, None, None),
        "crom_encode": (None, 1, None, None, None),
        "crom_trainer_save": (None, b"/nonexistent/ckpt"),
        "crom_trainer_load": (None, b"/nonexistent/ckpt"),
    }
    for name, args in calls.items():
        assert name in lib.EXPORTED, name
        assert lib.raw_call(name, *args) == lib.CROM_ERR_INVALID_ARG, name
        assert name in lib.last_error(), (name, lib.last_error())


def test_full_order_and_watchdog_argument_checks_on_the_host(lib):
    """crom_fom_step validates kind, sizes and dt, and crom_stream_wait its timeout,
    before touching a device."""
    bad = [(-1, 1, 8, 8, 1e-3), (99, 1, 8, 8, 1e-3), (lib.CROM_FOM_HEAT2D_NEUMANN, 1, 2, 2, 1e-3),
           (lib.CROM_FOM_HEAT2D_NEUMANN, 1, 8, 7, 1e-3), (lib.CROM_FOM_HEAT2D_NEUMANN, 1, 8, 8, 0.0),
           (lib.CROM_FOM_HEAT2D_NEUMANN, 1, 8, 8, float("nan")), (lib.CROM_FOM_HEAT2D_NEUMANN, -1, 8, 8, 1e-3),
           (lib.CROM_FOM_HEAT2D_NEUMANN, 70000, 8, 8, 1e-3)]
    for kind, nb, nx, ny, dt in bad:
        assert lib.raw_call("crom_fom_step", kind, nb, nx, ny, None, None, None, dt, 1, None, None, None) == \
            lib.CROM_ERR_INVALID_ARG, (kind, nb, nx, ny, dt)
    # nothing to do is not an error, and needs no device
    assert lib.raw_call("crom_fom_step", lib.CROM_FOM_HEAT2D_NEUMANN, 0, 8, 8, None, None, None, 1e-3, 1,
                        None, None, None) == lib.CROM_OK
    assert lib.raw_call("crom_stream_wait", None, -1.0) == lib.CROM_ERR_INVALID_ARG
    assert lib.raw_call("crom_stream_wait", None, float("nan")) == lib.CROM_ERR_INVALID_ARG
