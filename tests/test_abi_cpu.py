"""CPU checks of the C ABI: the library builds, loads, exports every symbol
that include/tde.h declares, and rejects calls without a usable context.  No
compute call is made (there may be no GPU)."""
import ctypes
import os
import re

import pytest

from paper_2509_19974_gb300 import build, tde

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "tde.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(tde_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return tde.load()


def test_header_declares_the_binding_exports():
    assert _declared() == sorted(tde.EXPORTS)


def test_library_exports_every_declared_symbol(lib):
    for name in _declared():
        assert hasattr(lib, name), name


def test_null_context_is_rejected(lib):
    assert lib.tde_quantize(None, None, 0, 1, None, None) == tde.TDE_ERR_INVALID
    assert lib.tde_ctx_sync(None, None) == tde.TDE_ERR_INVALID
    assert lib.tde_ctx_destroy(None) == tde.TDE_OK
    assert lib.tde_last_error(None) == b"null context"
    assert lib.tde_selftest_wait_timeout(None, None) == tde.TDE_ERR_INVALID
    assert lib.tde_ctx_set_ntt_primes(None, 0) == tde.TDE_ERR_INVALID


def test_bad_device_is_a_cuda_error(lib):
    h = ctypes.c_void_p()
    assert lib.tde_ctx_create(-1, ctypes.byref(h)) == tde.TDE_ERR_CUDA
    assert h.value is None


def test_autotune_entries_round_trip_and_null_context(lib):
    d = {"bits": 2, "log2_n": 16, "log2_lags": 17, "engine": "mma",
         "ns_per_pair": {"popc": 1000.0, "mma": 50.0, "ntt": None}}
    assert tde.entry_to_dict(tde.dict_to_entry(d)) == d
    arr = (tde.TuneEntry * 1)(tde.dict_to_entry(d))
    assert lib.tde_autotune_load(None, ctypes.addressof(arr), 1) == tde.TDE_ERR_INVALID
    assert lib.tde_autotune(None, 2, None, None, 1, 1) == tde.TDE_ERR_INVALID
    assert lib.tde_ctx_pick_engine(None, 2, 100, 100, 10) == -1
    cnt = ctypes.c_int()
    assert lib.tde_autotune_table(None, None, 0, ctypes.byref(cnt)) == tde.TDE_ERR_INVALID


def test_default_autotune_points_are_valid():
    pts = tde.DEFAULT_TUNE_POINTS
    assert len(set(pts)) == len(pts)
    for n, lags in pts:
        assert n >= 1 and 1 <= lags <= 2 * n - 1
