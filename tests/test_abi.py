"""Host-side checks of the C ABI: the library builds, loads, exports every entry point that
include/sfft.h declares, and validates descriptors without touching a GPU."""
import ctypes
import os
import re

import pytest

from paper_2509_18544_gb300 import build as sfft_build
from paper_2509_18544_gb300 import sfft

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    sfft_build.build()
    return sfft.load_library()


def _declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if not fn.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", fn)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*(sfft_[A-Za-z0-9_]+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return names


def test_every_declared_symbol_is_exported(lib):
    declared = _declared_functions()
    assert {"sfft_plan", "sfft_fit", "sfft_subtract", "sfft_batch", "sfft_normal"} <= declared
    for name in sorted(declared):
        assert hasattr(lib, name), name
    assert set(sfft.EXPORTED) <= declared


def test_workspace_size_and_validation_on_host(lib):
    d = sfft.make_desc(4088, 4088, 11, 2, 2)
    ws = sfft.sfft_workspace_size(d)
    # spectra dominate: 18 segments x 129 bins x 4088 rows x 10 base images x 8 bytes; the rest
    # is the y-correlation partials (at most 16 CTAs per frequency x 129 x 63 pairs x 128 x 16
    # bytes), the refinement's residual image and its compact spectrum (67 + 76 MB) and small
    # tables
    spec = 18 * 129 * 4088 * 10 * 8
    assert spec < ws < spec + 16 * 129 * 63 * 128 * 16 + 300 * 2 ** 20
    for bad in (dict(L=4), dict(L=0), dict(ny=3, L=5), dict(dk=-1), dict(dtype=7), dict(precision=9),
                dict(pitch=10, nx=20)):
        kw = dict(ny=64, nx=64, L=5, dk=0, db=0)
        kw.update(bad)
        with pytest.raises(sfft.SfftError) as ei:
            sfft.sfft_workspace_size(sfft.make_desc(**kw))
        assert ei.value.status == sfft.ERR_INVALID_ARG, bad


def test_status_strings(lib):
    for s in range(8):
        assert lib.sfft_status_string(s)
    assert sfft.OK == 0 and sfft.ERR_NOT_SPD == 4


def test_null_arguments_rejected_without_gpu(lib):
    assert lib.sfft_plan(None, None, None) == sfft.ERR_INVALID_ARG
    h = ctypes.c_void_p()
    assert lib.sfft_plan(ctypes.byref(h), None, None) == sfft.ERR_INVALID_ARG
    assert lib.sfft_n_unknowns(None, None) == sfft.ERR_INVALID_ARG
    assert lib.sfft_fit(None, None, None, None, None, None, None) == sfft.ERR_INVALID_ARG
    assert lib.sfft_subtract(None, None, None, None, None) == sfft.ERR_INVALID_ARG
    lib.sfft_destroy(None)


def test_cnn_file_calls_reject_null_arguments_without_gpu(lib):
    assert lib.sfft_cnn_save(None, b"/nonexistent") == sfft.ERR_INVALID_ARG
    assert lib.sfft_cnn_load(None, b"/nonexistent") == sfft.ERR_INVALID_ARG
    lib.sfft_cnn_destroy(None)
