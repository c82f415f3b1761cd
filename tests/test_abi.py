"""The C-ABI library builds, loads and exports every entry point of
include/moco.h; host-side validation rejects bad arguments before any launch.
No compute call runs here (no GPU needed)."""
import ctypes
import os
import re

import pytest

from paper_1506_06039_gb300 import binding, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return binding.lib()


def header_entry_points():
    text = open(os.path.join(ROOT, "include", "moco.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(moco_[a-z_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = header_entry_points()
    for required in ("moco_plan", "moco_align_stack", "moco_cost_surface", "moco_cost_backward",
                     "moco_plan_destroy", "moco_status_string"):
        assert required in names
    assert set(names) == set(binding.EXPORTS)


def test_library_exports_every_declared_symbol(lib):
    for name in header_entry_points():
        assert hasattr(lib, name), name


def test_status_strings(lib):
    assert binding.moco_status_string(0) == "MOCO_OK"
    assert binding.moco_status_string(1) == "MOCO_ERR_INVALID_ARG"
    assert binding.moco_status_string(5) == "MOCO_ERR_TIMEOUT"
    assert binding.moco_status_string(99) == "MOCO_ERR_UNKNOWN"


def _plan_status(lib, shape, template_ptr=0x1000):
    arr = (binding.MocoShape * 1)(shape)
    tp = (ctypes.c_void_p * 1)(template_ptr)
    out = ctypes.c_void_p(123)
    st = lib.moco_plan(arr, 1, tp, None, ctypes.byref(out))
    return st, out.value, lib.moco_last_error().decode()


@pytest.mark.parametrize("shape,msg", [
    (binding.MocoShape(128, 100, 10, -1, 0, 0, 0, 0), "n % 8"),       # n not a multiple of 8
    (binding.MocoShape(128, 128, 0, -1, 0, 0, 0, 0), "w >= 1"),        # empty window
    (binding.MocoShape(128, 128, 65, -1, 0, 0, 0, 0), "2w-1"),         # window larger than the image
    (binding.MocoShape(512, 512, 129, -1, 0, 0, 0, 0), "2w-1"),        # on the searched grid
    (binding.MocoShape(128, 128, 10, 5, 0, 0, 0, 0), "levels"),          # at most four levels
    (binding.MocoShape(128, 128, 10, 3, 0, 0, 0, 0), "2w-1"),            # 16 x 16 level-3 grid
    (binding.MocoShape(128, 128, 10, -1, 7, 0, 0, 0), "template_dtype"),
    (binding.MocoShape(128, 128, 10, -1, 0, 9, 0, 0), "xcorr"),
    (binding.MocoShape(128, 128, 10, -1, 0, 0, 0, 1), "reserved"),
    (binding.MocoShape(0, 128, 1, -1, 0, 0, 0, 0), "m"),
])
def test_plan_rejects_invalid_shapes(lib, shape, msg):
    st, handle, err = _plan_status(lib, shape)
    assert st == binding.MOCO_ERR_INVALID_ARG
    assert handle is None
    assert msg in err


def test_plan_rejects_unsupported(lib):
    st, handle, err = _plan_status(lib, binding.MocoShape(512, 512, 10, -1, 1, 0, 0, 0))
    assert st == binding.MOCO_ERR_UNSUPPORTED and "levels" in err
    st, handle, err = _plan_status(lib, binding.MocoShape(4096, 4096, 64, 0, 0, binding.XCORR_FFT_FP32, 0, 0))
    assert st == binding.MOCO_ERR_UNSUPPORTED and "FFT" in err
    # 384 x 384 without a level, w = 150: the FFT length fits (576) but the
    # combine's W x W costs (299^2 floats) do not fit in shared memory, and
    # W > 256 rules out the direct form.
    st, handle, err = _plan_status(lib, binding.MocoShape(384, 384, 150, 0, 0, binding.XCORR_FFT_FP32, 0, 0))
    assert st == binding.MOCO_ERR_UNSUPPORTED and "shared memory" in err
    st, handle, err = _plan_status(lib, binding.MocoShape(384, 384, 150, 0, 0, 0, 0, 0))
    assert st == binding.MOCO_ERR_UNSUPPORTED and "no cross-term form" in err


def test_null_arguments(lib):
    out = ctypes.c_void_p()
    assert lib.moco_plan(None, 1, None, None, ctypes.byref(out)) == binding.MOCO_ERR_INVALID_ARG
    assert lib.moco_plan(None, 1, None, None, None) == binding.MOCO_ERR_INVALID_ARG
    assert lib.moco_align_stack(None, None, 0, None) == binding.MOCO_ERR_INVALID_ARG
    assert lib.moco_cost_surface(None, 0, None, 1, None, None) == binding.MOCO_ERR_INVALID_ARG
    assert lib.moco_plan_destroy(None) == binding.MOCO_ERR_INVALID_ARG
    assert lib.moco_plan_query(None, 0, None) == binding.MOCO_ERR_INVALID_ARG
    assert lib.moco_align_host(None, 0, None, 1, None, None) == binding.MOCO_ERR_INVALID_ARG


def test_alu_peak_rejects_bad_arguments(lib):
    rate = ctypes.c_double(0.0)
    assert lib.moco_alu_peak(7, ctypes.c_void_p(16), ctypes.byref(rate), None) == binding.MOCO_ERR_INVALID_ARG
    assert lib.moco_alu_peak(binding.PEAK_DP2A, None, ctypes.byref(rate), None) == binding.MOCO_ERR_INVALID_ARG
    assert lib.moco_alu_peak(binding.PEAK_FP32_FMA, ctypes.c_void_p(16), None, None) == binding.MOCO_ERR_INVALID_ARG
    assert lib.moco_alu_peak(binding.PEAK_FP32_FMA, ctypes.c_void_p(18), ctypes.byref(rate), None) == \
        binding.MOCO_ERR_INVALID_ARG  # sink not 4-byte aligned


def test_binding_fails_loudly_without_library(monkeypatch, tmp_path):
    monkeypatch.setattr(binding, "_lib", None)
    monkeypatch.setattr(binding._build, "LIB", str(tmp_path / "missing.so"))
    with pytest.raises(RuntimeError, match="missing"):
        binding.lib()
