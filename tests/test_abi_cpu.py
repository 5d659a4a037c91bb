"""Host-side checks of the C ABI that need no GPU: the library loads, exports
every entry point that include/qsg.h declares, and validates shapes."""
from __future__ import annotations

import ctypes
import os
import re

import numpy as np
import pytest

from paper_2310_07486_gb300 import qsg as Q

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_entry_points():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names.update(re.findall(r"\b(qsg_[a-z0-9_]+)\s*\(", text))
    return sorted(names)


def test_library_exports_every_declared_symbol():
    lib = Q.load_library()
    names = declared_entry_points()
    assert len(names) >= 15
    for n in names:
        assert hasattr(lib, n), n
    assert set(Q.exported_symbols()) <= set(names)


@pytest.mark.parametrize("bad", [
    Q.Shape(7, 8, 1, 1, 1), Q.Shape(0, 8, 1, 1, 1), Q.Shape(8, 7, 1, 1, 1), Q.Shape(8, 8, 0, 1, 1),
    Q.Shape(8, 8, 1, 0, 1), Q.Shape(8, 8, 1, 1, 0), Q.Shape(8, 8, 1, 1, 129), Q.Shape(34, 8, 1, 1, 1),
    Q.Shape(8, 8, 1, 1, 1, algo=2), Q.Shape(8, 8, 1, 1, 1, boundary=3)])
def test_invalid_shapes_are_rejected(bad):
    assert Q.qsg_workspace_bytes([bad]) == 0


def test_workspace_grows_with_the_state():
    small = Q.qsg_workspace_bytes([Q.Shape(8, 16, 64, 2, 2)])
    big = Q.qsg_workspace_bytes([Q.Shape(8, 32, 64, 2, 2)])
    assert small > 0 and big > small
    state = 24 * 24 * 2048 * 2 * 4 * 32 * 8
    assert Q.qsg_workspace_bytes([Q.Shape(24, 2048, 128, 4, 32, Q.HEATBATH)]) > state


def test_create_rejects_missing_workspace():
    lib = Q.load_library()
    arr = Q._shape_array([Q.Shape(8, 8, 1, 1, 1)])
    h = ctypes.c_void_p()
    st = lib.qsg_create(ctypes.byref(h), ctypes.cast(arr, ctypes.c_void_p), 1, None, 0, None)
    assert st == -6 and not h.value
    st = lib.qsg_create(ctypes.byref(h), ctypes.cast(arr, ctypes.c_void_p), 0, None, 0, None)
    assert st == -1


def test_calls_on_null_context_fail_cleanly():
    lib = Q.load_library()
    assert lib.qsg_sweep(None, 1) == -1
    assert lib.qsg_tempering_swap(None) == -1
    assert lib.qsg_measure_correlators(None) == -1
    assert lib.qsg_read_correlators(None, 0, None, None, None, None) == -1
    assert lib.qsg_read_correlators_async(None, 0, None, None, None, None, None) == -1
    assert lib.qsg_wait_correlators(None) == -1
    assert lib.qsg_strerror(-4) == b"bounded device wait gave up"


def test_static_scratch_checks_shape_and_limits_before_buffers():
    """The allocation-free sweep rejects shapes beyond its fixed scratch with
    QSG_ERR_WORKSPACE before it looks at the buffers; with null buffers a
    regressed limit check would answer QSG_ERR_ARG instead, and never launch."""
    lib = Q.load_library()

    def call(shape, ladder):
        sh = shape.c()
        lad = np.ascontiguousarray(ladder, dtype=np.float64)
        return lib.qsg_sweep_static_scratch(None, None, None, ctypes.byref(sh), 0, Q._ptr(lad), 1, 0, 1, None)

    lad = np.linspace(0.1, 0.5, 129)
    assert call(Q.Shape(8, 24, 64, 1, 1), [0.3]) == -2  # L_tau not a multiple of 16
    assert call(Q.Shape(7, 16, 64, 1, 1), [0.3]) == -2  # odd L
    assert call(Q.Shape(8, 16, 64, 1, 129), lad) == -6  # more ladder positions than the static table
    assert call(Q.Shape(8, 16, 64 * 512, 64, 128), lad[:128]) == -6  # more slots x chunks than the counters
    assert call(Q.Shape(8, 16, 64, 1, 1), [0.3]) == -1  # null buffers
    sh = Q.Shape(8, 16, 64, 1, 1).c()
    assert lib.qsg_sweep_static_scratch(None, None, None, None, 0, None, 1, 0, 1, None) == -1  # null shape


def test_static_scratch_wrapper_requires_device_tensors():
    torch = pytest.importorskip("torch")

    class _Stream:  # stands in for a CUDA stream; the wrapper raises before using it
        device = torch.device("cuda", 0)
        cuda_stream = 0

    t = torch.zeros(8 * 8 * 16, dtype=torch.int64)
    with pytest.raises(Q.QSGError) as e:
        Q.qsg_sweep_static_scratch(t, t[:64], t[:64], Q.Shape(8, 16, 64, 1, 1), 0, [0.3], 1, 0, 1, stream=_Stream())
    assert e.value.status == -1
