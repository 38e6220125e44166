"""The C ABI library loads and exports every entry point that include/ewos.h declares; argument
checks that need no device return EWOS_EINVAL (no compute call is made here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "ewos.h")


@pytest.fixture(scope="module")
def L():
    from paper_2608_07017_b300 import build, ewos
    build.build()
    return ewos.lib()


def _declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(ewos_[a-z0-9_]+)\s*\(", src)))


def test_header_symbols_are_exported(L):
    names = _declared()
    assert "ewos_toolbox_build" in names and "ewos_solve" in names
    for n in names:
        assert hasattr(L, n), n


def test_status_strings(L):
    assert L.ewos_status_string(0) == b"ok"
    assert L.ewos_status_string(4) == b"singular matrix"
    assert L.ewos_status_string(99) == b"unknown status"


def test_invalid_arguments_are_rejected_before_any_device_work(L):
    from paper_2608_07017_b300 import ewos
    import numpy as np
    h = ctypes.c_void_p()
    prm = np.array([0.0, 0.0, 1.0])
    dom = ewos._Domain(0, 2, prm.ctypes.data, 3)
    x = np.zeros((4, 2)); z = np.zeros((3, 2))
    # walks = 0, eps <= 0, NULL nodes
    assert L.ewos_toolbox_build(ctypes.byref(dom), x.ctypes.data, 4, z.ctypes.data, 3, 0, 1e-3, 0, None, ctypes.byref(h)) == ewos.EINVAL
    assert L.ewos_toolbox_build(ctypes.byref(dom), x.ctypes.data, 4, z.ctypes.data, 3, 10, 0.0, 0, None, ctypes.byref(h)) == ewos.EINVAL
    assert L.ewos_toolbox_build(ctypes.byref(dom), None, 4, z.ctypes.data, 3, 10, 1e-3, 0, None, ctypes.byref(h)) == ewos.EINVAL
    # a node outside the unit disk
    xo = np.array([[0.0, 0.0], [1.5, 0.0]])
    assert L.ewos_toolbox_build(ctypes.byref(dom), xo.ctypes.data, 2, z.ctypes.data, 3, 10, 1e-3, 0, None, ctypes.byref(h)) == ewos.EINVAL
    assert b"not inside" in L.ewos_last_error()
    # bad domain: polygon in 3D, ball with the wrong parameter count
    dom3 = ewos._Domain(2, 3, prm.ctypes.data, 3)
    assert L.ewos_toolbox_build(ctypes.byref(dom3), x.ctypes.data, 4, z.ctypes.data, 3, 10, 1e-3, 0, None, ctypes.byref(h)) == ewos.EINVAL
    domb = ewos._Domain(0, 2, prm.ctypes.data, 2)
    assert L.ewos_toolbox_build(ctypes.byref(domb), x.ctypes.data, 4, z.ctypes.data, 3, 10, 1e-3, 0, None, ctypes.byref(h)) == ewos.EINVAL
    # solve / get with NULL handles
    assert L.ewos_solve(None, None, None, None, 0, None) == ewos.EINVAL
    assert L.ewos_toolbox_get(None, 0, None, 0, 0) == ewos.EINVAL
    assert L.ewos_debug_philox(None, None, None, 1) == ewos.EINVAL
    # the Euler-Lagrange route and the operator estimates with NULL handles
    s = np.zeros(4)
    pb = ewos._Problem()
    assert L.ewos_gradient(None, ctypes.byref(pb), s.ctypes.data, s.ctypes.data) == ewos.EINVAL
    assert L.ewos_gradient(None, None, None, None) == ewos.EINVAL
    o = ewos.AdamOpts(1e-3, 0.9, 0.999, 1e-10, 10, 0.0, 0)
    assert L.ewos_minimize_adam(None, ctypes.byref(pb), ctypes.byref(o), s.ctypes.data, None, None) == ewos.EINVAL
    assert L.ewos_operators(None, ctypes.byref(pb), s.ctypes.data, None, 0, None) == ewos.EINVAL


def test_binding_fails_loudly_without_library(monkeypatch, tmp_path):
    from paper_2608_07017_b300 import ewos
    monkeypatch.setattr(ewos, "_lib", None)
    monkeypatch.setattr(ewos, "LIB_PATH", str(tmp_path / "missing.so"))
    with pytest.raises(ImportError):
        ewos.lib()
