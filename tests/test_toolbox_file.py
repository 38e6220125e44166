"""Toolbox files (ewos_toolbox_save / ewos_toolbox_load): the loader rejects files that are not
toolbox files of this version, or whose header does not match their size, with EWOS_EIO before
any device memory is touched (so these run without a GPU)."""
import ctypes

import pytest

from paper_2608_07017_b300 import ewos


class _Header(ctypes.Structure):
    # the file header as the library writes it (natural alignment, build report at the end)
    _fields_ = [("magic", ctypes.c_char * 8), ("version", ctypes.c_uint32), ("dim", ctypes.c_int32),
                ("precision", ctypes.c_int32), ("flags", ctypes.c_int32), ("n", ctypes.c_int64),
                ("m", ctypes.c_int64), ("p", ctypes.c_int64), ("N", ctypes.c_int64), ("eps", ctypes.c_double),
                ("seed", ctypes.c_uint64), ("instance", ctypes.c_uint32), ("reserved", ctypes.c_uint32),
                ("rep", ewos.BuildReport)]


@pytest.fixture(scope="module")
def L():
    from paper_2608_07017_b300 import build
    build.build()
    return ewos.lib()


def _load(L, path):
    h = ctypes.c_void_p()
    st = L.ewos_toolbox_load(str(path).encode(), None, ctypes.byref(h))
    assert h.value is None
    return st, L.ewos_last_error().decode()


def _header(**kw):
    h = _Header(magic=b"EWOSTBX", version=1, dim=2, precision=32, flags=0, n=10, m=10, p=4, N=100, eps=1e-4)
    for k, v in kw.items():
        setattr(h, k, v)
    return bytes(h)


def _payload_bytes(dim, precision, n, m, p, flags):
    e = 8 if precision == 64 else 4
    return (8 * n * dim + 8 * p * dim + (8 * m * dim if flags & 2 else 0) + 8 * n + e * (dim + 1) * n * m
            + e * (dim + 1) * n * p + (4 * n * p if flags & 1 else 0))


def test_missing_file(L, tmp_path):
    st, msg = _load(L, tmp_path / "none.ewtb")
    assert st == ewos.EIO and "cannot open" in msg


def test_not_a_toolbox_file(L, tmp_path):
    f = tmp_path / "junk.ewtb"
    f.write_bytes(b"this is not a toolbox" * 20)
    st, msg = _load(L, f)
    assert st == ewos.EIO and "not a toolbox file" in msg


def test_header_size_mismatch(L, tmp_path):
    f = tmp_path / "short.ewtb"
    body = _payload_bytes(2, 32, 10, 10, 4, 0)
    f.write_bytes(_header() + bytes(body - 4))          # 4 bytes short
    st, msg = _load(L, f)
    assert st == ewos.EIO and "size" in msg
    f.write_bytes(_header() + bytes(body + 8))          # 8 bytes too many
    assert _load(L, f)[0] == ewos.EIO


@pytest.mark.parametrize("bad", [dict(version=2), dict(dim=4), dict(precision=16), dict(n=0), dict(flags=4),
                                 dict(m=12)])   # m != n needs the V-centres flag
def test_inconsistent_header(L, tmp_path, bad):
    f = tmp_path / "bad.ewtb"
    f.write_bytes(_header(**bad) + bytes(_payload_bytes(2, 32, 10, 10, 4, 0)))
    st, msg = _load(L, f)
    assert st == ewos.EIO and "header" in msg


def test_null_arguments(L, tmp_path):
    h = ctypes.c_void_p()
    assert L.ewos_toolbox_load(None, None, ctypes.byref(h)) == ewos.EINVAL
    assert L.ewos_toolbox_load(b"x", None, None) == ewos.EINVAL
    assert L.ewos_toolbox_save(None, b"x") == ewos.EINVAL
