"""Host-side checks of the C ABI (no GPU needed): the library loads, exports
every function include/rsvd.h declares, answers workspace queries, and rejects
invalid arguments with the documented negative codes before any launch."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1710_01463_gb300 import build, _lib
    try:
        build.build_library()
    except RuntimeError as e:  # pragma: no cover - toolkit missing
        pytest.skip(str(e))
    return _lib.load()


def header_functions():
    src = open(os.path.join(ROOT, "include", "rsvd.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^(?:const\s+)?\w+\s*\*?\s*(\w+)\s*\(", src, flags=re.M)))


def test_exports_every_declared_function(lib):
    from paper_1710_01463_gb300 import _lib
    names = header_functions()
    assert set(names) == set(_lib.EXPORTED)
    for n in names:
        assert hasattr(lib, n)


def test_status_strings(lib):
    for code in (0, -1, -2, -3, -4, -6, 1):
        assert len(lib.rsvd_status_string(code)) > 0


def params(k=32, p=8, q=2, prec=0):
    from paper_1710_01463_gb300 import _lib
    return _lib.RsvdParams(k, p, q, prec, 201, 0, 0, 0)


def test_workspace_size_grows_with_size(lib):
    sz1, sz2 = ctypes.c_size_t(0), ctypes.c_size_t(0)
    assert lib.rsvd_workspace_size(256, 256, ctypes.byref(params()), ctypes.byref(sz1)) == 0
    assert lib.rsvd_workspace_size(1024, 1024, ctypes.byref(params()), ctypes.byref(sz2)) == 0
    assert 0 < sz1.value < sz2.value
    assert sz1.value % 256 == 0


@pytest.mark.parametrize("m,n,k,p,q,prec,code", [
    (0, 10, 1, 0, 0, 0, -1), (10, 10, 0, 0, 0, 0, -1), (10, 10, 11, 0, 0, 0, -1),
    (10, 10, 5, -1, 0, 0, -1), (10, 10, 5, 2, -1, 0, -1), (10, 10, 5, 2, 1, 7, -3),
    (4000, 4000, 1020, 10, 1, 0, -1)])
def test_invalid_arguments_rejected(lib, m, n, k, p, q, prec, code):
    sz = ctypes.c_size_t(0)
    assert lib.rsvd_workspace_size(m, n, ctypes.byref(params(k, p, q, prec)), ctypes.byref(sz)) == code


def test_truncate_rejects_before_launch(lib):
    fake = ctypes.c_void_p(4096)
    par = params(5, 2, 1)
    # leading dimension too small
    assert lib.rsvd_truncate(10, 10, fake, 9, ctypes.byref(par), fake, fake, 5, fake, 10, fake, 1 << 20, fake, None) == -1
    # NULL input
    assert lib.rsvd_truncate(10, 10, None, 10, ctypes.byref(par), fake, fake, 5, fake, 10, fake, 1 << 20, fake, None) == -2
    # workspace too small
    assert lib.rsvd_truncate(10, 10, fake, 10, ctypes.byref(par), fake, fake, 5, fake, 10, fake, 16, fake, None) == -4
    # misaligned workspace
    assert lib.rsvd_truncate(10, 10, fake, 10, ctypes.byref(par), fake, fake, 5, fake, 10, ctypes.c_void_p(4100), 1 << 20, fake, None) == -4


def test_tebd_rejects_overlapping_bonds(lib):
    from paper_1710_01463_gb300 import _lib
    L = 6
    D = _lib.int_array([1, 2, 4, 8, 4, 2, 1])
    bonds = _lib.int_array([1, 2])
    fake = ctypes.c_void_p(4096)
    par = params(1, 10, 2)
    rc = lib.tebd_bond_update(L, 2, D, 2, bonds, fake, 64, fake, 8, fake, ctypes.byref(par), fake, fake, 1 << 30, fake, None)
    assert rc == -1
    par32 = params(1, 10, 2, 1)
    bonds = _lib.int_array([0, 2])
    rc = lib.tebd_bond_update(L, 2, D, 2, bonds, fake, 64, fake, 8, fake, ctypes.byref(par32), fake, fake, 1 << 30, fake, None)
    assert rc == -3
