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


def params(k=32, p=8, q=2, prec=0, flags=0):
    from paper_1710_01463_gb300 import _lib
    return _lib.RsvdParams(k, p, q, prec, 201, 0, 0, flags)


def wsize(m, n, **kw):
    sz = ctypes.c_size_t(0)
    assert lib_global().rsvd_workspace_size(m, n, ctypes.byref(params(**kw)), ctypes.byref(sz)) == 0
    return sz.value


def lib_global():
    from paper_1710_01463_gb300 import _lib
    return _lib.load()


def test_workspace_size_grows_with_size(lib):
    # within one product path (FP64 FMAs, or tensor-core slices for m, n <= 1024)
    assert 0 < wsize(256, 256, flags=1) < wsize(1024, 1024, flags=1) < wsize(2048, 2048)
    assert 0 < wsize(128, 128) < wsize(256, 256) < wsize(1024, 1024)
    assert wsize(256, 256) % 256 == 0


def test_workspace_holds_the_fp64_slices(lib):
    # nine BF16 slices of A and of A^T (256 x 256) and of the thin operand (48 x 256), exponents
    extra = wsize(256, 256) - wsize(256, 256, flags=1)
    assert extra >= 9 * 2 * (256 * 256 + 256 * 256 + 48 * 256)
    assert extra < 4 * 1024 * 1024
    # up to m, n = 1024 (K in chunks of 256); beyond, the FP64 FMA path holds no slices
    extra = wsize(1024, 1024) - wsize(1024, 1024, flags=1)
    assert extra >= 9 * 2 * (1024 * 1024 + 1024 * 1024 + 48 * 1024)
    assert wsize(1025, 1024) == wsize(1025, 1024, flags=1)


def test_unknown_flags_rejected(lib):
    sz = ctypes.c_size_t(0)
    assert lib.rsvd_workspace_size(64, 64, ctypes.byref(params(flags=2)), ctypes.byref(sz)) == -1


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
