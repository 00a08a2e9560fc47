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
    for code in (0, -1, -2, -3, -4, -5, -6, -7, -8, 1, 2):
        assert len(lib.rsvd_status_string(code)) > 0
        assert lib.rsvd_status_string(code) != b"unknown status"


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
    assert lib.rsvd_workspace_size(64, 64, ctypes.byref(params(flags=8)), ctypes.byref(sz)) == -1
    assert lib.rsvd_workspace_size(64, 64, ctypes.byref(params(flags=1 << 29)), ctypes.byref(sz)) == -1


def test_full_svd_flag_workspace_and_rejections(lib):
    # Alg. TSVD on the same engine: B = A holds all m rows (m <= 1024), so the workspace
    # grows beyond the sampled path's; entry points without a TSVD form reject the flag
    from paper_1710_01463_gb300 import _lib
    full = _lib.RSVD_FLAG_FULL_SVD
    assert wsize(256, 256, flags=full) > wsize(256, 256)
    sz = ctypes.c_size_t(0)
    assert lib.rsvd_workspace_size(1025, 64, ctypes.byref(params(flags=full)), ctypes.byref(sz)) == -1
    assert lib.rsvd_factored_workspace_size(64, 16, 64, ctypes.byref(params(k=8, flags=full)), ctypes.byref(sz)) == -1
    assert lib.rsvd_tol_workspace_size(64, 64, 16, ctypes.byref(params(k=8, flags=full)), ctypes.byref(sz)) == -1
    m = _lib.int_array([64, 80])
    n = _lib.int_array([70, 90])
    assert lib.rsvd_sectors_adaptive_workspace_size(2, m, n, 16, ctypes.byref(params(k=8, flags=full)),
                                                    ctypes.byref(sz)) == -1
    D = _lib.int_array([1, 2, 4, 2, 1])
    assert lib.tebd_workspace_size(4, 2, D, 2, ctypes.byref(params(k=1, flags=full)), ctypes.byref(sz)) == 0
    assert lib.tebd_product_workspace_size(4, 2, D, 2, 2, ctypes.byref(params(k=1, flags=full)),
                                           ctypes.byref(sz)) == -1


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


def test_product_update_host_checks(lib):
    from paper_1710_01463_gb300 import _lib
    L = 6
    D = _lib.int_array([1, 4, 16, 64, 16, 4, 1])  # d = 4
    par = params(1, 10, 2)
    s2, s3 = ctypes.c_size_t(0), ctypes.c_size_t(0)
    assert lib.tebd_product_workspace_size(L, 4, D, 2, 2, ctypes.byref(par), ctypes.byref(s2)) == 0
    assert lib.tebd_product_workspace_size(L, 4, D, 2, 3, ctypes.byref(par), ctypes.byref(s3)) == 0
    assert 0 < s2.value < s3.value  # X, Y and the Grams grow with K
    assert lib.tebd_product_workspace_size(L, 4, D, 2, 0, ctypes.byref(par), ctypes.byref(s2)) == -1
    fake = ctypes.c_void_p(4096)
    big = ctypes.c_size_t(1 << 40)
    adjacent = _lib.int_array([1, 2])
    assert lib.tebd_product_update(L, 4, D, 2, adjacent, fake, 4096, fake, 64, 2, fake, fake, ctypes.byref(par), fake,
                                   fake, big, fake, None) == -1
    ok_bonds = _lib.int_array([0, 2])
    assert lib.tebd_product_update(L, 4, D, 2, ok_bonds, fake, 4096, fake, 64, 0, fake, fake, ctypes.byref(par), fake,
                                   fake, big, fake, None) == -1
    assert lib.tebd_product_update(L, 4, D, 2, ok_bonds, fake, 4096, fake, 64, 2, fake, fake,
                                   ctypes.byref(params(1, 10, 2, 1)), fake, fake, big, fake, None) == -3
    # a tensor stride too small for the bond's tensors
    assert lib.tebd_product_update(L, 4, D, 2, ok_bonds, fake, 16, fake, 64, 2, fake, fake, ctypes.byref(par), fake,
                                   fake, big, fake, None) == -1


def test_factored_host_checks(lib):
    s32, s64 = ctypes.c_size_t(0), ctypes.c_size_t(0)
    par = params(20, 8, 2)
    assert lib.rsvd_factored_workspace_size(300, 32, 200, ctypes.byref(par), ctypes.byref(s32)) == 0
    assert lib.rsvd_factored_workspace_size(300, 64, 200, ctypes.byref(par), ctypes.byref(s64)) == 0
    assert s32.value < s64.value  # the r x l buffer between the two products
    assert lib.rsvd_factored_workspace_size(300, 32, 200, ctypes.byref(params(20, 8, 2, 3)), ctypes.byref(s32)) == -3
    assert lib.rsvd_factored_workspace_size(10, 32, 200, ctypes.byref(params(20, 8, 2)), ctypes.byref(s32)) == -1
    fake = ctypes.c_void_p(4096)
    big = ctypes.c_size_t(1 << 40)
    # ldx < r
    assert lib.rsvd_truncate_factored(300, 32, 200, fake, 31, fake, 200, ctypes.byref(par), fake, fake, 20, fake, 200,
                                      fake, big, fake, None) == -1
    # misaligned workspace
    assert lib.rsvd_truncate_factored(300, 32, 200, fake, 32, fake, 200, ctypes.byref(par), fake, fake, 20, fake, 200,
                                      ctypes.c_void_p(4100), big, fake, None) == -4


def test_fixed_error_host_checks(lib):
    sz = ctypes.c_size_t(0)
    par = params(8, 10, 2)
    assert lib.rsvd_tol_workspace_size(256, 256, 200, ctypes.byref(par), ctypes.byref(sz)) == 0 and sz.value > 0
    assert lib.rsvd_tol_workspace_size(256, 256, 200, ctypes.byref(params(8, 10, 2, 1)), ctypes.byref(sz)) == -3
    assert lib.rsvd_tol_workspace_size(256, 256, 0, ctypes.byref(par), ctypes.byref(sz)) == -1
    fake = ctypes.c_void_p(4096)
    k = ctypes.c_int(0)
    err = ctypes.c_double(0.0)
    big = ctypes.c_size_t(1 << 40)
    for eps in (-1.0, float("nan")):
        assert lib.rsvd_truncate_tol(256, 256, fake, 256, eps, 200, ctypes.byref(par), fake, fake, 200, fake, 256,
                                     ctypes.byref(k), ctypes.byref(err), fake, big, fake, None) == -1
    # ldu below min(k_max, m, n)
    assert lib.rsvd_truncate_tol(256, 256, fake, 256, 1e-6, 200, ctypes.byref(par), fake, fake, 100, fake, 256,
                                 ctypes.byref(k), ctypes.byref(err), fake, big, fake, None) == -1


def test_adaptive_sectors_host_checks(lib):
    from paper_1710_01463_gb300 import _lib
    m = _lib.int_array([512, 300, 64])
    n = _lib.int_array([512, 200, 100])
    par = params(1, 8, 2)
    sz, ref = ctypes.c_size_t(0), ctypes.c_size_t(0)
    assert lib.rsvd_sectors_adaptive_workspace_size(3, m, n, 64, ctypes.byref(par), ctypes.byref(sz)) == 0
    caps = _lib.int_array([64, 64, 64])
    assert lib.rsvd_batched_workspace_size(3, m, n, caps, ctypes.byref(par), ctypes.byref(ref)) == 0
    # sized for the largest trial rank, min(chi, m_b, n_b), plus the device rounds' state
    # (2 batch + 1 ints, one 256-byte aligned slot)
    assert sz.value == ref.value + 256
    assert lib.rsvd_sectors_adaptive_workspace_size(3, m, n, 0, ctypes.byref(par), ctypes.byref(sz)) == -1
    m65 = _lib.int_array([64] * 65)
    assert lib.rsvd_sectors_adaptive_workspace_size(65, m65, m65, 8, ctypes.byref(par), ctypes.byref(sz)) == -1
    fake = ctypes.c_void_p(4096)
    ptrs = _lib.ptr_array([4096] * 3)
    lds = _lib.int_array([512, 200, 100])
    kt = _lib.int_array([4, 4, 4])
    rounds = ctypes.c_int(0)
    big = ctypes.c_size_t(1 << 40)
    bf16 = params(1, 8, 2, 3)
    m2 = _lib.int_array([512, 512, 512])
    assert lib.rsvd_truncate_sectors_adaptive(3, m2, m2, ptrs, _lib.int_array([512] * 3), kt, ctypes.byref(bf16), 64,
                                              ptrs, ptrs, _lib.int_array([64] * 3), ptrs, _lib.int_array([512] * 3),
                                              fake, ctypes.byref(rounds), fake, big, fake, None) == -3
    # ldu below the block's cap
    assert lib.rsvd_truncate_sectors_adaptive(3, m, n, ptrs, lds, kt, ctypes.byref(par), 64, ptrs, ptrs,
                                              _lib.int_array([8, 64, 64]), ptrs, lds, fake, ctypes.byref(rounds), fake,
                                              big, fake, None) == -1
    # the device-rounds form: same checks (nothing is launched when they fail)
    assert lib.rsvd_truncate_sectors_adaptive_device(3, m2, m2, ptrs, _lib.int_array([512] * 3), kt,
                                                     ctypes.byref(bf16), 64, ptrs, ptrs, _lib.int_array([64] * 3),
                                                     ptrs, _lib.int_array([512] * 3), fake, fake, fake, fake, big,
                                                     fake, None) == -3
    assert lib.rsvd_truncate_sectors_adaptive_device(3, m, n, ptrs, lds, kt, ctypes.byref(par), 64, ptrs, ptrs,
                                                     _lib.int_array([8, 64, 64]), ptrs, lds, fake, fake, fake, fake,
                                                     big, fake, None) == -1
    assert lib.rsvd_truncate_sectors_adaptive_device(3, m, n, ptrs, lds, kt, ctypes.byref(par), 64, ptrs, ptrs,
                                                     _lib.int_array([64] * 3), ptrs, lds, fake, None, fake, fake,
                                                     big, fake, None) == -2
    assert lib.rsvd_truncate_sectors_adaptive_device(3, m, n, ptrs, lds, kt, ctypes.byref(par), 64, ptrs, ptrs,
                                                     _lib.int_array([64] * 3), ptrs, lds, fake, fake, fake, fake,
                                                     ctypes.c_size_t(sz.value - 1), fake, None) == -4


def test_autotune_cache_round_trip(lib, tmp_path):
    # the host cache of measured tile choices: enable / clear / entries, and the text file
    # written and read back (no GPU needed: nothing is timed here)
    assert lib.rsvd_autotune_clear() == 0
    assert lib.rsvd_autotune_entries() == 0
    path = tmp_path / "tiles.txt"
    path.write_text("# tin tout ta tx count M N K choice\n8 8 0 0 3 256 144 256 5\n4 4 1 0 16 1024 144 1024 2\n"
                    "4 4 0 0 1 64 64 64 4\n")  # the last choice does not exist for FP32: skipped
    assert lib.rsvd_autotune_load(str(path).encode()) == 2
    assert lib.rsvd_autotune_entries() == 2
    out = tmp_path / "out.txt"
    assert lib.rsvd_autotune_save(str(out).encode()) == 0
    rows = [r for r in out.read_text().splitlines() if not r.startswith("#")]
    assert sorted(rows) == sorted(["8 8 0 0 3 256 144 256 5", "4 4 1 0 16 1024 144 1024 2"])
    assert lib.rsvd_autotune_load(str(tmp_path / "missing.txt").encode()) == -1
    assert lib.rsvd_autotune_enable(1) == 0 and lib.rsvd_autotune_enable(0) == 0
    assert lib.rsvd_autotune_clear() == 0 and lib.rsvd_autotune_entries() == 0


def test_autotune_cache_wide_fp32_tile(lib, tmp_path):
    # tile choice 3 is the 128 x 128 FP32 tile for FP32 -> FP32 products and the 48 x 32 tile
    # for FP64; the FP32 -> FP64 products (the projection B = Q^T A) have no choice 3, so the
    # loader skips such a line
    assert lib.rsvd_autotune_clear() == 0
    path = tmp_path / "tiles.txt"
    path.write_text("4 4 0 0 64 1024 128 1024 3\n"   # FP32 -> FP32: the wide tile
                    "4 4 1 0 64 1024 144 1024 3\n"   # FP32 -> FP32, A transposed
                    "4 8 1 0 64 144 1024 1024 3\n"   # FP32 -> FP64: no choice 3, skipped
                    "4 4 0 0 64 1024 128 1024 4\n"   # FP32 has no choice 4, skipped
                    "8 8 0 0 2 256 144 256 3\n")     # FP64: the 48 x 32 tile
    assert lib.rsvd_autotune_load(str(path).encode()) == 3
    out = tmp_path / "out.txt"
    assert lib.rsvd_autotune_save(str(out).encode()) == 0
    rows = sorted(r for r in out.read_text().splitlines() if not r.startswith("#"))
    assert rows == sorted(["4 4 0 0 64 1024 128 1024 3", "4 4 1 0 64 1024 144 1024 3", "8 8 0 0 2 256 144 256 3"])
    assert lib.rsvd_autotune_clear() == 0
