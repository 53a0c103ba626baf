"""CPU-side checks of the C ABI: the library builds, loads and exports every
function that include/*.h declares; host-side argument checks fire before any
GPU work (no compute call is made here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    inc = os.path.join(ROOT, "include")
    for f in os.listdir(inc):
        if f.endswith(".h"):
            txt = open(os.path.join(inc, f)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\bint\s+(scqr3_\w+)\s*\(", txt))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    from paper_1809_11085_gb300 import build, scqr3

    build.build()
    return scqr3.lib()


def test_header_declares_the_boundary():
    names = declared_functions()
    assert "scqr3_factor" in names and "scqr3_workspace_bytes" in names


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_info_struct_layout_matches_header():
    from paper_1809_11085_gb300 import scqr3

    # 2 ints + 2 x MAX_PASSES ints + 2 x MAX_PASSES doubles + the `more` int,
    # padded to the doubles' 8-byte alignment
    raw = 8 + 8 * scqr3.MAX_PASSES + 16 * scqr3.MAX_PASSES + 4
    assert scqr3.INFO_BYTES == (raw + 7) // 8 * 8
    assert scqr3._Info.more.offset == 8 + 8 * scqr3.MAX_PASSES + 16 * scqr3.MAX_PASSES


def test_argument_errors_are_reported_on_the_host(lib):
    from paper_1809_11085_gb300 import scqr3

    out = ctypes.c_size_t(0)
    # m < n
    assert lib.scqr3_workspace_bytes(3, 5, None, None, ctypes.byref(out)) == -2
    # n < 1
    assert lib.scqr3_workspace_bytes(3, 0, None, None, ctypes.byref(out)) == -3
    # bad block size
    b = scqr3._B(3, ctypes.c_void_p(8), 0.0)
    assert lib.scqr3_workspace_bytes(30, 5, ctypes.byref(b), None, ctypes.byref(out)) == -5
    # m not a multiple of bs
    b = scqr3._B(8, ctypes.c_void_p(8), 0.0)
    assert lib.scqr3_workspace_bytes(30, 5, ctypes.byref(b), None, ctypes.byref(out)) == -5
    # CSR form (bs = 0): missing arrays, too few entries for a diagonal per row, n > 128
    b = scqr3._B(0, None, 0.0, None, None, None, 0)
    assert lib.scqr3_workspace_bytes(30, 5, ctypes.byref(b), None, ctypes.byref(out)) == -5
    b = scqr3._B(0, None, 0.0, ctypes.c_void_p(8), ctypes.c_void_p(8), ctypes.c_void_p(8), 29)
    assert lib.scqr3_workspace_bytes(30, 5, ctypes.byref(b), None, ctypes.byref(out)) == -5
    b = scqr3._B(0, None, 0.0, ctypes.c_void_p(8), ctypes.c_void_p(8), ctypes.c_void_p(8), 3000)
    assert lib.scqr3_workspace_bytes(1000, 200, ctypes.byref(b), None, ctypes.byref(out)) == \
        scqr3.E_UNSUPPORTED
    # bad max_passes
    o = scqr3._Opts(2, 0, 0.0)
    assert lib.scqr3_workspace_bytes(30, 5, None, ctypes.byref(o), ctypes.byref(out)) == -12
    # n beyond the FP64 path
    assert lib.scqr3_workspace_bytes(1000, 300, None, None, ctypes.byref(out)) == scqr3.E_UNSUPPORTED
    # the tensor-core Gram: n <= 128 (n <= 256 for the FP64-accurate form with
    # B = I), m <= 2^31
    for prec in (scqr3.PREC_TC, scqr3.PREC_MIXED_TC):
        o = scqr3._Opts(0, prec, 0.0)
        assert lib.scqr3_workspace_bytes(1000, 257, None, ctypes.byref(o), ctypes.byref(out)) == \
            scqr3.E_UNSUPPORTED
        r129 = lib.scqr3_workspace_bytes(1000, 129, None, ctypes.byref(o), ctypes.byref(out))
        if prec == scqr3.PREC_TC:  # accepted (the size needs the device: E_CUDA on a host without one)
            assert r129 in (0, scqr3.E_CUDA)
        else:
            assert r129 == scqr3.E_UNSUPPORTED
        assert lib.scqr3_workspace_bytes(2 ** 31 + 1, 8, None, ctypes.byref(o), ctypes.byref(out)) == \
            scqr3.E_UNSUPPORTED
        b = scqr3._B(16, ctypes.c_void_p(8), 0.0)  # blocks of 16 rows: FP64 only
        assert lib.scqr3_workspace_bytes(800, 16, ctypes.byref(b), ctypes.byref(o), ctypes.byref(out)) == \
            scqr3.E_UNSUPPORTED
        b = scqr3._B(0, None, 0.0, ctypes.c_void_p(8), ctypes.c_void_p(8), ctypes.c_void_p(8), 3000)  # CSR
        assert lib.scqr3_workspace_bytes(1000, 16, ctypes.byref(b), ctypes.byref(o), ctypes.byref(out)) == \
            scqr3.E_UNSUPPORTED
    b = scqr3._B(8, ctypes.c_void_p(8), 0.0)  # the mixed substitution takes no B
    o = scqr3._Opts(0, scqr3.PREC_MIXED_TC, 0.0)
    assert lib.scqr3_workspace_bytes(800, 16, ctypes.byref(b), ctypes.byref(o), ctypes.byref(out)) == \
        scqr3.E_UNSUPPORTED
    # null pointers in scqr3_factor are rejected before any CUDA call
    assert lib.scqr3_factor(None, 10, 2, 2, None, None, 2, None, None, None, 0, None, None,
                            None) == -1


def test_shard_argument_errors_are_reported_on_the_host(lib):
    """The row-partitioned calls number their argument codes by their own
    prototypes and reject the forms they do not take before any CUDA call."""
    import ctypes

    from paper_1809_11085_gb300 import scqr3

    wb, gw = ctypes.c_size_t(0), ctypes.c_size_t(0)
    o = scqr3._Opts(0, scqr3.PREC_MIXED, 0.0, 0.0, 3, 0.0)
    assert lib.scqr3_shard_sizes(1000, 16, None, ctypes.byref(o), ctypes.byref(wb), ctypes.byref(gw)) == \
        scqr3.E_UNSUPPORTED
    assert lib.scqr3_shard_sizes(1000, 0, None, None, ctypes.byref(wb), ctypes.byref(gw)) == -2
    assert lib.scqr3_shard_sizes(0, 16, None, None, ctypes.byref(wb), ctypes.byref(gw)) == -1
    assert lib.scqr3_shard_sizes(1000, 16, None, None, None, ctypes.byref(gw)) == -5
    # a block shorter than n is allowed (m_local >= 1); a B without ||B||_2 is not
    b = scqr3._B(8, ctypes.c_void_p(8), 0.0)
    assert lib.scqr3_gram_partial(None, 1000, 16, 16, ctypes.byref(b), None, None, 0, None, None, None) == -5
    csr = scqr3._B(0, None, 1.0, ctypes.c_void_p(8), ctypes.c_void_p(8), ctypes.c_void_p(8), 5000)
    assert lib.scqr3_gram_partial(None, 1000, 16, 16, ctypes.byref(csr), None, None, 0, None, None, None) == \
        scqr3.E_UNSUPPORTED
    assert lib.scqr3_gram_partial(None, 1000, 16, 16, None, None, None, 0, None, None, None) == -1
    assert lib.scqr3_apply_pass(-1, None, 1000, None, 1000, 16, 16, None, None, 16, None, None, None, 0, None,
                                None, None) == -1
    assert lib.scqr3_apply_pass(0, None, 1000, None, 1000, 16, 16, None, None, 16, None, None, None, 0, None,
                                None, None) == -2


def test_backward_options_are_checked_on_the_host(lib):
    """scqr3_backward_ex / scqr3_backward_workspace_bytes_ex: the precision and
    the shape limits of the tensor-core adjoint are rejected before any CUDA
    call; argument codes follow the prototype (opts is argument 12)."""
    from paper_1809_11085_gb300 import scqr3

    out = ctypes.c_size_t(0)
    for prec in (scqr3.PREC_MIXED, scqr3.PREC_MIXED_TC, 7):
        o = scqr3._Opts(0, prec, 0.0)
        assert lib.scqr3_backward_workspace_bytes_ex(1000, 16, ctypes.byref(o), ctypes.byref(out)) == \
            scqr3.E_UNSUPPORTED
        assert lib.scqr3_backward_ex(ctypes.c_void_p(256), 1000, 16, 16, ctypes.c_void_p(256), 3,
                                     ctypes.c_void_p(256), 16, None, ctypes.c_void_p(256), 16, ctypes.byref(o),
                                     ctypes.c_void_p(256), 1 << 30, None, None) == scqr3.E_UNSUPPORTED
    o = scqr3._Opts(0, scqr3.PREC_TC, 0.0)
    assert lib.scqr3_backward_workspace_bytes_ex(1000, 129, ctypes.byref(o), ctypes.byref(out)) == \
        scqr3.E_UNSUPPORTED
    assert lib.scqr3_backward_workspace_bytes_ex(2 ** 31 + 1, 8, ctypes.byref(o), ctypes.byref(out)) == \
        scqr3.E_UNSUPPORTED
    assert lib.scqr3_backward_workspace_bytes_ex(5, 8, ctypes.byref(o), ctypes.byref(out)) == -1
    assert lib.scqr3_backward_workspace_bytes_ex(5, 0, ctypes.byref(o), ctypes.byref(out)) == -2
    assert lib.scqr3_backward_workspace_bytes_ex(50, 8, ctypes.byref(o), None) == -4
    args = [ctypes.c_void_p(256), 1000, 16, 16, ctypes.c_void_p(256), 3, ctypes.c_void_p(256), 16, None,
            ctypes.c_void_p(256), 16, ctypes.byref(o), ctypes.c_void_p(256), 1 << 30, None, None]
    for idx, bad, code in [(0, None, -1), (3, 8, -4), (4, None, -5), (5, 0, -6), (6, None, -7), (7, 3, -8),
                           (9, None, -10), (10, 2, -11), (12, ctypes.c_void_p(8), scqr3.E_WORKSPACE)]:
        a = list(args)
        a[idx] = bad
        assert lib.scqr3_backward_ex(*a) == code, (idx, code)
