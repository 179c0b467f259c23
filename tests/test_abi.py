"""The C ABI library builds, loads, and exports every entry point that
include/*.h declares.  CPU only: no kernel is launched."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?\w[\w\s\*]*?\b(wc_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1612_06556_gb300 as wc
    return ctypes.CDLL(wc.LIB_PATH)


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ["wc_create_lattice", "wc_load_gauge", "wc_load_clover", "wc_apply_M",
                     "wc_apply_Mdag", "wc_ras_precond", "wc_solve_bicgstab", "wc_solve_batch",
                     "wc_action_force", "wc_last_error"]:
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_lists_match_header():
    import paper_1612_06556_gb300 as wc
    assert sorted(wc.EXPORTED) == sorted(n for n in declared_functions() if n in wc.EXPORTED)
    assert set(declared_functions()) <= set(wc.EXPORTED)


def test_argument_errors_are_reported_without_a_gpu(lib):
    import paper_1612_06556_gb300 as wc
    with pytest.raises(wc.WCError) as e:
        wc.Lattice((1, 4, 4, 4))
    assert e.value.status == 1 and "extent" in str(e.value)
    with pytest.raises(wc.WCError) as e:
        wc.Lattice((4, 4, 4, 4), t_bc=3)
    assert e.value.status == 1


def test_null_handles_are_argument_errors_without_a_gpu(lib):
    """Entry points reject NULL handles with WC_ERR_ARG before touching the
    device (host-side checks of the double-FP32 switch, the complex64 and
    asynchronous transfers and the lattice sync)."""
    import paper_1612_06556_gb300 as wc
    L = wc._L
    buf = (ctypes.c_double * 24)()
    assert L.wc_set_fp64_arith(None, wc.ARITH_DF32) == 1
    assert L.wc_sync(None) == 1
    assert L.wc_field_import_f32(None, buf) == 1
    assert L.wc_field_export_f32(None, buf) == 1
    assert L.wc_field_import_async(None, buf, 0) == 1
    assert L.wc_field_export_async(None, buf, 1) == 1
    rp = wc.ras_params((4, 4, 4, 4), 1, 4, True)
    assert L.wc_ras_schur(None, None, None, ctypes.byref(rp), 0) == 1
    assert L.wc_last_error(None)


def test_dot_noalloc_argument_errors_without_a_gpu(lib):
    """The allocation-free inner product rejects NULL or misaligned pointers
    and negative sizes with WC_ERR_ARG before any CUDA call (the pointer
    values below are never dereferenced)."""
    import paper_1612_06556_gb300 as wc
    L = wc._L
    p16, p8 = wc._vp(0x10000), wc._vp(0x20008)
    assert L.wc_dot_noalloc(None, p16, 4, p16, None) == 1
    assert L.wc_dot_noalloc(p16, None, 4, p16, None) == 1
    assert L.wc_dot_noalloc(p16, p16, 4, None, None) == 1
    assert L.wc_dot_noalloc(p16, p16, -1, p16, None) == 1
    assert L.wc_dot_noalloc(p8, p16, 4, p16, None) == 1
    assert "aligned" in L.wc_last_error(None).decode()
    assert L.wc_dot_noalloc(p16, p8, 4, p16, None) == 1
    assert L.wc_dot_noalloc(p16, p16, 4, wc._vp(0x10004), None) == 1
    assert "aligned" in L.wc_last_error(None).decode()


def test_subdomain_argument_errors_without_a_gpu(lib):
    """wc_create_subdomain checks its extents and offsets before any CUDA
    call."""
    import paper_1612_06556_gb300 as wc
    for local, glob, off in [((4, 4, 4, 4), (4, 4, 4, 4), (0, 0, 0, 0)),    # nothing cut
                             ((4, 4, 4, 8), (4, 4, 4, 4), (0, 0, 0, 0)),    # local > global
                             ((4, 4, 4, 4), (4, 4, 4, 8), (0, 0, 0, 5)),    # outside the lattice
                             ((4, 4, 4, 1), (4, 4, 4, 8), (0, 0, 0, 0))]:   # extent < 2
        with __import__("pytest").raises(wc.WCError) as e:
            wc.SubDomain(local, glob, off)
        assert e.value.status == 1


def test_checked_violations_needs_the_checked_build(lib):
    """The normal build answers WC_ERR_STATE before touching the device."""
    import paper_1612_06556_gb300 as wc
    n = ctypes.c_ulonglong(7)
    assert wc._L.wc_checked_violations(ctypes.byref(n)) == 3 and n.value == 0
    assert wc._L.wc_checked_violations(None) == 1
