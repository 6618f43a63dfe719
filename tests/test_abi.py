"""The C-ABI library loads and exports every entry point include/recon.h declares
(no device calls), and host-side argument checks fail cleanly without a GPU."""
import ctypes as C
import os
import re

import pytest

from paper_1706_07075_b300 import binding as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "recon.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(recon_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_the_boundary_calls():
    names = declared_functions()
    for required in ["recon_create", "recon_sensitivity", "recon_split_regions", "recon_mlem", "recon_destroy",
                     "recon_mlem_regions", "recon_last_error"]:
        assert required in names


def test_library_exports_every_declared_symbol():
    lib = B.load()
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_checked_build_exports_every_declared_symbol():
    # librecon_check.so, the bounds-checked build, has the same boundary
    from paper_1706_07075_b300 import build as lib_build
    lib = C.CDLL(lib_build.build(checked=True))
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_normal_build_reports_no_bounds_checks():
    # the host-side query needs no device in the normal build: -1, no checks compiled in
    if os.environ.get("RECON_BOUNDS_CHECK") != "1":
        assert B.recon_debug_bounds_violations() == -1


def test_binding_covers_every_declared_symbol():
    assert sorted(B.SIGNATURES) == declared_functions()
    for name in declared_functions():
        assert callable(getattr(B, name))


def test_null_and_invalid_arguments_fail_without_a_device():
    lib = B.load()
    out = C.c_void_p()
    geo = B.recon_geometry(400.0, 2400.0, 45.0)
    grid = B.recon_grid(4, 4, 4, 1.0, 1.0, 1.0, 0.0, 0.0, 0.0)
    assert lib.recon_create(None, C.byref(grid), 300.0, C.byref(out)) == B.RECON_EINVAL
    assert lib.recon_create(C.byref(geo), None, 300.0, C.byref(out)) == B.RECON_EINVAL
    assert lib.recon_create(C.byref(geo), C.byref(grid), 300.0, None) == B.RECON_EINVAL
    assert lib.recon_create(C.byref(geo), C.byref(grid), -1.0, C.byref(out)) == B.RECON_EINVAL
    assert b"tof_fwhm_ps" in lib.recon_last_error(None)
    bad = B.recon_grid(0, 4, 4, 1.0, 1.0, 1.0, 0.0, 0.0, 0.0)
    assert lib.recon_create(C.byref(geo), C.byref(bad), 300.0, C.byref(out)) == B.RECON_EINVAL
    huge = B.recon_grid(2048, 2048, 2048, 1.0, 1.0, 1.0, 0.0, 0.0, 0.0)
    assert lib.recon_create(C.byref(geo), C.byref(huge), 300.0, C.byref(out)) == B.RECON_EINVAL
    nan = B.recon_grid(4, 4, 4, float("nan"), 1.0, 1.0, 0.0, 0.0, 0.0)
    assert lib.recon_create(C.byref(geo), C.byref(nan), 300.0, C.byref(out)) == B.RECON_EINVAL
    badgeo = B.recon_geometry(400.0, 2400.0, 120.0)
    assert lib.recon_create(C.byref(badgeo), C.byref(grid), 300.0, C.byref(out)) == B.RECON_EINVAL
    assert out.value is None
    # NULL context: every call reports EINVAL, destroy is NULL-safe
    lib.recon_destroy(None)
    assert lib.recon_mlem(None, None, 1, None, None, None) == B.RECON_EINVAL
    assert lib.recon_sensitivity(None, None, 0, 0, None) == B.RECON_EINVAL
    assert lib.recon_split_regions(None, None, 1, None, 0.0, 0.0, None, None, None) == B.RECON_EINVAL
    assert lib.recon_set_brick_layout(None, 1) == B.RECON_EINVAL


def test_python_binding_raises_with_message():
    with pytest.raises(B.ReconError) as e:
        B.recon_create(B.recon_geometry(400.0, 2400.0, 45.0), B.recon_grid(0, 1, 1, 1, 1, 1, 0, 0, 0), 300.0)
    assert e.value.status == B.RECON_EINVAL
    assert "grid" in str(e.value)


def test_event_struct_marshalling():
    import numpy as np
    ev = np.zeros((7, 5), np.float32)
    e = B.make_events(ev)
    assert e.n == 5 and e.fmt == B.RECON_EV_F32_SOA and e.on_device == 0
    base = ev.ctypes.data
    assert [e.planes[k] for k in range(7)] == [base + 4 * 5 * k for k in range(7)]
    rec = np.zeros((5, 8), np.int16)
    p = B.make_events(rec, packed=True, lattice_mm=0.05)
    assert p.fmt == B.RECON_EV_PACKED_I16_F16 and p.planes[0] == rec.ctypes.data and p.lattice_mm == 0.05
