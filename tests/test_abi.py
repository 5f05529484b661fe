"""The C-ABI library builds, loads and exports every symbol include/cg.h declares.
No compute calls here (no GPU needed)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not h.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", h)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"\b(cg_[a-z0-9_]+)\s*\(", text):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    from paper_1409_0001_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_path():
    names = declared_symbols()
    for must in ("cg_create_mesh_structured", "cg_create_mesh_tet", "cg_deposit", "cg_diffuse",
                 "cg_coarse_grain", "cg_locate"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_symbols() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    import paper_1409_0001_gb300 as cg
    assert sorted(cg.exported_symbols()) == declared_symbols()


def test_status_strings_and_defaults(lib):
    import paper_1409_0001_gb300 as cg
    L = cg.load_library()
    assert L.cg_status_string(6) == b"CG_EDOMAIN"
    p = cg.CgParams()
    L.cg_params_default(ctypes.byref(p))
    assert p.nsteps == 10 and p.tol == 1e-13 and p.precision == 0


def test_bad_arguments_fail_without_a_gpu(lib):
    import paper_1409_0001_gb300 as cg
    L = cg.load_library()
    h = ctypes.c_void_p()
    org = (ctypes.c_double * 3)(0, 0, 0)
    assert L.cg_create_mesh_structured(0, 4, 4, org, 0.1, ctypes.byref(h)) == 1
    assert b"dimensions" in L.cg_last_error()
    assert L.cg_create_mesh_structured(4, 4, 4, org, -1.0, ctypes.byref(h)) == 1
    assert L.cg_create_mesh_structured(4, 4, 4, org, 0.25, ctypes.byref(h)) == 0
    assert L.cg_mesh_num_cells(h) == 64
    vol = (ctypes.c_double * 64)()
    assert L.cg_mesh_cell_volumes(h, vol) == 0 and vol[5] == 0.25 ** 3
    p = cg.CgParams()
    L.cg_params_default(ctypes.byref(p))
    p.nsteps = 0
    assert L.cg_diffuse(h, 1, None, ctypes.byref(p), None, None) == 1
    assert L.cg_destroy_mesh(h) == 0


def test_size_limits_refused_before_any_device_work(lib):
    """Particle counts outside [0, 2^31) and field counts outside [1, 64] are refused by
    the argument checks, which run before any pointer is inspected or any device call."""
    import paper_1409_0001_gb300 as cg
    L = cg.load_library()
    h = ctypes.c_void_p()
    org = (ctypes.c_double * 3)(0, 0, 0)
    assert L.cg_create_mesh_structured(4, 4, 4, org, 0.25, ctypes.byref(h)) == 0
    p = cg.CgParams()
    L.cg_params_default(ctypes.byref(p))
    for n, nf, what in (((1 << 31), 1, b"n must be"), (-1, 1, b"n must be"),
                        (10, 0, b"nfields"), (10, 65, b"nfields")):
        assert L.cg_deposit(h, n, None, nf, None, None, ctypes.byref(p), None, None) == 1
        assert what in L.cg_last_error()
        assert L.cg_coarse_grain(h, n, None, nf, None, None, ctypes.byref(p), None, None) == 1
        assert what in L.cg_last_error()
    assert L.cg_diffuse(h, 65, None, ctypes.byref(p), None, None) == 1
    assert b"nfields" in L.cg_last_error()
    assert L.cg_destroy_mesh(h) == 0


def test_mesh_sizes_whose_product_overflows_are_refused(lib):
    """nx * ny * nz is bounded factor by factor, so dimensions whose product would wrap
    around 64 bits (2^21 * 2^21 * 2^22 = 2^64) are refused, not taken as a small mesh."""
    import paper_1409_0001_gb300 as cg
    L = cg.load_library()
    h = ctypes.c_void_p()
    org = (ctypes.c_double * 3)(0, 0, 0)
    for dims in ((1 << 21, 1 << 21, 1 << 22), (2 ** 31 - 1, 2 ** 31 - 1, 2 ** 31 - 1),
                 (1 << 16, 1 << 16, 1), (2, 1, 1 << 30)):
        assert L.cg_create_mesh_structured(*dims, org, 0.1, ctypes.byref(h)) == 1
        assert b"too large" in L.cg_last_error()
    assert L.cg_create_mesh_structured(1 << 10, 1 << 10, (1 << 11) - 1, org, 0.1,
                                       ctypes.byref(h)) == 0
    assert L.cg_mesh_num_cells(h) == (1 << 20) * ((1 << 11) - 1)
    assert L.cg_destroy_mesh(h) == 0


def test_noalloc_deposition_refuses_bad_sizes_before_any_device_work(lib):
    """cg_deposit_fixed_noalloc checks its sizes against the static scratch without
    forming a product that could overflow, and refuses a non-finite origin, before it
    touches the device."""
    import paper_1409_0001_gb300 as cg
    L = cg.load_library()
    org = (ctypes.c_double * 3)(0, 0, 0)
    dummy = ctypes.c_void_p(16)
    for dims, nf in (((1 << 21, 1 << 21, 1 << 22), 1), ((160, 160, 160), 1),
                     ((128, 128, 128), 2), ((2 ** 31 - 1, 2 ** 31 - 1, 2 ** 31 - 1), 8)):
        st = L.cg_deposit_fixed_noalloc(*dims, org, 0.01, 1, dummy, nf, dummy, dummy, None, None)
        assert st == 1
        assert b"exceeds the static scratch" in L.cg_last_error()
    for bad in (float("inf"), float("-inf"), float("nan")):
        o = (ctypes.c_double * 3)(0.0, bad, 0.0)
        st = L.cg_deposit_fixed_noalloc(8, 8, 8, o, 0.01, 1, dummy, 1, dummy, dummy, None, None)
        assert st == 1 and b"origin" in L.cg_last_error()
    big = (ctypes.c_double * 3)(1.7e308, 0.0, 0.0)        # origin + n dx overflows
    st = L.cg_deposit_fixed_noalloc(8, 8, 8, big, 1e307, 1, dummy, 1, dummy, dummy, None, None)
    assert st == 1 and b"finite" in L.cg_last_error()


def test_workspace_limit_is_validated_without_a_gpu(lib):
    """The workspace cap is host state: a negative limit is refused, 0 clears it, and no
    workspace is held before any device call."""
    import paper_1409_0001_gb300 as cg
    L = cg.load_library()
    assert L.cg_workspace_bytes() == 0
    assert L.cg_set_workspace_limit(-1) == 1 and b"limit" in L.cg_last_error()
    assert L.cg_set_workspace_limit(1 << 20) == 0
    assert L.cg_set_workspace_limit(0) == 0
