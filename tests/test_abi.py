"""The C-ABI library builds for sm_103a, loads without a GPU and exports every
symbol include/rsi.h declares; host-only calls (layout, argument checks) work
on the CPU.  No compute call is made here."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2408_06765_gb300 import build, rsi
    build.build()
    return rsi.load()


def declared_symbols():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            text = open(os.path.join(ROOT, "include", h)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(rsi_\w+)\s*\(", text))
    return sorted(names)


def test_header_declares_the_path():
    names = declared_symbols()
    for required in ("rsi_make_qmc_points", "rsi_propagate_stage", "rsi_field_image",
                     "rsi_interface_transmit", "rsi_grid_points"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in declared_symbols() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_header(lib):
    from paper_2408_06765_gb300 import rsi
    assert set(rsi.SYMBOLS) <= set(declared_symbols())


def test_version_and_layout(lib):
    from paper_2408_06765_gb300 import rsi
    assert lib.rsi_version() == 1
    for n in (1, 7, 1000, 1 << 18):
        offs = [lib.rsi_points_offset(f, n) for f in range(16)]
        assert offs[0] == 0 and all(o % 256 == 0 for o in offs)
        assert offs == sorted(offs)
        sizes = [4] * 3 + [8] * 7 + [4] * 6
        for f in range(15):
            assert offs[f + 1] - offs[f] >= sizes[f] * n
        assert lib.rsi_points_bytes(n) >= offs[15] + 4 * n
    assert lib.rsi_points_offset(16, 10) == -1
    assert lib.rsi_points_offset(-1, 10) == -1


def test_invalid_arguments_are_rejected_before_any_launch(lib):
    from paper_2408_06765_gb300 import rsi
    st = rsi.stage_struct(rsi.STAGE_PISTON, "fp32c", 1000.0)
    rc = lib.rsi_propagate_stage(ctypes.byref(st), None, 10, None, None, 10, None, None, 0, None)
    assert rc == -1 and b"null" in lib.rsi_last_error()
    s = rsi.surface_struct({"kind": "disk", "a": 1e-3})
    rc = lib.rsi_make_qmc_points(ctypes.byref(s), 0, 0, 0, ctypes.c_void_p(256), 1 << 20, None)
    assert rc == -1
    bad = rsi.stage_struct(7, "fp32c", 1000.0)
    assert lib.rsi_stage_workspace_bytes(ctypes.byref(bad), 10, 10) == 0
    it = rsi.interface_struct({"rho": 1000, "c": 1480}, {"rho": -1, "c": 5900}, 0.0)
    rc = lib.rsi_interface_transmit(ctypes.byref(it), ctypes.c_void_p(256), 10, ctypes.c_void_p(256),
                                    ctypes.c_void_p(256), None)
    assert rc == -1
    g = rsi.grid_struct({"x0": 0, "x1": 1, "z0": 0, "z1": 1, "nx": 0, "nz": 4})
    assert lib.rsi_grid_points(ctypes.byref(g), ctypes.c_void_p(256), 1 << 20, None) == -1


def test_library_has_no_cpu_fallback_symbols(lib):
    # the product library holds no host implementation of the sums: its only
    # exported entry points are those of the header
    path = os.path.join(ROOT, "paper_2408_06765_gb300", "_build", "librsi.so")
    out = os.popen(f"nm -D --defined-only {path}").read()
    exported = set(re.findall(r" T (rsi_\w+)", out))
    assert exported == set(declared_symbols())
