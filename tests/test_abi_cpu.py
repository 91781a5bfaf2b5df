"""The C-ABI library builds, loads and exports every entry point declared in
include/*.h; host-side argument checks answer without touching a GPU."""
import ctypes
import glob
import os
import re

import pytest

import paper_2403_12340_gb300 as pkg

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(pkg.LIB_PATH):
        from paper_2403_12340_gb300 import build

        build.build()
    return pkg.load_library()


def declared_functions():
    names = []
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        names += re.findall(r"ISDF_API\s+[\w\s\*]+?\b(\w+)\s*\(", src)
    return sorted(set(names))


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert {"isdf_create", "isdf_fit", "build_polarizability", "smw_inverse", "apply_eps_inv"} <= set(names)
    for n in names:
        assert hasattr(lib, n), n
    assert set(pkg.EXPORTED) <= set(names) | {"isdf_version"}


def test_library_is_sm103a_build(lib):
    assert "sm_103a" in pkg.version()


def test_create_rejects_bad_shapes_on_host(lib):
    h = ctypes.c_void_p()
    for args in [(1, 8, 8), (8, 0, 8), (17, 8, 8), (8, 8, 600)]:
        rc = lib.isdf_create(ctypes.byref(h), *args, 4.0, 4.0, 4.0, None)
        assert rc == -2, args
        assert h.value is None
        assert lib.isdf_last_error(None).decode().startswith("isdf_create")
    rc = lib.isdf_create(ctypes.byref(h), 8, 8, 8, -1.0, 4.0, 4.0, None)
    assert rc == -2
    assert lib.isdf_create(None, 8, 8, 8, 1.0, 1.0, 1.0, None) == -1


def test_null_context_is_an_argument_error(lib):
    assert lib.isdf_fit(None, None, 1, 1, None, 1, 0, None, None) == -1
    assert lib.build_polarizability(None, None, None, 1, None, None) == -1
    assert lib.smw_inverse(None, 0, None) == -1
    assert lib.apply_eps_inv(None, 0, None, 1, None) == -1
    assert lib.isdf_destroy(None) == -1


def test_binding_raises_without_library(tmp_path):
    saved = pkg._lib
    try:
        pkg._lib = None
        with pytest.raises(ImportError):
            pkg.load_library(str(tmp_path / "missing.so"))
    finally:
        pkg._lib = saved
