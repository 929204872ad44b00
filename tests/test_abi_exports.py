"""The C-ABI library builds for sm_103a, loads without a GPU and exports every
entry point that include/iga.h declares (no compute calls)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = []
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not fn.endswith(".h"):
            continue
        txt = open(os.path.join(ROOT, "include", fn)).read()
        txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
        names += re.findall(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(iga_\w+)\s*\(", txt, flags=re.M)
    return sorted(set(names))


def test_library_exports_every_declared_symbol():
    from paper_2004_05197_gb300 import build
    lib_path = build.build()
    lib = ctypes.CDLL(lib_path)
    names = declared_symbols()
    assert len(names) >= 18, names
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    from paper_2004_05197_gb300 import build
    build.build()
    from paper_2004_05197_gb300 import iga
    assert set(declared_symbols()) <= set(iga.EXPORTED)
    for n in declared_symbols():
        assert callable(getattr(iga, n)), n


def test_error_path_without_gpu_compute():
    """Argument validation happens on the host before any device call."""
    from paper_2004_05197_gb300 import build
    build.build()
    from paper_2004_05197_gb300 import iga
    import pytest
    with pytest.raises(iga.IgaError) as e:
        iga.iga_space_create(4, 2, 64, iga.IGA_MAP_IDENTITY)
    assert e.value.code == iga.IGA_ERR_ARG
    assert "dim" in iga.iga_last_error()
    with pytest.raises(iga.IgaError):
        iga.iga_space_create(2, 2, 5, iga.IGA_MAP_IDENTITY)      # n_el < 4p+2
    with pytest.raises(iga.IgaError):
        iga.iga_space_create(3, 2, 16, iga.IGA_MAP_ANNULUS_QUARTER)
