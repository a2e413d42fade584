"""The C ABI library loads and exports every entry point include/rms.h
declares (no GPU needed: nothing is called that touches a device)."""
import ctypes as C
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"^\s*(?:const\s+)?[a-z_0-9]+\s*\*?\s*(rms_[a-z_0-9]+)\s*\(", text, re.M))
    return names


def test_library_builds_and_exports_every_declared_symbol():
    import __graft_entry__
    path = __graft_entry__._builder().build()
    lib = C.CDLL(path)
    names = declared_functions()
    assert {"rms_create_substrate", "rms_set_sequence", "rms_run", "rms_read_signal"} <= names
    missing = [n for n in sorted(names) if not hasattr(lib, n)]
    assert not missing, missing
    from paper_2012_06478_gb300 import _lib
    assert set(_lib.SIGNATURES) == names


def test_version_and_error_string_without_gpu():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2012_06478_gb300 import _lib
    assert _lib.lib.rms_version() == 10000
    assert isinstance(_lib.last_error(), str)


def test_invalid_arguments_rejected_on_host():
    """Descriptor checks happen before any device work."""
    from paper_2012_06478_gb300 import _lib
    h = C.c_void_p()
    assert _lib.lib.rms_create_substrate(None, C.byref(h)) == _lib.RMS_E_INVALID_ARG
    d = _lib.SubstrateDesc()
    d.nx = d.ny = d.nz = 4
    assert _lib.lib.rms_create_substrate(C.byref(d), C.byref(h)) == _lib.RMS_E_INVALID_ARG
    assert "null" in _lib.last_error()
    assert _lib.lib.rms_run(None, None, C.byref(h)) == _lib.RMS_E_INVALID_ARG
