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


def test_ctypes_structs_match_the_header_layout(tmp_path):
    """Every descriptor the binding passes by pointer has, field by field, the
    offsets and size that a C compiler gives the struct in include/rms.h
    (gcc on this host; the header includes only stddef.h and stdint.h)."""
    import subprocess
    from paper_2012_06478_gb300 import _lib
    structs = {"rms_substrate_desc": _lib.SubstrateDesc, "rms_sequence_desc": _lib.SequenceDesc,
               "rms_run_desc": _lib.RunDesc, "rms_run_state": _lib.RunState,
               "rms_server_config": _lib.ServerConfig}
    c_name = {"lam": "lambda"}  # the C member `lambda` is a Python keyword
    lines = ['#include <stdio.h>', '#include "rms.h"', "int main(void) {"]
    for cname, py in structs.items():
        lines.append(f'printf("{cname} size %zu\\n", sizeof({cname}));')
        for fname, _ in py._fields_:
            lines.append(f'printf("{cname} {fname} %zu\\n", offsetof({cname}, {c_name.get(fname, fname)}));')
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    c_layout = {}
    for ln in subprocess.check_output([str(exe)], text=True).splitlines():
        cname, field, val = ln.split()
        c_layout[(cname, field)] = int(val)
    for cname, py in structs.items():
        assert C.sizeof(py) == c_layout[(cname, "size")], cname
        for fname, _ in py._fields_:
            assert getattr(py, fname).offset == c_layout[(cname, fname)], (cname, fname)


def test_binding_argument_counts_match_the_prototypes():
    """Each ctypes signature takes as many arguments as its prototype in
    include/rms.h, and returns a pointer-sized value exactly where the
    prototype returns a pointer."""
    from paper_2012_06478_gb300 import _lib
    text = ""
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text += open(os.path.join(ROOT, "include", fn)).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    protos = {}
    for m in re.finditer(r"^\s*((?:const\s+)?[a-z_0-9]+\s*\**)\s*(rms_[a-z_0-9]+)\s*\(([^;{]*?)\)\s*;", text, re.M | re.S):
        ret, name, params = m.group(1), m.group(2), " ".join(m.group(3).split())
        n = 0 if params in ("", "void") else params.count(",") + 1
        protos[name] = (n, "*" in ret)
    assert set(protos) == set(_lib.SIGNATURES)
    for name, (args, res) in _lib.SIGNATURES.items():
        n, ptr = protos[name]
        assert len(args) == n, (name, len(args), n)
        assert ptr == (res in (C.c_char_p, C.c_void_p)), name


def test_package_refuses_to_import_without_the_library(tmp_path):
    """No CPU fallback: a copy of the package without librms.so fails to
    import, naming the missing library."""
    import shutil
    import subprocess
    import sys
    src = os.path.join(ROOT, "paper_2012_06478_gb300")
    dst = tmp_path / "paper_2012_06478_gb300"
    dst.mkdir()
    for fn in os.listdir(src):
        if fn.endswith(".py"):
            shutil.copy(os.path.join(src, fn), dst / fn)
    r = subprocess.run([sys.executable, "-c", "import paper_2012_06478_gb300"], cwd=tmp_path,
                       capture_output=True, text=True, env={**os.environ, "PYTHONPATH": str(tmp_path)})
    assert r.returncode != 0
    assert "ImportError" in r.stderr and "librms.so" in r.stderr and "no CPU fallback" in r.stderr


def test_product_code_never_reaches_the_oracle():
    """The oracle is test infrastructure: neither the package nor the input
    generators import it, and the package links nothing from oracle/."""
    pat = re.compile(r"^\s*(import\s+oracle\b|from\s+oracle\b)|librms_oracle|rms_oracle\.c", re.M)
    for top in ("paper_2012_06478_gb300", "rms_inputs"):
        for dirpath, _, files in os.walk(os.path.join(ROOT, top)):
            for fn in files:
                if fn.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                    text = open(os.path.join(dirpath, fn), encoding="utf-8").read()
                    assert not pat.search(text), os.path.join(dirpath, fn)


def test_normalise_partials_on_the_host():
    """rms_normalise_partials is host arithmetic (no device): S = num / sum
    alpha element by element, the division rms_read_signal applies; bad
    sizes and null arrays are refused."""
    import numpy as np
    from paper_2012_06478_gb300 import _lib
    import paper_2012_06478_gb300 as rms
    rng = np.random.default_rng(5)
    num = rng.normal(size=(2, 3, 4)) + 1j * rng.normal(size=(2, 3, 4))
    S = rms.rms_normalise_partials(num, 7.25)
    np.testing.assert_array_equal(S.real, num.real / 7.25)
    np.testing.assert_array_equal(S.imag, num.imag / 7.25)
    assert S.shape == num.shape
    assert _lib.lib.rms_normalise_partials(-1, None, None, 1.0, None, None) == _lib.RMS_E_INVALID_ARG
    assert _lib.lib.rms_normalise_partials(3, None, None, 1.0, None, None) == _lib.RMS_E_INVALID_ARG
    assert _lib.lib.rms_normalise_partials(0, None, None, 1.0, None, None) == _lib.RMS_OK


def test_binding_constants_match_the_header():
    """Every integer #define of include/*.h that the ctypes binding also
    defines has the same value there (status codes, precision forms, run
    flags, interactions, serving policies, peak kinds)."""
    from paper_2012_06478_gb300 import _lib
    seen = 0
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if not fn.endswith(".h"):
            continue
        for name, val in re.findall(r"^#define\s+(RMS_[A-Z0-9_]+)\s+\(?(-?\d+)u?\)?\s", open(
                os.path.join(ROOT, "include", fn)).read(), re.M):
            if hasattr(_lib, name):
                assert getattr(_lib, name) == int(val), (name, getattr(_lib, name), val)
                seen += 1
    assert seen >= 25, seen
