"""The C-ABI library builds, loads without a GPU and exports every entry point
that include/*.h declares (no compute calls are made here)."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        src = re.sub(r"//[^\n]*", "", src)
        for m in re.finditer(r"\b(iga_[A-Za-z0-9_]+)\s*\(", src):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def lib_path():
    from paper_2010_10232_gb300 import build
    return build.build()


def test_library_exports_every_declared_symbol(lib_path):
    L = ctypes.CDLL(lib_path)
    declared = _declared()
    assert len(declared) >= 25
    missing = [n for n in sorted(declared) if not hasattr(L, n)]
    assert not missing, missing


def test_binding_declares_every_symbol(lib_path):
    from paper_2010_10232_gb300 import _ffi
    assert _declared() <= set(_ffi.exported_names()) | {"iga_ctx"}


def test_status_strings_and_defaults(lib_path):
    from paper_2010_10232_gb300 import _ffi
    L = _ffi.lib()
    assert L.iga_status_str(0) == b"IGA_OK"
    assert L.iga_status_str(-7) == b"IGA_E_UNSUPPORTED"
    prm = _ffi.IgaParams()
    L.iga_default_params(ctypes.byref(prm))
    assert prm.dim == 2 and prm.p == 3 and abs(prm.omega - 0.6) < 1e-15 and prm.nu_pre == 1
    assert prm.precond == 0 and prm.deflation == 1


def test_setup_rejects_bad_parameters_without_gpu_work(lib_path):
    """Argument validation happens before any device call."""
    from paper_2010_10232_gb300 import _ffi
    L = _ffi.lib()
    prm = _ffi.IgaParams()
    L.iga_default_params(ctypes.byref(prm))
    h = ctypes.c_void_p()
    for bad in ({"p": 0}, {"p": 6}, {"dim": 3}, {"n_el": 1}, {"n_vcycles": -1}, {"precision": 7},
                {"precond": 2}, {"deflation": 3}, {"n_vcycles": 0, "deflation": 0},
                {"deflation": 2, "precision": 1}, {"deflation": 2, "flexible": 1}):
        q = _ffi.IgaParams()
        ctypes.memmove(ctypes.byref(q), ctypes.byref(prm), ctypes.sizeof(prm))
        for field, v in bad.items():
            setattr(q, field, v)
        assert L.iga_setup(ctypes.byref(q), ctypes.byref(h)) == -1, bad
    q = _ffi.IgaParams()
    ctypes.memmove(ctypes.byref(q), ctypes.byref(prm), ctypes.sizeof(prm))
    q.precond, q.n_lines = 1, 1                 # exact CSLP needs constant k
    assert L.iga_setup(ctypes.byref(q), ctypes.byref(h)) == -7
    q = _ffi.IgaParams()
    ctypes.memmove(ctypes.byref(q), ctypes.byref(prm), ctypes.sizeof(prm))
    q.omega = 0.0
    assert L.iga_setup(ctypes.byref(q), ctypes.byref(h)) == -1
    assert L.iga_setup(None, ctypes.byref(h)) == -1
    assert L.iga_solve(None, None, None, 1e-7, 10, None, None, None) == -1


def test_params_struct_layout_matches_header(tmp_path):
    """The ctypes mirror of iga_params has the header's size and field offsets
    (checked by compiling a small C program against include/iga_helmholtz.h)."""
    import shutil
    import subprocess
    from paper_2010_10232_gb300 import _ffi
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    fields = [f for f, _ in _ffi.IgaParams._fields_]
    src = tmp_path / "layout.c"
    prog = ['#include <stdio.h>', '#include <stddef.h>', '#include "iga_helmholtz.h"', 'int main(void) {',
            '  printf("size %zu\\n", sizeof(iga_params));']
    prog += [f'  printf("{f} %zu\\n", offsetof(iga_params, {f}));' for f in fields]
    prog += ['  return 0;', '}']
    src.write_text("\n".join(prog) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = dict(line.split() for line in subprocess.run([str(exe)], check=True, capture_output=True,
                                                         text=True).stdout.splitlines())
    assert int(out["size"]) == ctypes.sizeof(_ffi.IgaParams)
    for f in fields:
        assert int(out[f]) == getattr(_ffi.IgaParams, f).offset, f
