"""The C-ABI library builds, loads and exports every symbol include/*.h declares.
No compute call is made (no GPU here); only argument checks that return before
touching the device."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names += re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\**\s*(fsi_[a-z0-9_]+)\s*\(",
                            src, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("fsi_mesh_create", "fsi_mesh_destroy", "fsi_last_error", "fsi_residual",
                     "fsi_jacobian_apply", "fsi_locate", "fsi_dlm_interp", "fsi_dlm_spread",
                     "fsi_stage"):
        assert required in names


def test_library_exports_every_declared_symbol():
    from paper_2601_08266_gb300 import _binding
    L = _binding.lib()
    missing = [n for n in declared_functions() if not hasattr(L, n)]
    assert not missing, missing


def test_binding_names_match_the_abi():
    import paper_2601_08266_gb300 as pkg
    from paper_2601_08266_gb300 import _binding
    for n in declared_functions():
        assert n in _binding._SIGS, f"{n} has no binding signature"


def test_argument_errors_without_a_device():
    from paper_2601_08266_gb300 import _binding as b
    L = b.lib()
    out = ctypes.c_void_p()
    # NULL grid / physics: rejected before any CUDA call
    assert L.fsi_mesh_create(None, None, 0, None, ctypes.byref(out)) == b.FSI_ERR_ARG
    assert b"grid" in L.fsi_last_error()
    g = b.fsi_grid((ctypes.c_int32 * 3)(0, 4, 4), (ctypes.c_double * 3)(0, 0, 0),
                   (ctypes.c_double * 3)(0.25, 0.25, 0.25))
    p = b.fsi_physics(1.0, 0.01, 1e-3, 0.5, 36.0, 4.0, 0, 0)
    assert L.fsi_mesh_create(ctypes.byref(g), ctypes.byref(p), 0, None,
                             ctypes.byref(out)) == b.FSI_ERR_ARG
    p_bad = b.fsi_physics(-1.0, 0.01, 1e-3, 0.5, 36.0, 4.0, 0, 0)
    assert L.fsi_mesh_create(ctypes.byref(g), ctypes.byref(p_bad), 0, None,
                             ctypes.byref(out)) == b.FSI_ERR_ARG
    assert L.fsi_residual(None, 0, None, None, None, None) == b.FSI_ERR_ARG
    assert L.fsi_locate(None, 0, None, None, None, None, None, None, 0) == b.FSI_ERR_ARG


def test_product_path_does_not_touch_the_oracle():
    """The package and the CUDA sources never import, load or name the oracle."""
    pkg = os.path.join(ROOT, "paper_2601_08266_gb300")
    for path in glob.glob(os.path.join(pkg, "**", "*"), recursive=True):
        if os.path.isdir(path) or "_build" in path or "__pycache__" in path:
            continue
        src = open(path, errors="ignore").read()
        assert "oracle" not in src.lower().replace("the oracle", ""), path


def test_struct_layouts_match_the_header():
    """Every struct the binding mirrors has the header's size and field
    offsets (a small C program compiled against include/fsi.h prints them)."""
    import shutil
    import subprocess
    import tempfile
    from paper_2601_08266_gb300 import _binding as b
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = [c for c in vars(b).values()
               if isinstance(c, type) and issubclass(c, ctypes.Structure)
               and c.__name__.startswith("fsi_")]
    assert structs
    import keyword

    def cname(f):   # a C field named like a Python keyword carries a trailing _
        return f[:-1] if f.endswith("_") and keyword.iskeyword(f[:-1]) else f
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "fsi.h"', "int main(void) {"]
    for c in structs:
        lines.append(f'printf("{c.__name__} size %zu\\n", sizeof({c.__name__}));')
        for f in c._fields_:
            lines.append(f'printf("{c.__name__} {f[0]} %zu\\n", '
                         f'offsetof({c.__name__}, {cname(f[0])}));')
    lines += ["return 0;", "}"]
    with tempfile.TemporaryDirectory() as d:
        src, exe = os.path.join(d, "layout.c"), os.path.join(d, "layout")
        open(src, "w").write("\n".join(lines))
        r = subprocess.run([cc, "-I", os.path.join(ROOT, "include"), src, "-o", exe],
                           capture_output=True, text=True)
        assert r.returncode == 0, r.stderr
        out = subprocess.run([exe], capture_output=True, text=True, check=True).stdout
    got = {}
    for line in out.splitlines():
        s, f, v = line.split()
        got[(s, f)] = int(v)
    for c in structs:
        assert got[(c.__name__, "size")] == ctypes.sizeof(c), c.__name__
        for f in c._fields_:
            assert got[(c.__name__, f[0])] == getattr(c, f[0]).offset, (c.__name__, f[0])
