"""The C-ABI library builds, loads without a GPU and exports every symbol its
headers declare; the binding declares a signature for each of them."""

import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
INC = os.path.join(ROOT, "include")


def _declared():
    names = set()
    for f in os.listdir(INC):
        if not f.endswith(".h"):
            continue
        src = open(os.path.join(INC, f)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w \*]*?\b(cs_\w+)\s*\(", src, flags=re.M):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_2412_18379_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_headers_declare_entry_points():
    names = _declared()
    for n in ("cs_create", "cs_mesh_upload", "cs_track", "cs_track_host", "cs_destroy"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in sorted(_declared()) if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    from paper_2412_18379_gb300 import _capi
    assert _declared() <= set(_capi.SIGNATURES), _declared() - set(_capi.SIGNATURES)


def test_create_without_gpu_fails_cleanly(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = ctypes.c_void_p()
    lib.cs_create.restype = ctypes.c_int32
    rc = lib.cs_create(ctypes.byref(h), 0, ctypes.c_size_t(0))
    assert rc != 0 and not h.value


def test_struct_layouts_match_the_header(tmp_path):
    """Every struct the binding mirrors has the header's size and field
    offsets (a C program built with gcc against include/cnnsns.h prints
    them): a field added, moved or retyped on one side only would make the
    library read or write the wrong bytes."""
    import shutil
    import subprocess
    from paper_2412_18379_gb300 import _capi
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no gcc")
    pairs = [("cs_mesh_info", _capi.MeshInfo), ("cs_serve_cfg", _capi.ServeCfg),
             ("cs_request", _capi.Request), ("cs_serve_stats", _capi.ServeStats),
             ("cs_serve_record", _capi.ServeRecord), ("cs_error_stats", _capi.ErrorStats),
             ("cs_profile", _capi.Profile)]
    lines = ['#include <stddef.h>', '#include <stdio.h>', '#include "cnnsns.h"', 'int main(void) {']
    want = []
    for cname, cls in pairs:
        lines.append('printf("%%zu\\n", sizeof(%s));' % cname)
        want.append(ctypes.sizeof(cls))
        for field, _ in cls._fields_:
            lines.append('printf("%%zu\\n", offsetof(%s, %s));' % (cname, field))
            want.append(getattr(cls, field).offset)
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([gcc, "-std=c11", "-I", INC, str(src), "-o", str(exe)], check=True)
    got = [int(x) for x in subprocess.run([str(exe)], check=True, capture_output=True,
                                          text=True).stdout.split()]
    assert got == want
