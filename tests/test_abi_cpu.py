"""CPU-side checks of the C boundary: libeg.so loads and exports every entry
point include/eg.h declares, the header keeps to plain C types, and the
binding refuses to run without the library (no fallback)."""
from __future__ import annotations

import ctypes
import os
import re
import subprocess

import pytest

from paper_1710_03647_gb300 import build as egbuild
from paper_1710_03647_gb300 import eg

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", h) for h in sorted(os.listdir(os.path.join(ROOT, "include")))
           if h.endswith(".h")]


def declared_functions():
    names = []
    for h in HEADERS:
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for mt in re.finditer(r"^\s*(?:const\s+)?[a-z_0-9]+\s*\**\s*(eg_[a-z_0-9]+)\s*\(", text, flags=re.M):
            names.append(mt.group(1))
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    egbuild.build()
    return ctypes.CDLL(egbuild.LIB)


def test_header_declares_entry_points():
    names = declared_functions()
    for want in ("eg_create", "eg_destroy", "eg_bound", "eg_solve_credit", "eg_last_error", "eg_version"):
        assert want in names


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), f"{name} declared in include/*.h but not exported"


def test_binding_covers_every_declared_symbol():
    for name in declared_functions():
        assert name in eg.SIGNATURES, f"{name} has no binding"


def test_header_is_plain_c():
    for h in HEADERS:
        text = open(h).read()
        assert "torch" not in text.lower().replace("no torch", "")
        assert 'extern "C"' in text
        for bad in ("std::", "template", "class "):
            assert bad not in text


def test_version_string(lib):
    lib.eg_version.restype = ctypes.c_char_p
    assert lib.eg_version().startswith(b"eg-gb300")


def test_null_arguments_rejected_without_gpu(lib):
    # argument checks run before any CUDA call
    assert eg.load().eg_solve_credit(None, 0, 1, 0, None, None, None, 0) == eg.EG_ERR_INVALID
    out = ctypes.c_void_p()
    rc = eg.load().eg_create(0, 0, None, None, None, None, None, None, None, 0, ctypes.byref(out))
    assert rc == eg.EG_ERR_INVALID
    assert "n" in eg.eg_last_error()


def test_missing_library_fails_loudly(tmp_path):
    saved = eg._lib
    eg._lib = None
    try:
        with pytest.raises(ImportError):
            eg.load(str(tmp_path / "nope.so"))
    finally:
        eg._lib = saved


@pytest.mark.parametrize("struct", [eg.eg_stats, eg.eg_tuning, eg.eg_server_counters],
                         ids=lambda s: s.__name__)
def test_struct_layout_matches_header(tmp_path, struct):
    # each binding struct must have the C struct's size and field offsets
    name = struct.__name__
    src = tmp_path / "layout.c"
    fields = [f for f, _ in struct._fields_]
    body = "\n".join(f'printf("{f} %zu\\n", offsetof({name}, {f}));' for f in fields)
    src.write_text('#include <stddef.h>\n#include <stdio.h>\n#include "eg.h"\nint main(void) {\n'
                   f'printf("size %zu\\n", sizeof({name}));\n{body}\nreturn 0;\n}}\n')
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-std=c99", "-I", os.path.join(ROOT, "include"), "-o", str(exe), str(src)])
    got = dict(line.split() for line in subprocess.check_output([str(exe)], text=True).splitlines())
    assert int(got["size"]) == ctypes.sizeof(struct)
    for f in fields:
        assert int(got[f]) == getattr(struct, f).offset, f


def test_binding_constants_match_header():
    # every EG_* integer macro of the header has the same value in the binding
    # and the other way round (options, phases, statuses, server options)
    defined = {}
    for h in HEADERS:
        for mt in re.finditer(r"^#define\s+(EG_[A-Z0-9_]+)\s+\(?(-?\d+)\)?\s*(?:/\*.*)?$", open(h).read(), flags=re.M):
            defined[mt.group(1)] = int(mt.group(2))
    assert {"EG_OPT_SWEEPS", "EG_OPT_CHUNK_EDGES", "EG_OPT_KICK_ROUNDS", "EG_PHASE_LEVEL"} <= set(defined)
    for name, value in defined.items():
        if hasattr(eg, name):
            assert getattr(eg, name) == value, name
    opts = {n for n in defined if n.startswith("EG_OPT_")}
    assert opts == {n for n in dir(eg) if n.startswith("EG_OPT_")}
