"""The C-ABI library builds, loads and exports every symbol include/fglt.h declares.

No compute call is made here (this runs without a GPU)."""
import ctypes
import os
import re

import pytest

import paper_2007_11111_gb300 as fg

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    include = os.path.join(ROOT, "include")
    for fn in os.listdir(include):
        if not fn.endswith(".h"):
            continue
        text = open(os.path.join(include, fn)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"\b(fglt_\w+)\s*\(", text):
            names.add(m.group(1))
    return names


def test_header_declares_the_boundary():
    names = declared_symbols()
    for must in ["fglt_create", "fglt_transform", "fglt_destroy", "fglt_transform_batched",
                 "fglt_stream_submit", "fglt_stream_poll"]:
        assert must in names


def test_library_exports_every_declared_symbol():
    lib = fg.load()
    missing = [s for s in sorted(declared_symbols()) if not hasattr(lib, s)]
    assert not missing, f"not exported: {missing}"


def test_binding_covers_every_declared_symbol():
    assert set(declared_symbols()) <= set(fg.EXPORTED)


def test_status_strings():
    lib = fg.load()
    assert lib.fglt_status_string(0) == b"ok"
    assert b"simple" in lib.fglt_status_string(fg.FGLT_ERR_INVALID_GRAPH)
    assert lib.fglt_status_string(12345) == b"unknown status"


def test_options_default_zeroes():
    opt = fg.fglt_options_default()
    assert opt.validate == 0 and opt.profile_stages == 0 and opt.serve_memory_budget == 0


def test_options_layout_matches_header(tmp_path):
    """The ctypes mirror of fglt_options has the C struct's size and field
    offsets (a small C program compiled against include/fglt.h prints them)."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    fields = [name for name, _ in fg.fglt_options._fields_]
    src = tmp_path / "layout.c"
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "fglt.h"', 'int main(void) {',
             '  printf("%zu\\n", sizeof(fglt_options));']
    lines += [f'  printf("%zu\\n", offsetof(fglt_options, {f}));' for f in fields]
    lines += ['  return 0;', '}']
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = [int(x) for x in subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split()]
    assert out[0] == ctypes.sizeof(fg.fglt_options)
    for f, off in zip(fields, out[1:]):
        assert getattr(fg.fglt_options, f).offset == off, f
