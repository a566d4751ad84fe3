"""The ctypes mirrors of the C ABI's structs (paper_2603_01915_gb300) have
the size and field offsets the C compiler gives the structs declared in
include/dtans.h (checked with a small program built by the host compiler)."""
import os
import shutil
import subprocess
import tempfile

import pytest

import paper_2603_01915_gb300 as D

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
MIRRORS = {"dtans_encode_opts": D.EncodeOpts, "dtans_info_t": D.Info, "dtans_view_t": D.View,
           "dtans_tune_opts": D.TuneOpts, "dtans_tune_report": D.TuneReport}


def _c_layout():
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no host C compiler")
    lines = ['#include <stddef.h>', '#include <stdio.h>', '#include "dtans.h"', "int main(void) {"]
    for cname, py in MIRRORS.items():
        lines.append(f'  printf("{cname} sizeof %zu\\n", sizeof({cname}));')
        for f, _ in py._fields_:
            lines.append(f'  printf("{cname} {f} %zu\\n", offsetof({cname}, {f}));')
    lines += ["  return 0;", "}"]
    with tempfile.TemporaryDirectory() as d:
        src, exe = os.path.join(d, "layout.c"), os.path.join(d, "layout")
        with open(src, "w") as fh:
            fh.write("\n".join(lines) + "\n")
        subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), src, "-o", exe], check=True,
                       capture_output=True)
        out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout
    return {(a, b): int(c) for a, b, c in (ln.split() for ln in out.splitlines())}


def test_ctypes_structs_match_the_header():
    import ctypes as C
    lay = _c_layout()
    for cname, py in MIRRORS.items():
        assert C.sizeof(py) == lay[(cname, "sizeof")], cname
        for f, _ in py._fields_:
            assert getattr(py, f).offset == lay[(cname, f)], (cname, f)
