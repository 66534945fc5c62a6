"""The ctypes structures of the binding match include/stereo.h field by field:
a small C program built against the header prints every field's offset and
each structure's size, and they must equal the ctypes layout (CPU only)."""
import ctypes
import os
import shutil
import subprocess
import tempfile

import pytest

import paper_1511_00758_gb300 as S

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
STRUCTS = {"stereo_config": S.Config, "stereo_result": S.Result, "stereo_stats": S.Stats,
           "stereo_tuning": S.Tuning, "stereo_pair": S.Pair}


def _c_layout():
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "stereo.h"', "int main(void) {"]
    for cname, cls in STRUCTS.items():
        lines.append(f'    printf("{cname} size %zu\\n", sizeof({cname}));')
        for fname, _ in cls._fields_:
            lines.append(f'    printf("{cname} {fname} %zu\\n", offsetof({cname}, {fname}));')
    lines += ["    return 0;", "}"]
    with tempfile.TemporaryDirectory() as d:
        src, exe = os.path.join(d, "layout.c"), os.path.join(d, "layout")
        with open(src, "w") as f:
            f.write("\n".join(lines) + "\n")
        subprocess.check_call([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), src, "-o", exe])
        out = subprocess.check_output([exe], text=True)
    got = {}
    for line in out.splitlines():
        parts = line.split()
        got[(parts[0], parts[1])] = int(parts[2])
    return got


def test_ctypes_structures_match_the_header():
    c = _c_layout()
    for cname, cls in STRUCTS.items():
        assert c[(cname, "size")] == ctypes.sizeof(cls), cname
        for fname, _ in cls._fields_:
            assert c[(cname, fname)] == getattr(cls, fname).offset, (cname, fname)


def test_binding_signatures_match_the_prototypes():
    """Every prototype of the header has a binding signature with its argument count."""
    import re
    hdr = re.sub(r"/\*.*?\*/", "", open(os.path.join(ROOT, "include", "stereo.h")).read(), flags=re.S)
    protos = re.findall(r"\b(?:int|void|size_t)\s+\**(stereo_\w+)\s*\(([^;]*?)\)\s*;", hdr, flags=re.S)
    assert len(protos) >= 20
    for name, args in protos:
        a = args.strip()
        n = 0 if a in ("", "void") else a.count(",") + 1
        assert name in S._SIGS, name
        assert len(S._SIGS[name][1]) == n, name
