"""The ctypes structures of the Python binding have the layout of the C
structures in include/fblts.h: a small C program compiled with the host
compiler prints sizeof and offsetof of every field, and each must equal the
binding's (a mismatch would pass wrong arguments silently)."""
import os
import shutil
import subprocess

import ctypes as C
import pytest

import paper_2405_10505_gb300 as fb

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PAIRS = [("fblts_mesh_desc", fb.MeshDesc), ("fblts_mesh_info", fb.MeshInfo), ("fblts_params", fb.Params),
         ("fblts_batch_opts", fb.BatchOpts), ("fblts_batch_info", fb.BatchInfo),
         ("fblts_server_opts", fb.ServerOpts), ("fblts_request_desc", fb.RequestDesc),
         ("fblts_request_info", fb.RequestInfo), ("fblts_server_stats", fb.ServerStats)]


def _c_layout(tmp_path):
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "fblts.h"', "int main(void) {"]
    for cname, cls in PAIRS:
        lines.append(f'    printf("{cname} sizeof %zu\\n", sizeof({cname}));')
        for f in cls._fields_:
            lines.append(f'    printf("{cname} {f[0]} %zu\\n", offsetof({cname}, {f[0]}));')
    lines += ["    return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    cuda_inc = "/usr/local/cuda/include"
    cmd = ["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), "-I", cuda_inc, str(src), "-o", str(exe)]
    subprocess.run(cmd, check=True, capture_output=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    return {(a, b): int(c) for a, b, c in (ln.split() for ln in out.splitlines())}


@pytest.mark.skipif(shutil.which("gcc") is None, reason="needs a C compiler")
def test_ctypes_structures_match_the_header(tmp_path):
    lay = _c_layout(tmp_path)
    for cname, cls in PAIRS:
        assert lay[(cname, "sizeof")] == C.sizeof(cls), cname
        for f in cls._fields_:
            assert lay[(cname, f[0])] == getattr(cls, f[0]).offset, (cname, f[0])
