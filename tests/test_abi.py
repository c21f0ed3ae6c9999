"""The C-ABI library builds for sm_103a, loads without a GPU and exports every
symbol include/rascas_gb300.h declares (no compute calls here)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "rascas_gb300.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(rascas_[a-z_0-9]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ["rascas_create", "rascas_destroy", "rascas_load_octree", "rascas_set_domain",
                 "rascas_set_lines", "rascas_set_physics", "rascas_set_detector", "rascas_propagate",
                 "rascas_get_tally", "rascas_ray_tau", "rascas_trace", "rascas_last_error"]:
        assert must in names


def test_library_loads_and_exports_all_symbols():
    from paper_2001_11252_gb300 import build
    path = build.build()
    lib = ctypes.CDLL(path)
    for name in declared_functions():
        assert hasattr(lib, name), name
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (rascas_\w+)", out))
    assert set(declared_functions()) <= exported


def test_binding_fails_loudly_without_gpu():
    """No CPU fallback: without a CUDA device context creation raises."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    import paper_2001_11252_gb300 as rg
    with pytest.raises(Exception):
        rg.Context(0)


def test_binding_constants_match_header():
    """The enum values the binding passes through the ABI are the header's."""
    import paper_2001_11252_gb300 as rg
    src = open(HEADER).read()
    enums = dict((k, int(v)) for k, v in re.findall(r"\b(RASCAS_[A-Z_0-9]+)\s*=\s*(-?\d+)", src))
    for name in ["DOMAIN_SPHERE", "DOMAIN_SLAB", "DOMAIN_CUBE", "DOMAIN_SHELL", "VOIGT_TASITSIOMI", "VOIGT_FADDEEVA"]:
        assert getattr(rg, name) == enums["RASCAS_" + name], name


def test_binding_struct_layouts_match_header(tmp_path):
    """Every struct the binding passes through the ABI has the header's size
    and field offsets (a C program built against the header prints them)."""
    from paper_2001_11252_gb300 import _native as N
    structs = {"rascas_octree": N.Octree, "rascas_domain": N.Domain, "rascas_line": N.Line,
               "rascas_dust": N.Dust, "rascas_physics": N.Physics, "rascas_detector": N.Detector,
               "rascas_packets_in": N.PacketsIn, "rascas_packets_out": N.PacketsOut,
               "rascas_run_stats": N.Stats, "rascas_event": N.Event, "rascas_model": N.Model,
               "rascas_tune": N.Tune}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "rascas_gb300.h"', "int main(void) {"]
    for cname, py in structs.items():
        lines.append('printf("%s __sizeof__ %%zu\\n", sizeof(%s));' % (cname, cname))
        for f in py._fields_:
            lines.append('printf("%s %s %%zu\\n", offsetof(%s, %s));' % (cname, f[0], cname, f[0]))
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    got = {}
    for ln in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.splitlines():
        a, b, c = ln.split()
        got[(a, b)] = int(c)
    for cname, py in structs.items():
        assert got[(cname, "__sizeof__")] == ctypes.sizeof(py), cname
        for f in py._fields_:
            assert got[(cname, f[0])] == getattr(py, f[0]).offset, (cname, f[0])
