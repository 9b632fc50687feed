"""CPU-side checks of the C ABI: the library builds for sm_103a, loads, and exports every
function include/lbe.h declares; struct layouts match the header."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def libpath():
    from paper_1612_04488_gb300 import build, lbe
    if not os.path.exists(lbe.LIB_PATH):
        build.build()
    return lbe.LIB_PATH


def declared_functions():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", f)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(lbe_[A-Za-z_0-9]+)\s*\(", txt))
    return names


def test_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    names = declared_functions()
    assert {"lbe_create", "lbe_solve", "lbe_apply_L", "lbe_sweep", "lbe_submit"} <= names
    for n in sorted(names):
        assert hasattr(lib, n), n


def test_status_strings_and_cells(libpath):
    from paper_1612_04488_gb300 import lbe
    L = lbe.lib()
    for s in range(8):
        assert L.lbe_status_str(s)
    assert lbe.cells_of(lbe.problem(dim=1, ns=100)) == 101
    assert lbe.cells_of(lbe.problem(dim=2, nx=64, ny=32)) == 2048


def test_struct_layouts():
    from paper_1612_04488_gb300 import lbe
    # lbe_geometry: 5 ints + pad + double; lbe_problem and lbe_result as laid out by a C compiler
    assert ctypes.sizeof(lbe.Geometry) == 32
    assert ctypes.sizeof(lbe.Problem) == 112
    assert ctypes.sizeof(lbe.Result) == 48


def test_no_cuda_device_gives_error_not_crash(libpath):
    import torch
    if torch.cuda.is_available():
        pytest.skip("device present")
    from paper_1612_04488_gb300 import lbe
    with pytest.raises(lbe.LbeError):
        lbe.Context(0)


def test_mixture_struct_layouts_match_the_header(tmp_path):
    """Offsets and sizes of the mixture structs, as a C compiler lays out include/lbe.h,
    against the ctypes binding."""
    import subprocess
    from paper_1612_04488_gb300 import lbe
    structs = {"lbe_mixture": lbe.Mixture, "lbe_mix_problem": lbe.MixProblem, "lbe_mix_result": lbe.MixResult}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "lbe.h"', "int main(void) {"]
    for cname, py in structs.items():
        lines.append('printf("%%s %%zu\\n", "%s", sizeof(%s));' % (cname, cname))
        for f, _ in py._fields_:
            lines.append('printf("%%s.%%s %%zu\\n", "%s", "%s", offsetof(%s, %s));' % (cname, f, cname, f))
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = dict(l.rsplit(" ", 1) for l in subprocess.run([str(exe)], capture_output=True, text=True,
                                                        check=True).stdout.split("\n") if l)
    for cname, py in structs.items():
        assert int(got[cname]) == ctypes.sizeof(py), cname
        for f, _ in py._fields_:
            assert int(got["%s.%s" % (cname, f)]) == getattr(py, f).offset, (cname, f)


def test_every_entry_point_rejects_null_arguments_without_a_device(libpath):
    """Every call that takes a context, batch or output pointer returns LBE_BAD_ARG for null
    arguments, before any CUDA call (so this runs without a GPU)."""
    from paper_1612_04488_gb300 import lbe
    lib = ctypes.CDLL(libpath)
    txt = ""
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            txt += re.sub(r"/\*.*?\*/", "", open(os.path.join(ROOT, "include", f)).read(), flags=re.S)
    decls = re.findall(r"\blbe_status\s+(lbe_[A-Za-z_0-9]+)\s*\(([^)]*)\)\s*;", txt)
    flags_only = {"lbe_set_kernel_timing", "lbe_debug_expire_waits"}   # take an int switch, nothing to reject
    checked = 0
    for name, params in decls:
        if name in flags_only:
            continue
        nargs = len([p for p in params.split(",") if p.strip() and p.strip() != "void"])
        fn = getattr(lib, name)
        fn.restype = ctypes.c_int
        assert fn(*([None] * nargs)) == lbe.BAD_ARG, name
        checked += 1
    assert checked >= 20
