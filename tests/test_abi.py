"""The C ABI without a GPU: the library builds, loads and exports every entry
point that include/riot.h declares, and the descriptor structs of the Python
binding have the layout the C compiler gives them."""
import ctypes
import os
import re
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "riot.h")


def _declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(riot_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("no CUDA toolkit to build the library")
    from paper_1906_01413_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_every_declared_entry_point_is_exported(lib):
    names = _declared_functions()
    assert len(names) >= 20
    missing = [nm for nm in names if not hasattr(lib, nm)]
    assert not missing, missing


def test_binding_structs_match_the_c_layout(tmp_path, lib):
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no C compiler")
    from paper_1906_01413_gb300 import riot as R
    structs = {"riot_model_desc": R.ModelDesc, "riot_obs_desc": R.ObsDesc, "riot_bcov_desc": R.BcovDesc,
               "riot_options": R.Options, "riot_advdiff_desc": R.AdvDiffDesc}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "riot.h"', "int main(void) {"]
    for cname, py in structs.items():
        lines.append('printf("%s size %%zu\\n", sizeof(%s));' % (cname, cname))
        for fname, _ in py._fields_:
            lines.append('printf("%s.%s %%zu\\n", offsetof(%s, %s));' % (cname, fname, cname, fname))
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run([gcc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = dict(line.rsplit(" ", 1) for line in out if line)
    for cname, py in structs.items():
        assert int(got["%s size" % cname]) == ctypes.sizeof(py), cname
        for fname, _ in py._fields_:
            assert int(got["%s.%s" % (cname, fname)]) == getattr(py, fname).offset, (cname, fname)


def test_status_strings_without_a_device(lib):
    lib.riot_status_string.restype = ctypes.c_char_p
    lib.riot_status_string.argtypes = [ctypes.c_int32]
    assert lib.riot_status_string(0) == b"ok"
    assert lib.riot_status_string(-1) == b"invalid argument"
    assert lib.riot_status_string(12345) == b"unknown status"


def test_every_entry_point_has_a_typed_binding(lib):
    """Each declared function has ctypes argtypes in the binding: without them Python ints
    would be passed as 32-bit ints (64-bit strides, stream ids and sizes truncated)."""
    from paper_1906_01413_gb300 import riot as R
    L = R.load()
    untyped = [nm for nm in _declared_functions() if getattr(L, nm).argtypes is None]
    assert not untyped, untyped
