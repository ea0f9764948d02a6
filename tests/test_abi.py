"""The C-ABI library builds, loads and exports every entry point include/fluoro.h declares, and the
ctypes mirrors have the C layouts (no compute call: runs without a GPU)."""
import ctypes as C
import os
import re
import subprocess

import pytest

from paper_1706_03024_gb300 import build as B
from paper_1706_03024_gb300 import native as N

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "fluoro.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(flr_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    B.build()
    return N.load()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("flr_create", "flr_destroy", "flr_set_spectrum", "flr_set_dyes",
                     "flr_set_medium", "flr_set_sources", "flr_set_sensor", "flr_render",
                     "flr_read_tallies", "flr_status", "flr_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", B.LIB], capture_output=True, text=True,
                         check=True).stdout
    exported = set(re.findall(r"\b(flr_\w+)\b", out))
    for name in declared_functions():
        assert name in exported, name
        assert hasattr(lib, name)
    assert set(declared_functions()) == set(N.SIGNATURES), "binding and header disagree"


def test_binding_forwards_every_declared_entry_point():
    """native.py has a same-name Python function for each C entry point (argument marshalling
    only), so no call of the boundary is reachable only through the raw library object."""
    for name in declared_functions():
        assert callable(getattr(N, name, None)), name


def test_checked_build_exports_the_same_symbols(lib):
    """libfluoro_checked.so (FLR_CHECKED: device index tests) is the same boundary."""
    B.build(checked=True)
    out = subprocess.run(["nm", "-D", "--defined-only", B.LIB_CHECKED], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\b(flr_\w+)\b", out))
    assert set(declared_functions()) <= exported
    chk = C.CDLL(B.LIB_CHECKED)
    assert chk.flr_checked_build() == 1
    assert lib.flr_checked_build() == 0


def test_struct_layouts_match_header(tmp_path):
    src = tmp_path / "sizes.c"
    src.write_text(
        '#include <stdio.h>\n#include <stddef.h>\n#include "fluoro.h"\n'
        "int main(void){printf(\"%zu %zu %zu %zu %zu %zu %zu %zu\\n\","
        "sizeof(flr_source), sizeof(flr_medium), sizeof(flr_sensor), sizeof(flr_params),"
        "offsetof(flr_medium, conc), offsetof(flr_medium, solvent),"
        "offsetof(flr_params, film), offsetof(flr_params, regroup_interval));return 0;}\n")
    exe = tmp_path / "sizes"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True)
    got = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True,
                                          check=True).stdout.split()]
    want = [C.sizeof(N.flr_source), C.sizeof(N.flr_medium), C.sizeof(N.flr_sensor),
            C.sizeof(N.flr_params), N.flr_medium.conc.offset, N.flr_medium.solvent.offset,
            N.flr_params.film.offset, N.flr_params.regroup_interval.offset]
    assert got == want


def test_counter_names_match_header():
    text = open(HEADER).read()
    enum = re.search(r"enum\s*\{(.*?)\};", text, flags=re.S).group(1)
    enum = re.sub(r"/\*.*?\*/", "", enum, flags=re.S)
    names = [n.strip().split("=")[0].strip() for n in enum.split(",") if n.strip()]
    assert [n[len("FLR_C_"):].lower() for n in names] == N.COUNTER_NAMES
    assert len(names) == N.FLR_NCOUNTERS


def test_create_without_gpu_fails_cleanly(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    ctx = C.c_void_p()
    assert lib.flr_create(C.byref(ctx), 0) == N.FLR_ERR_ARG
    assert lib.flr_set_spectrum(None, 380.0, 5.0, 81) == N.FLR_ERR_ARG
    assert lib.flr_render(None, None, None) == N.FLR_ERR_ARG


def test_sources_compile_for_sm103a_only():
    assert B.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]
