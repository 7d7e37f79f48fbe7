"""The C ABI without a GPU: the library builds, loads and exports every
function include/pa.h declares, and the ctypes layout of pa_options matches
the C compiler's."""
import ctypes as C
import re
import subprocess
from pathlib import Path

import pytest

from paper_2409_11515_gb300 import build, pa

ROOT = Path(__file__).resolve().parent.parent
HEADER = ROOT / "include" / "pa.h"


@pytest.fixture(scope="module")
def lib():
    build.build()
    return pa.load()


def declared_functions():
    text = re.sub(r"/\*.*?\*/", "", HEADER.read_text(), flags=re.S)
    names = set(re.findall(r"\b(pa_[a-z_]+)\s*\(", text))
    # typedef'd function pointer types are not exports
    names -= set(re.findall(r"\(\s*\*\s*(pa_[a-z_]+)\s*\)", text))
    return sorted(names)


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("pa_create", "pa_estimate", "pa_estimate_batched", "pa_run", "pa_destroy",
                 "pa_last_error", "pa_get_vector"):
        assert must in names


def test_every_declared_function_is_exported(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", str(pa.LIB_PATH)], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\bT (pa_[a-z_]+)$", out, flags=re.M))
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, missing
    assert set(pa.EXPORTS) <= exported


def test_options_layout_matches_c(tmp_path, lib):
    src = tmp_path / "layout.c"
    src.write_text(
        '#include <stdio.h>\n#include <stddef.h>\n#include "pa.h"\n'
        "int main(void){printf(\"%zu %zu %zu %zu\\n\", sizeof(pa_options),"
        " offsetof(pa_options, barrier_timeout_ns), offsetof(pa_options, grid_blocks),"
        " offsetof(pa_options, debug_skip_arrival));"
        "printf(\" %zu %zu\\n\", offsetof(pa_options, fp64_tail),"
        " offsetof(pa_options, autotune));return 0;}\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", str(ROOT / "include"), str(src), "-o", str(exe)], check=True)
    got = list(map(int, subprocess.run([str(exe)], capture_output=True, text=True,
                                       check=True).stdout.split()))
    O = pa.Options
    assert got == [C.sizeof(O), O.barrier_timeout_ns.offset, O.grid_blocks.offset,
                   O.debug_skip_arrival.offset, O.fp64_tail.offset, O.autotune.offset]


def test_defaults_and_errors_without_gpu(lib):
    o = pa.options()
    assert o.loss == pa.LOSS_LOGRATIO and o.precision == pa.FP64 and o.barrier_timeout_ns > 0
    # argument checks run before any CUDA call
    raw = C.c_void_p()
    st = lib.pa_create(C.byref(raw), -1, 3, 0, None, None, None, pa.HOST, C.byref(o), None)
    assert st == -1 and b"negative" in lib.pa_last_error()
    assert lib.pa_estimate(None, 1, 10, 1e-2, 0.9, 0.999, 1e-12, 1, None, None, None) == -1
    lib.pa_destroy(None)  # NULL-safe
    assert lib.pa_kernel_launches(None) == -1
