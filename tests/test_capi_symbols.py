"""CPU checks of the C ABI library: it builds, loads, and exports every entry
point include/dses.h declares; host-only calls behave without a GPU."""
import os
import re
import subprocess

import pytest

from paper_2502_00115_b300 import build as b
from paper_2502_00115_b300 import capi

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            text = open(os.path.join(ROOT, "include", f)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(dses_[a-z_]+)\s*\(", text))
    return names


@pytest.fixture(scope="module")
def lib():
    b.build()
    return capi.load()


def test_library_exports_every_declared_symbol(lib):
    declared = _declared()
    assert len(declared) >= 15
    out = subprocess.run(["nm", "-D", "--defined-only", b.LIB], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\bT (dses_[a-z_]+)\b", out))
    assert declared <= exported, declared - exported
    for name in declared:
        assert hasattr(lib, name)
    assert set(capi.SIGNATURES) >= declared


def test_status_strings(lib):
    assert capi.status_string(0) == "DSES_OK"
    assert capi.status_string(-6) == "DSES_ERR_NO_CANDIDATE"
    assert capi.status_string(-7) == "DSES_ERR_UNKNOWN_TICKET"
    assert capi.status_string(42) == "unknown status"


def test_struct_layouts_match_header(lib, tmp_path):
    # the ctypes mirrors must have the C compiler's sizes and field offsets
    import ctypes

    fields = {
        "dses_result": ["R", "t", "rot_index", "inliers", "votes", "cost", "status"],
        "dses_rotation_grid": ["kind", "hopf_n", "K", "delta_r", "R0", "explicit_R", "n_explicit"],
        "dses_params": ["metric", "epsilon", "delta_t", "tau", "huber_h", "p", "t_center", "t_half", "q_milli",
                        "top_k", "nn_mode", "refine_top_k", "refine_K", "refine_delta_r"],
        "dses_problem": ["target", "src", "n_src", "src_is_device", "grid", "params"],
    }
    prog = ["#include <stdio.h>", "#include <stddef.h>", '#include "dses.h"', "int main(void){"]
    for st, fs in fields.items():
        prog.append(f'printf("%zu\\n", sizeof({st}));')
        for f in fs:
            prog.append(f'printf("%zu\\n", offsetof({st}, {f}));')
    prog.append("return 0;}")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(prog))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I" + os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = [int(x) for x in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()]
    want = []
    for st, fs in fields.items():
        cls = getattr(capi, st)
        want.append(ctypes.sizeof(cls))
        want += [getattr(cls, f).offset for f in fs]
    assert got == want


def test_null_arguments_are_rejected_without_a_device(lib):
    assert lib.dses_destroy(None) == capi.DSES_ERR_INVALID_ARG
    assert lib.dses_register(None, None, None) == capi.DSES_ERR_INVALID_ARG
    assert lib.dses_poll(None, 1, None) == capi.DSES_ERR_INVALID_ARG
    assert lib.dses_last_error(None) == b"null context"
