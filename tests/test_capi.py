"""The C-ABI library loads, exports every symbol include/krl.h declares, its
structs have the layout the binding assumes, and argument errors come back as
status codes (none of these calls touch a GPU)."""
import ctypes as C
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "krl.h")


@pytest.fixture(scope="module")
def krl():
    from paper_2608_09340_gb300 import build as b
    b.build()
    import paper_2608_09340_gb300 as k
    k.load_library()
    return k


def _declared():
    txt = open(HEADER).read()
    return sorted(set(re.findall(r"^KRL_API[^;(]*?\b(krl_\w+)\s*\(", txt, flags=re.M)))


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("krl_grid_create", "krl_line_set", "krl_run_packets", "krl_tallies_get", "krl_tallies_reset"):
        assert n in names


def test_library_exports_every_declared_symbol(krl):
    out = subprocess.check_output(["nm", "-D", "--defined-only", krl.LIB_PATH], text=True)
    exported = set(re.findall(r"\sT\s(krl_\w+)", out))
    missing = [n for n in _declared() if n not in exported]
    assert not missing, missing
    assert set(krl.EXPORTS) <= exported


def test_struct_layouts_match_the_header(krl, tmp_path):
    """Compile a tiny C program against include/krl.h and compare sizeof /
    offsetof with the ctypes mirrors."""
    checks = {
        "krl_grid_desc": krl.krl_grid_desc, "krl_line_desc": krl.krl_line_desc,
        "krl_line_info": krl.krl_line_info, "krl_tune": krl.krl_tune, "krl_run_stats": krl.krl_run_stats,
    }
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "krl.h"', "int main(void){"]
    for cname, py in checks.items():
        lines.append(f'printf("{cname} %zu\\n", sizeof({cname}));')
        for f, _ in py._fields_:
            lines.append(f'printf("{cname}.{f} %zu\\n", offsetof({cname}, {f}));')
    lines.append('printf("krl_packet_record %zu\\n", sizeof(krl_packet_record));')
    lines.append("return 0;}")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    got = dict(l.split() for l in subprocess.check_output([str(exe)], text=True).splitlines())
    for cname, py in checks.items():
        assert int(got[cname]) == C.sizeof(py), cname
        for f, _ in py._fields_:
            assert int(got[f"{cname}.{f}"]) == getattr(py, f).offset, f"{cname}.{f}"
    assert int(got["krl_packet_record"]) == krl.RECORD_DTYPE.itemsize


def test_argument_errors_need_no_gpu(krl):
    lib = krl.load_library()
    h = C.c_void_p()
    assert lib.krl_grid_create(C.byref(h), None, None) == krl.KRL_ERR_ARG
    d = krl.krl_grid_desc()
    d.nx, d.ny, d.nz, d.cell_cm, d.T_K = 0, 1, 1, 1.0, 1e4
    assert lib.krl_grid_create(C.byref(h), C.byref(d), None) == krl.KRL_ERR_ARG
    assert b"dimensions" in lib.krl_last_error()
    d.nx, d.opacity_kind = 1, 7
    assert lib.krl_grid_create(C.byref(h), C.byref(d), None) == krl.KRL_ERR_ARG
    d.opacity_kind, d.cell_cm = 0, -1.0
    assert lib.krl_grid_create(C.byref(h), C.byref(d), None) == krl.KRL_ERR_ARG
    d.cell_cm, d.opacity = 1.0, None
    assert lib.krl_grid_create(C.byref(h), C.byref(d), None) == krl.KRL_ERR_ARG
    assert lib.krl_line_set(None, None, None) == krl.KRL_ERR_ARG
    assert lib.krl_run_packets(None, 1, 0, 0, None, None, None, None) == krl.KRL_ERR_ARG
    assert lib.krl_tallies_get(None, 0, None, 0, None) == krl.KRL_ERR_ARG
    assert lib.krl_tallies_reset(None, None) == krl.KRL_ERR_ARG
    assert lib.krl_tally_bytes(None, 0) == 0
    assert lib.krl_grid_destroy(None) == krl.KRL_OK
    assert lib.krl_version() >= 100


def test_missing_library_fails_loudly(krl, tmp_path):
    with pytest.raises(ImportError):
        krl.load_library(str(tmp_path / "nope.so"))
