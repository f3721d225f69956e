"""CPU-side checks of the C ABI: the library builds, loads, and exports every
function that include/tfft.h declares.  No compute call (no GPU here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if not fn.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", fn)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][\w \*]*?\b(tfft_\w+)\s*\(", text, re.M):
            names.add(m.group(1))
    return sorted(names)


def test_header_declares_the_core_calls():
    names = declared_functions()
    for core in ("tfft_plan", "tfft_exec", "tfft_report", "tfft_destroy"):
        assert core in names


def test_library_exports_every_declared_symbol():
    import paper_2405_02520_gb300 as t
    lib = t.lib()
    for name in declared_functions():
        assert hasattr(lib, name), name
        assert isinstance(getattr(lib, name), ctypes._CFuncPtr)


def test_error_strings_and_no_device_status():
    import paper_2405_02520_gb300 as t
    assert t.tfft_error_string(0) == "success"
    assert "invalid" in t.tfft_error_string(-1)
    try:
        import torch
        if torch.cuda.is_available():
            pytest.skip("GPU present: covered by the GPU tests")
    except ImportError:
        pass
    with pytest.raises(t.TfftError) as e:
        t.tfft_plan(1024, 4)
    assert e.value.code == -6


def test_struct_layouts_match_header_sizes():
    """The ctypes mirrors must have the C sizes (8-byte aligned fields)."""
    import paper_2405_02520_gb300 as t
    assert ctypes.sizeof(t.PlanOpts) == 88
    assert ctypes.sizeof(t.Stats) == 7 * 8
    assert ctypes.sizeof(t.FaultEvent) == 3 * 8 + 2 * 4 + 4 * 8
    assert ctypes.sizeof(t.Fault) == 4 * 4 + 3 * 8 + 8


def test_invalid_arguments_rejected_before_device_query():
    import paper_2405_02520_gb300 as t
    for n, b in ((12, 4), (0, 4), (1 << 30, 1), (8, 0)):
        with pytest.raises(t.TfftError) as e:
            t.tfft_plan(n, b)
        assert e.value.code == -1


def test_struct_layouts_match_compiled_header(tmp_path):
    """Sizes and field offsets of the ctypes mirrors equal those a C compiler
    gives the structs of include/tfft.h."""
    import shutil
    import subprocess
    import paper_2405_02520_gb300 as t
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = {"tfft_plan_opts": t.PlanOpts, "tfft_info": t.Info, "tfft_stats": t.Stats}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "tfft.h"', "int main(void) {"]
    for cname, py in structs.items():
        lines.append(f'  printf("{cname} size %zu\\n", sizeof({cname}));')
        for f, _ in py._fields_:
            lines.append(f'  printf("{cname} {f} %zu\\n", offsetof({cname}, {f}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    inc = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")
    subprocess.run([cc, "-I", inc, str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    got = {tuple(l.split()[:2]): int(l.split()[2]) for l in out if l.strip()}
    for cname, py in structs.items():
        assert got[(cname, "size")] == ctypes.sizeof(py), cname
        for f, _ in py._fields_:
            assert got[(cname, f)] == getattr(py, f).offset, (cname, f)
