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
    assert ctypes.sizeof(t.PlanOpts) == 64
    assert ctypes.sizeof(t.Stats) == 7 * 8
    assert ctypes.sizeof(t.FaultEvent) == 3 * 8 + 2 * 4 + 4 * 8
    assert ctypes.sizeof(t.Fault) == 4 * 4 + 3 * 8 + 8


def test_invalid_arguments_rejected_before_device_query():
    import paper_2405_02520_gb300 as t
    for n, b in ((12, 4), (0, 4), (1 << 27, 1), (8, 0)):
        with pytest.raises(t.TfftError) as e:
            t.tfft_plan(n, b)
        assert e.value.code == -1
