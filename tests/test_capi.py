"""Host-side checks of the C ABI: the library loads, exports every declared
symbol, the header is valid C, and calls fail cleanly without a GPU."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "wd.h")


def declared_symbols():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(wd_[a-z0-9_]+)\s*\(", text)))


def test_header_is_plain_c():
    subprocess.check_call(["gcc", "-fsyntax-only", "-std=c99", "-Wall", "-Werror", "-x", "c", HEADER])
    subprocess.check_call(["g++", "-fsyntax-only", "-std=c++17", "-Wall", "-Werror", "-x", "c++", HEADER])


def test_library_exports_every_declared_symbol():
    import paper_2304_06340_b300 as wd
    lib = wd.library()
    syms = declared_symbols()
    assert "wd_distance" in syms and "wd_mesh_ft" in syms and len(syms) >= 18
    for s in syms:
        assert hasattr(lib, s), s
        assert hasattr(wd, s), "binding lacks " + s


def test_calls_fail_cleanly_without_a_gpu():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    import paper_2304_06340_b300 as wd
    with pytest.raises(wd.WDError) as e:
        wd.wd_create(0)
    assert e.value.status in (wd.WD_ECUDA, wd.WD_EINVAL)
    # null-argument paths return WD_EINVAL without touching the device
    lib = wd.library()
    assert lib.wd_rule_info(None, None, None) == wd.WD_EINVAL
    assert lib.wd_distance(None, None, None, None, ctypes.c_double(1.0), 0, None) == wd.WD_EINVAL
    assert lib.wd_last_error(None).decode()
    assert lib.wd_launch_count(None) == 0
