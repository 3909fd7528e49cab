"""The C-ABI library builds for sm_103a, loads without a GPU and exports every symbol that
include/lbw.h declares (no compute calls here)."""
import ctypes
import os
import re

import pytest

from paper_1705_01801_gb300 import lbw

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "lbw.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(lbw_[a-z0-9_]+)\s*\(", text)))


def test_header_matches_binding_list():
    assert declared_symbols() == sorted(lbw.EXPORTS)


def test_library_exports_every_declared_symbol():
    L = lbw.lib()
    for name in declared_symbols():
        assert hasattr(L, name), name


def test_struct_layout_matches_header():
    # kind(4) n(12) pad(0) h(24)...: offsets follow C rules for the declared field order
    d = lbw.lbw_grid_desc
    assert d.h.offset == 16 and d.c.offset == 64 and d.geom.offset == 96
    assert ctypes.sizeof(d) == 168
    assert ctypes.sizeof(lbw.lbw_pulse) == 40


def test_invalid_descriptor_rejected_without_gpu():
    """Validation runs on the host before any CUDA call."""
    desc = lbw.lbw_grid_desc()
    desc.kind = 2
    desc.n[0] = desc.n[1] = desc.n[2] = 8
    desc.tau = 0.7  # only tau = 1/2 is defined
    out = ctypes.c_void_p()
    st = lbw.lib().lbw_create_grid(ctypes.byref(desc), None, ctypes.byref(out))
    assert st == lbw.LBW_EINVAL
    assert "tau" in lbw.lbw_last_error()
