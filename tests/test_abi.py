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
    assert d.geom_mode.offset == 160 and d.equilibrium.offset == 164 and d.reserved.offset == 168
    assert ctypes.sizeof(d) == 176
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


def _desc(**kw):
    """A valid 8 x 16 x 8 cylinder descriptor with fields overridden by kw."""
    import math
    import lbw_workloads as W
    spec = W.GridSpec(kind=W.KIND_CYLINDRICAL, n=(8, 16, 8), h=(1, 2 * math.pi / 16, 1),
                      x0=(4, 0, 0), c=0.3,
                      bc=(W.BC_BOUNCE, W.BC_ANTIBOUNCE, 0, 0, W.BC_BOUNCE, W.BC_BOUNCE))
    d = lbw.make_desc(spec)
    for k, v in kw.items():
        if k == "bc":
            for i, b in enumerate(v):
                d.bc[i] = b
        else:
            setattr(d, k, v)
    return d


@pytest.mark.parametrize("fields,message", [
    ({"kind": 7}, "kind"),
    ({"damping": 1.5}, "damping"),
    ({"prec": 9}, "prec"),
    ({"bc": (0, 1, 0, 0, 1, 1)}, "pairs"),           # periodic on one q1 face only
    ({"bc": (1, 2, 1, 1, 1, 1)}, "angular"),         # theta not periodic
    ({"kind": 3, "horn_profile": 5}, "horn_profile"),
    ({"c": 1.5}, "too coarse"),                      # beyond the stability bound
    ({"x0": (-6.0, 0.0, 0.0)}, "metric undefined"),  # r <= 0 on the lattice
    ({"geom_mode": 3}, "geom_mode"),
    ({"equilibrium": 3}, "equilibrium"),
    ({"equilibrium": 1}, "Cartesian"),                # moment matching on a cylinder
    ({"reserved": 2}, "reserved"),
], ids=["kind", "damping", "prec", "periodic-pair", "angular", "horn", "stability", "metric",
        "geom-mode", "equilibrium", "eq-kind", "reserved"])
def test_descriptor_rules_are_checked_on_the_host(fields, message):
    """Every descriptor rule of lbw_create_grid is decided before any CUDA call: the status is
    LBW_EINVAL and the thread's last error names the rule."""
    d = _desc(**fields)
    out = ctypes.c_void_p()
    st = lbw.lib().lbw_create_grid(ctypes.byref(d), None, ctypes.byref(out))
    assert st == lbw.LBW_EINVAL
    assert message in lbw.lbw_last_error(), lbw.lbw_last_error()


def test_valid_descriptor_passes_the_host_checks():
    """The base descriptor of the rule table satisfies every rule (so each case above fails on
    its own field): it gets past validation to the first CUDA call, which fails without a GPU
    (LBW_ECUDA) and succeeds with one."""
    d = _desc()
    out = ctypes.c_void_p()
    st = lbw.lib().lbw_create_grid(ctypes.byref(d), None, ctypes.byref(out))
    assert st in (lbw.LBW_ECUDA, lbw.LBW_OK), lbw.lbw_last_error()
    if st == lbw.LBW_OK:
        lbw.lbw_destroy(out)
