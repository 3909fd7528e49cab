"""Reduced-precision storage forms against the FP64 oracle.

FP16 / BF16 storage keeps f_i / w_i (the deviation from the rest state P = 0, scaled by the
weight) in 16 bits and does all arithmetic in FP32.  Each stored value is rounded once per
step with unit roundoff u (FP16: 2^-11, BF16: 2^-8).  The scheme is non-dissipative
(tau = 1/2), so independent roundings accumulate like a random walk: after S steps the field
error is about u sqrt(S) relative; the bounds below allow 3 u sqrt(S).  Mode frequencies are
far less sensitive (rounding noise is broadband): the spectra must match within 0.5%, the
spec bound for the reduced-precision forms.
"""
import math

import numpy as np
import pytest

import oracle
from lbw_workloads import PREC_BF16S, PREC_F16S, PREC_F32, pulses, probes

from test_gpu_parity import SPECS, _run_both

pytestmark = pytest.mark.gpu

UNIT = {PREC_F16S: 2.0 ** -11, PREC_BF16S: 2.0 ** -8}
STEPS = 200


@pytest.mark.parametrize("prec", [PREC_F16S, PREC_BF16S], ids=["f16", "bf16"])
@pytest.mark.parametrize("name", ["cylinder", "torus", "trumpet_exp", "polar", "cartesian_tiled",
                                  "cylinder_wide"])
def test_sixteen_bit_field_error_bound(name, prec):
    spec = SPECS[name].with_(prec=prec)
    g, o, _, _ = _run_both(spec, STEPS, seed=31)
    Pg, Po = g.get_P(), o.get_P()
    rel = np.linalg.norm(Pg - Po) / np.linalg.norm(Po)
    assert rel <= 3 * UNIT[prec] * math.sqrt(STEPS), rel


@pytest.mark.parametrize("prec", [PREC_F32, PREC_F16S, PREC_BF16S], ids=["f32", "f16", "bf16"])
def test_mode_frequencies_within_half_percent(prec):
    """Polar annulus, 3000 steps: the device spectrum of a reduced-precision run against the
    oracle estimator on the FP64 oracle's series."""
    spec = SPECS["polar"].with_(prec=prec)
    g, o, _, _ = _run_both(spec, 3000, seed=41, nprobe=2)
    fg, _ = g.spectrum(0, 4)
    fo, _ = oracle.spectrum(o.read_probes()[0], 4)
    assert len(fg) == len(fo)
    np.testing.assert_allclose(fg, fo, rtol=5e-3 if prec != PREC_F32 else 1e-5)
