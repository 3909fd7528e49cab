"""CUDA path (through the C ABI) against the FP64 oracle on the same seeded inputs.

Tolerances:
  FP64 storage: populations agree element by element to 1e-11 relative to the field's
      largest magnitude (both sides are FP64; only the summation order differs).
  FP32 storage: relative L2 of P <= 1e-5 after 200 steps; element-wise populations within
      2e-5 of the field's largest magnitude.  One FP32 step from a shared state agrees with
      the oracle to 1e-6 of the largest population (rounding of one step, ~6e-8 per op).
  Probe series and spectra: the same estimator on both sides; peak frequencies to 1e-8
      relative for FP64 inputs (the golden-section comparisons turn over at rounding level
      once the bracket is ~1e-10 rad/step wide).
"""
import math

import numpy as np
import pytest

import oracle
from lbw_workloads import (BC_ANTIBOUNCE, BC_BOUNCE, BC_FREE, BC_PERIODIC, KIND_CARTESIAN,
                           KIND_CYLINDRICAL, KIND_POLAR, KIND_TOROIDAL, KIND_TRUMPET,
                           PREC_F32, PREC_F64, PROFILE_BESSEL, PROFILE_EXP, GridSpec, pulses,
                           probes)

pytestmark = pytest.mark.gpu

TWO_PI = 2 * math.pi

# shapes span several CTA tiles along q2 and q1 with ragged tails; q2 extents that are
# multiples of 64 run the TMA tile kernel, the others the register-pipelined kernel
SPECS = {
    "cartesian_mixed": GridSpec(kind=KIND_CARTESIAN, n=(9, 40, 11), h=(1, 1, 1), x0=(0, 0, 0),
                                c=0.45, bc=(BC_FREE, BC_BOUNCE, BC_ANTIBOUNCE, BC_FREE,
                                            BC_PERIODIC, BC_PERIODIC), damping=0.9),
    "polar": GridSpec(kind=KIND_POLAR, n=(40, 64, 1), h=(1, TWO_PI / 64, 1), x0=(7, 0, 0),
                      c=0.4, bc=(BC_BOUNCE, BC_ANTIBOUNCE, 0, 0, 0, 0)),
    "cylinder": GridSpec(kind=KIND_CYLINDRICAL, n=(23, 192, 19), h=(1, TWO_PI / 192, 1),
                         x0=(13, 0, 0), c=0.4,
                         bc=(BC_BOUNCE, BC_ANTIBOUNCE, 0, 0, BC_ANTIBOUNCE, BC_FREE)),
    "trumpet_exp": GridSpec(kind=KIND_TRUMPET, n=(17, 96, 33), h=(1, TWO_PI / 96, 1),
                            x0=(7, 0, 0), c=0.4, geom=(20.0, 4.0, 0.05, 0),
                            profile=PROFILE_EXP,
                            bc=(BC_FREE, BC_BOUNCE, 0, 0, BC_BOUNCE, BC_FREE), damping=0.65),
    "trumpet_bessel": GridSpec(kind=KIND_TRUMPET, n=(12, 64, 20), h=(1, TWO_PI / 64, 1),
                               x0=(14, 0, 0), c=0.4, geom=(60.0, 0.2, 0, 0),
                               profile=PROFILE_BESSEL,
                               bc=(BC_BOUNCE, BC_BOUNCE, 0, 0, BC_BOUNCE, BC_FREE)),
    # q2 extent of 50 is not a whole number of 16-byte vectors: register-pipelined kernel
    "cylinder_unstaged": GridSpec(kind=KIND_CYLINDRICAL, n=(11, 50, 9), h=(1, TWO_PI / 50, 1),
                                  x0=(9, 0, 0), c=0.4,
                                  bc=(BC_BOUNCE, BC_FREE, 0, 0, BC_BOUNCE, BC_ANTIBOUNCE)),
    "torus": GridSpec(kind=KIND_TOROIDAL, n=(13, 128, 24), h=(1, TWO_PI / 128, TWO_PI / 24),
                      x0=(4, 0, 0), c=0.4, geom=(40.0, 0, 0, 0),
                      bc=(BC_FREE, BC_BOUNCE, 0, 0, 0, 0)),
    # tile kernel with every q2 face rule (two tiles of 64, or one of 128 for 16-bit storage)
    "cartesian_tiled": GridSpec(kind=KIND_CARTESIAN, n=(9, 128, 11), h=(1, 1, 1), x0=(0, 0, 0),
                                c=0.45, bc=(BC_FREE, BC_BOUNCE, BC_ANTIBOUNCE, BC_FREE,
                                            BC_BOUNCE, BC_ANTIBOUNCE), damping=0.9),
    # 16-bit storage: two 128-column tiles, q3 faces with anti-bounce-back and free ends
    "cylinder_wide": GridSpec(kind=KIND_CYLINDRICAL, n=(21, 256, 17), h=(1, TWO_PI / 256, 1),
                              x0=(26, 0, 0), c=0.4,
                              bc=(BC_BOUNCE, BC_ANTIBOUNCE, 0, 0, BC_ANTIBOUNCE, BC_FREE)),
}


def _run_both(spec, steps, seed, nprobe=4):
    pl = pulses(spec, seed, 2, sigma=2.5, random_phase=True, margin=2)
    pr = probes(spec, seed, nprobe, margin=0)
    from paper_1705_01801_gb300 import lbw
    g = lbw.Grid(spec)
    g.init(pl)
    g.set_probes(pr, steps)
    o = oracle.OracleGrid(spec)
    o.init(pl)
    o.set_probes(pr, steps)
    f0_gpu, f0_or = g.get_f(), o.get_f()
    g.step(steps)
    o.step(steps)
    return g, o, f0_gpu, f0_or


@pytest.mark.parametrize("name", list(SPECS))
def test_fp64_populations_match_oracle(name):
    spec = SPECS[name].with_(prec=PREC_F64)
    g, o, f0g, f0o = _run_both(spec, 150, seed=11)
    scale = np.abs(f0o).max()
    np.testing.assert_allclose(f0g, f0o, rtol=0, atol=1e-12 * scale)  # initial state
    fg, fo = g.get_f(), o.get_f()
    assert np.isfinite(fg).all()
    np.testing.assert_allclose(fg, fo, rtol=0, atol=1e-11 * np.abs(fo).max())
    np.testing.assert_allclose(g.get_P(), o.get_P(), rtol=0,
                               atol=1e-11 * np.abs(o.get_P()).max())
    sg, so = g.read_probes(), o.read_probes()
    assert sg.shape == so.shape == (4, 150)
    np.testing.assert_allclose(sg, so, rtol=0, atol=1e-11 * np.abs(so).max())
    assert g.step_count() == 150


@pytest.mark.parametrize("name", list(SPECS))
def test_fp32_field_within_tolerance(name):
    spec = SPECS[name].with_(prec=PREC_F32)
    g, o, _, _ = _run_both(spec, 200, seed=12)
    Pg, Po = g.get_P(), o.get_P()
    rel = np.linalg.norm(Pg - Po) / np.linalg.norm(Po)
    assert rel <= 1e-5, rel
    fg, fo = g.get_f(), o.get_f()
    np.testing.assert_allclose(fg, fo, rtol=0, atol=2e-5 * np.abs(fo).max())


def test_single_step_from_shared_state_fp32_full_size():
    """Full-size cylinder 128 x 128 x 256 in the benchmark's launch configuration: one GPU
    step from a random shared state equals one oracle step (every node compared)."""
    import lbw_workloads as W
    spec = W.cylinder()
    rng = np.random.default_rng(5)
    f = rng.standard_normal((7,) + (spec.n[2], spec.n[0], spec.n[1])).astype(np.float32)
    from paper_1705_01801_gb300 import lbw
    g = lbw.Grid(spec)
    g.set_f(f.astype(np.float64))
    o = oracle.OracleGrid(spec)
    o.set_f(f.astype(np.float64))
    g.step(1)
    o.step(1)
    fg, fo = g.get_f(), o.get_f()
    np.testing.assert_allclose(fg, fo, rtol=0, atol=1e-6 * np.abs(fo).max())


def test_graph_chain_equals_single_launches():
    """64-step CUDA-graph chains and single launches give identical bits."""
    spec = SPECS["cylinder"].with_(prec=PREC_F32)
    from paper_1705_01801_gb300 import lbw
    pl = pulses(spec, 3, 1, sigma=2.5)
    a = lbw.Grid(spec)
    a.init(pl)
    a.step(131)
    b = lbw.Grid(spec)
    b.init(pl)
    for _ in range(131):
        b.step(1)
    assert np.array_equal(a.get_f(), b.get_f())


def test_zero_steps_and_empty_probe_set():
    spec = SPECS["polar"].with_(prec=PREC_F64)
    from paper_1705_01801_gb300 import lbw
    g = lbw.Grid(spec)
    g.init(pulses(spec, 1, 1))
    f0 = g.get_f()
    g.step(0)
    assert np.array_equal(g.get_f(), f0)
    g.set_probes(np.zeros((0, 3), np.int32), 0)
    g.step(3)
    assert g.read_probes().shape == (0, 0)


def test_step_before_init_is_a_state_error():
    from paper_1705_01801_gb300 import lbw
    g = lbw.Grid(SPECS["polar"])
    with pytest.raises(lbw.LbwError) as e:
        g.step(1)
    assert e.value.status == lbw.LBW_ESTATE


def test_spectrum_series_matches_oracle_estimator():
    from paper_1705_01801_gb300 import lbw
    t = np.arange(6000)
    rng = np.random.default_rng(3)
    x = (np.cos(0.0211 * t + 0.3) + 0.4 * np.cos(0.0537 * t + 1.1) + 0.2 * np.cos(0.131 * t)
         + 0.01 * rng.standard_normal(t.size))
    (fg, ag), = lbw.lbw_spectrum_series(x, 3)
    fo, ao = oracle.spectrum(x, 3)
    np.testing.assert_allclose(fg, fo, rtol=1e-8)
    np.testing.assert_allclose(ag, ao, rtol=1e-7)


def test_probe_spectrum_matches_oracle_on_polar_run():
    """Device spectrum of a recorded probe vs the oracle estimator on the oracle's series."""
    spec = SPECS["polar"].with_(prec=PREC_F64)
    g, o, _, _ = _run_both(spec, 3000, seed=21, nprobe=2)
    fg, ag = g.spectrum(0, 4)
    fo, ao = oracle.spectrum(o.read_probes()[0], 4)
    np.testing.assert_allclose(fg, fo, rtol=1e-8)
    fsum, _ = g.spectrum(-1, 4)
    fosum, _ = oracle.spectrum(o.read_probes().sum(0), 4)
    np.testing.assert_allclose(fsum, fosum, rtol=1e-8)


# one- and two-node extents on each axis, through the tile kernel (q2 = 64 or 128) and the
# register-pipelined kernel (q2 = 1, 3 or 40), with walls of every kind on the short axes
DEGENERATE = {
    "n1=1 tile": ((1, 64, 9), (BC_BOUNCE, BC_ANTIBOUNCE, 0, 0, BC_FREE, BC_BOUNCE)),
    "n1=2 tile": ((2, 128, 5), (BC_FREE, BC_FREE, 0, 0, 0, 0)),
    "n3=1 tile walls": ((9, 64, 1), (BC_BOUNCE, BC_FREE, 0, 0, BC_ANTIBOUNCE, BC_BOUNCE)),
    "n1=n3=1 tile": ((1, 64, 1), (BC_ANTIBOUNCE, BC_BOUNCE, 0, 0, BC_BOUNCE, BC_FREE)),
    "n3=2 tile": ((3, 64, 2), (BC_BOUNCE, BC_BOUNCE, 0, 0, BC_FREE, BC_ANTIBOUNCE)),
    "n1=1 generic": ((1, 40, 2), (BC_FREE, BC_ANTIBOUNCE, 0, 0, BC_BOUNCE, BC_FREE)),
    "n2=1 walls": ((5, 1, 6), (BC_BOUNCE, BC_FREE, BC_ANTIBOUNCE, BC_BOUNCE, 0, 0)),
    "n2=3 periodic": ((4, 3, 3), (0, 0, 0, 0, 0, 0)),
}


@pytest.mark.parametrize("name", list(DEGENERATE))
def test_degenerate_extents_match_oracle(name):
    """Lattices one or two nodes thick along an axis (both faces of the axis act on every
    node; the tile kernel's first tile starts at q1 = -1 where n1 - 1 is a multiple of its
    rows): 40 steps from seeded random populations, FP64, device against the oracle."""
    from paper_1705_01801_gb300 import lbw
    n, bc = DEGENERATE[name]
    spec = GridSpec(kind=KIND_CARTESIAN, n=n, h=(1, 1, 1), x0=(0, 0, 0), c=0.4, bc=bc,
                    damping=0.8, prec=PREC_F64)
    f = np.random.default_rng(sum(n)).standard_normal((7, n[2], n[0], n[1]))
    q = [[n[0] - 1, n[1] - 1, n[2] - 1], [0, 0, 0]]
    g = lbw.Grid(spec)
    try:
        g.set_f(f)
        g.set_probes(q, 40)
        g.step(40)
        fg, sg = g.get_f(), g.read_probes()
    finally:
        g.close()
    o = oracle.OracleGrid(spec)
    o.set_f(f)
    o.set_probes(q, 40)
    o.step(40)
    fo, so = o.get_f(), o.read_probes()
    np.testing.assert_allclose(fg, fo, rtol=0, atol=1e-11 * np.abs(fo).max())
    np.testing.assert_allclose(sg, so, rtol=0, atol=1e-11 * np.abs(so).max())
