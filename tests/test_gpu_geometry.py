"""The analytic geometry mode (geometry recomputed per row and plane inside the step kernel
from the closed-form metric of Sec. IV) against the FP64 oracle and against the host-built
table, on the tile-kernel lattices of every kind and face rule.

Tolerances as in test_gpu_parity: FP64 populations within 1e-11 of the field's largest
magnitude (the device's FP64 cos / exp / pow and the host's agree to a few ulp); FP32 within
2e-5 (the FP32 closed forms differ from the FP64-built table by an ulp per coefficient).
"""
import math

import numpy as np
import pytest

import lbw_workloads as W
import oracle
from lbw_workloads import PREC_F32, PREC_F64, pulses, probes
from test_gpu_parity import SPECS

pytestmark = pytest.mark.gpu

# tile-kernel lattices (q2 extent a multiple of 64); the exponential trumpet of the parity
# set widened from 96 to 128 columns
LATTICES = dict(SPECS)
LATTICES["trumpet_exp"] = SPECS["trumpet_exp"].with_(n=(17, 128, 33), h=(1, 2 * math.pi / 128, 1))
TILED = ["polar", "cylinder", "trumpet_exp", "trumpet_bessel", "torus", "cartesian_tiled",
         "cylinder_wide"]


@pytest.mark.parametrize("prec,tol", [(PREC_F64, 1e-11), (PREC_F32, 2e-5)], ids=["f64", "f32"])
@pytest.mark.parametrize("name", TILED)
def test_analytic_geometry_matches_oracle(name, prec, tol):
    from paper_1705_01801_gb300 import lbw
    spec = LATTICES[name].with_(prec=prec, geom_mode=W.GEOM_ANALYTIC)
    steps = 150
    pl = pulses(spec, 31, 2, sigma=2.5, random_phase=True, margin=2)
    pr = probes(spec, 31, 4, margin=0)
    g = lbw.Grid(spec)
    o = oracle.OracleGrid(spec)
    for grid in (g, o):
        grid.init(pl)
        grid.set_probes(pr, steps)
        grid.step(steps)  # 64-step graph chains and single launches
    fo = o.get_f()
    np.testing.assert_allclose(g.get_f(), fo, rtol=0, atol=tol * np.abs(fo).max())
    so = o.read_probes()
    np.testing.assert_allclose(g.read_probes(), so, rtol=0, atol=10 * tol * np.abs(so).max())


@pytest.mark.parametrize("name", ["torus", "trumpet_exp"])
def test_analytic_and_table_agree_in_fp64(name):
    """In FP64 the two geometry sources give the same run to rounding."""
    from paper_1705_01801_gb300 import lbw
    runs = []
    for mode in (W.GEOM_TABLE, W.GEOM_ANALYTIC):
        spec = LATTICES[name].with_(prec=PREC_F64, geom_mode=mode)
        g = lbw.Grid(spec)
        g.init(pulses(spec, 32, 1, sigma=2.5, margin=2))
        g.step(100)
        runs.append(g.get_f())
    np.testing.assert_allclose(runs[1], runs[0], rtol=0, atol=1e-12 * np.abs(runs[0]).max())


def test_analytic_geometry_needs_the_tile_kernel():
    from paper_1705_01801_gb300 import lbw
    spec = SPECS["cylinder_unstaged"].with_(prec=PREC_F32, geom_mode=W.GEOM_ANALYTIC)
    with pytest.raises(lbw.LbwError) as e:
        lbw.Grid(spec)
    assert e.value.status == lbw.LBW_EINVAL and "tile kernel" in str(e.value)
    with pytest.raises(lbw.LbwError) as e:  # the analytic kernels are built for 32 / 64-bit storage
        lbw.Grid(SPECS["cylinder_wide"].with_(prec=W.PREC_F16S, geom_mode=W.GEOM_ANALYTIC))
    assert e.value.status == lbw.LBW_EINVAL and "FP32" in str(e.value)
    specs, _ = W.ensemble(2, seed=3, r_range=(9, 12), theta_range=(33, 40), z_range=(18, 20))
    with pytest.raises(lbw.LbwError) as e:
        lbw.Batch([specs[0], specs[1].with_(geom_mode=W.GEOM_ANALYTIC)])
    assert e.value.status == lbw.LBW_EINVAL and "ensembles" in str(e.value)


# ---------------------------------------------------------------- Cartesian schemes (Sec. II)

@pytest.mark.parametrize("prec,tol", [(PREC_F64, 1e-11), (PREC_F32, 2e-5)], ids=["f64", "f32"])
@pytest.mark.parametrize("eq", [W.EQ_MOMENT_MATCHING, W.EQ_HERMITE], ids=["moment-matching", "hermite"])
@pytest.mark.parametrize("n2", [40, 128], ids=["pipelined", "tiled"])
def test_cartesian_equilibria_match_oracle(eq, prec, tol, n2):
    """Chopard's moment-matching and the Hermite equilibrium of Sec. II on the device (both
    step kernels, every face rule, a point source) against the FP64 oracle."""
    from paper_1705_01801_gb300 import lbw
    spec = W.GridSpec(kind=W.KIND_CARTESIAN, n=(9, n2, 11), h=(1, 1, 1), x0=(0, 0, 0), c=0.35,
                      equilibrium=eq, prec=prec, damping=0.9,
                      bc=(W.BC_FREE, W.BC_BOUNCE, W.BC_ANTIBOUNCE, W.BC_FREE, W.BC_BOUNCE, W.BC_ANTIBOUNCE))
    pl = pulses(spec, 33, 2, sigma=2.0, random_phase=True, margin=2)
    pr = probes(spec, 33, 3, margin=0)
    g = lbw.Grid(spec)
    o = oracle.OracleGrid(spec)
    for grid in (g, o):
        grid.init(pl)
        grid.set_sources([[4, n2 // 2, 5]], kind=0, amp=0.3, omega=0.2)
        grid.set_probes(pr, 140)
        grid.step(140)
    fo = o.get_f()
    np.testing.assert_allclose(g.get_f(), fo, rtol=0, atol=tol * np.abs(fo).max())
    so = o.read_probes()
    np.testing.assert_allclose(g.read_probes(), so, rtol=0, atol=10 * tol * np.abs(so).max())


def test_cartesian_equilibria_are_checked():
    from paper_1705_01801_gb300 import lbw
    base = W.GridSpec(kind=W.KIND_CARTESIAN, n=(9, 64, 11), h=(1, 1, 1), x0=(0, 0, 0), c=0.35,
                      equilibrium=W.EQ_MOMENT_MATCHING, prec=PREC_F32,
                      bc=(W.BC_BOUNCE, W.BC_BOUNCE, 0, 0, 0, 0))
    for bad in (base.with_(prec=W.PREC_F16S), base.with_(geom_mode=W.GEOM_ANALYTIC),
                base.with_(c=0.7)):
        with pytest.raises(lbw.LbwError) as e:
            lbw.Grid(bad)
        assert e.value.status == lbw.LBW_EINVAL
