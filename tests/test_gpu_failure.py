"""Failure detection and checkpoint / resume on the device, without faulting the GPU.

* An unstable state is made on the host: a NaN written into one node's populations through
  lbw_set_populations.  Every call that hands results back (lbw_probe_read, lbw_spectrum,
  lbw_get_field) must then return LBW_EUNSTABLE, and lbw_init must bring the lattice back to
  a state whose run matches the FP64 oracle.
* Checkpoint / resume: a run split at step s by lbw_get_populations -> a new lattice ->
  lbw_set_populations must equal the straight run bit for bit (populations and the probe
  series of the second part), for every storage format: the checkpoint holds the stored
  values exactly (16-bit formats store f / w with w a power of two).
"""
import math

import numpy as np
import pytest

import oracle
from lbw_workloads import (BC_ANTIBOUNCE, BC_BOUNCE, KIND_CYLINDRICAL, KIND_TOROIDAL, PREC_BF16S,
                           PREC_F16S, PREC_F32, PREC_F64, GridSpec, probes, pulses)

pytestmark = pytest.mark.gpu


def _cyl(prec, n=(13, 64, 10)):
    return GridSpec(kind=KIND_CYLINDRICAL, n=n, h=(1, 2 * math.pi / n[1], 1), x0=(8, 0, 0),
                    c=0.4, prec=prec,
                    bc=(BC_BOUNCE, BC_ANTIBOUNCE, 0, 0, BC_ANTIBOUNCE, BC_ANTIBOUNCE))


def test_nan_state_is_reported_as_unstable_and_init_recovers():
    from paper_1705_01801_gb300 import lbw
    spec = _cyl(PREC_F32)
    pl = pulses(spec, 3, 1, sigma=2.5, margin=3)
    pr = np.array([[5, 17, 4], [9, 40, 6]], dtype=np.int32)
    g = lbw.Grid(spec)
    g.init(pl)
    g.step(3)
    f = g.get_f()
    f[:, 4, 5, 17] = np.nan  # populations of node (q1, q2, q3) = (5, 17, 4)
    g.set_f(f)
    g.set_probes(pr, 50)
    g.step(20)
    for call in (g.read_probes, lambda: g.spectrum(-1, 3), g.get_P):
        with pytest.raises(lbw.LbwError) as e:
            call()
        assert e.value.status == lbw.LBW_EUNSTABLE, str(e.value)
    # lbw_init rebuilds a clean state; the run then matches the oracle
    g.init(pl)
    g.set_probes(pr, 60)
    g.step(60)
    o = oracle.OracleGrid(spec)
    o.init(pl)
    o.set_probes(pr, 60)
    o.step(60)
    Pg, Po = g.get_P(), o.get_P()
    assert np.linalg.norm(Pg - Po) / np.linalg.norm(Po) < 2e-5
    np.testing.assert_allclose(g.read_probes(), o.read_probes(), rtol=0, atol=2e-5 * np.abs(Po).max())


@pytest.mark.parametrize("prec", [PREC_F64, PREC_F32, PREC_F16S, PREC_BF16S],
                         ids=["f64", "f32", "f16s", "bf16s"])
def test_split_run_equals_straight_run(prec):
    from paper_1705_01801_gb300 import lbw
    spec = _cyl(prec, n=(13, 128, 10))
    pl = pulses(spec, 5, 2, sigma=2.5, margin=3)
    pr = probes(spec, 5, 3)
    total, split = 90, 37
    a = lbw.Grid(spec)
    a.init(pl)
    a.step(split)
    a.set_probes(pr, total)
    a.step(total - split)
    straight_f, straight_series = a.get_f(), a.read_probes()

    b = lbw.Grid(spec)
    b.init(pl)
    b.step(split)
    ckpt = b.get_f()
    b.close()
    c = lbw.Grid(spec)  # a fresh lattice resumes from the checkpoint
    c.set_f(ckpt)
    c.set_probes(pr, total)
    c.step(total - split)
    assert np.array_equal(c.get_f(), straight_f)
    assert np.array_equal(c.read_probes(), straight_series)


def test_torus_checkpoint_round_trip_is_exact():
    """A checkpoint written and read back without stepping is the identity on the stored
    values, on a lattice large enough for the tile kernel (torus, 16-bit storage)."""
    from paper_1705_01801_gb300 import lbw
    n = (19, 128, 16)
    spec = GridSpec(kind=KIND_TOROIDAL, n=n, h=(1, 2 * math.pi / n[1], 2 * math.pi / n[2]),
                    x0=(3, 0, 0), c=0.4, geom=(70.0, 0, 0, 0), prec=PREC_F16S,
                    bc=(BC_BOUNCE, BC_BOUNCE, 0, 0, 0, 0))
    g = lbw.Grid(spec)
    g.init(pulses(spec, 9, 1, sigma=2.0, margin=3))
    g.step(11)
    f = g.get_f()
    g.set_f(f)
    assert np.array_equal(g.get_f(), f)


def test_injected_wait_timeout_is_reported_and_init_recovers():
    """A step whose bounded device wait runs out (made to happen on purpose: the consumer warps
    wait on a barrier that nothing completes, for a few hundred tries) raises the timeout flag;
    the calls that synchronise then return LBW_ETIMEOUT, the GPU stays usable, and lbw_init
    brings back a state whose run matches the FP64 oracle."""
    from paper_1705_01801_gb300 import lbw
    spec = _cyl(PREC_F32, n=(13, 128, 10))  # q2 extent a multiple of the tile width: tile kernel
    pl = pulses(spec, 4, 1, sigma=2.5, margin=3)
    pr = probes(spec, 4, 2)
    g = lbw.Grid(spec)
    g.init(pl)
    g.set_probes(pr, 100)
    g.step(4)
    g.read_probes()  # no flag before the injection
    lbw.lbw_inject_wait_timeout(g.handle)
    g.step(70)  # single launches and one 64-step graph chain
    for call in (g.read_probes, lambda: g.spectrum(-1, 2), g.get_P, g.get_f):
        with pytest.raises(lbw.LbwError) as e:
            call()
        assert e.value.status == lbw.LBW_ETIMEOUT, str(e.value)
    g.init(pl)
    g.set_probes(pr, 80)
    g.step(80)
    o = oracle.OracleGrid(spec)
    o.init(pl)
    o.set_probes(pr, 80)
    o.step(80)
    Pg, Po = g.get_P(), o.get_P()
    assert np.linalg.norm(Pg - Po) / np.linalg.norm(Po) < 2e-5


def test_injected_timeout_needs_the_tile_kernel():
    from paper_1705_01801_gb300 import lbw
    spec = _cyl(PREC_F32, n=(13, 40, 10))  # 40 columns: register-pipelined kernel, no waits
    g = lbw.Grid(spec)
    with pytest.raises(lbw.LbwError) as e:
        lbw.lbw_inject_wait_timeout(g.handle)
    assert e.value.status == lbw.LBW_ESTATE
    g.init(pulses(spec, 4, 1, sigma=2.5, margin=3))
    with pytest.raises(lbw.LbwError) as e:
        lbw.lbw_inject_wait_timeout(g.handle)
    assert e.value.status == lbw.LBW_EINVAL
