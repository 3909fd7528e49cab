"""Harmonic sources (the paper's ring / plate sources) on the device against the FP64 oracle,
single lattices and ensembles, and the resonance sweep built on them."""
import math

import numpy as np
import pytest

import oracle
from lbw_workloads import (BC_BOUNCE, BC_FREE, BC_PERIODIC, KIND_CYLINDRICAL, PREC_F16S, PREC_F32, PREC_F64, GridSpec,
                           ensemble, pulses, probes)
from test_gpu_parity import SPECS

pytestmark = pytest.mark.gpu


def _ring(spec, q1, q3):
    return [[q1, j, q3] for j in range(spec.n[1])]


def _plate(spec, q3):
    return [[i, j, q3] for i in range(spec.n[0]) for j in range(spec.n[1])]


@pytest.mark.parametrize("prec,tol", [(PREC_F64, 1e-11), (PREC_F32, 2e-5)], ids=["f64", "f32"])
@pytest.mark.parametrize("name", ["cylinder", "cylinder_unstaged", "cylinder_wide"])
@pytest.mark.parametrize("kind", [0, 1], ids=["P", "Jz"])
def test_sources_match_oracle(name, kind, prec, tol):
    from paper_1705_01801_gb300 import lbw
    spec = SPECS[name].with_(prec=prec)
    src = _ring(spec, 0, 2) if kind == 0 else _plate(spec, 0)
    pl = pulses(spec, 5, 1, sigma=2.5, margin=2)
    pr = probes(spec, 5, 4, margin=0)
    g = lbw.Grid(spec)
    g.init(pl)
    g.set_sources(src, kind=kind, amp=0.8, omega=0.21)
    g.set_probes(pr, 130)
    o = oracle.OracleGrid(spec)
    o.init(pl)
    o.set_sources(src, kind=kind, amp=0.8, omega=0.21)
    o.set_probes(pr, 130)
    g.step(130)  # 64-step graph chains and single launches both carry the sources
    o.step(130)
    fo = o.get_f()
    np.testing.assert_allclose(g.get_f(), fo, rtol=0, atol=tol * np.abs(fo).max())
    so = o.read_probes()
    np.testing.assert_allclose(g.read_probes(), so, rtol=0, atol=tol * 10 * np.abs(so).max())


def test_removing_sources_restores_the_free_run():
    from paper_1705_01801_gb300 import lbw
    spec = SPECS["cylinder"].with_(prec=PREC_F64)
    pl = pulses(spec, 6, 1, sigma=2.5, margin=2)
    a, b = lbw.Grid(spec), lbw.Grid(spec)
    a.init(pl)
    b.init(pl)
    b.set_sources(_ring(spec, 0, 2), omega=0.3)
    b.set_sources([])
    a.step(70)
    b.step(70)
    np.testing.assert_array_equal(a.get_f(), b.get_f())


@pytest.mark.parametrize("prec,tol", [(PREC_F64, 1e-11), (PREC_F32, 2e-5)], ids=["f64", "f32"])
def test_ensemble_sources_per_member_frequency(prec, tol):
    """One frequency per member; a source next to the periodic wrap exercises the ghost
    copies of the padded rows."""
    from paper_1705_01801_gb300 import lbw
    specs, _ = ensemble(4, seed=12, r_range=(9, 15), theta_range=(33, 70), z_range=(18, 30), prec=prec)
    omegas = [0.05, 0.11, 0.17, 0.23]
    src = [[[2, 0, 1], [2, s.n[1] - 1, 1], [3, s.n[1] // 2, 1]] for s in specs]
    b = lbw.Batch(specs)
    b.init([np.zeros((0, 5))] * len(specs))
    b.set_sources(np.array(src), omegas, kind=0, amp=1.0)
    b.step(90)
    for m, s in enumerate(specs):
        o = oracle.OracleGrid(s)
        o.init(np.zeros((0, 5)))
        o.set_sources(src[m], kind=0, amp=1.0, omega=omegas[m])
        o.step(90)
        fo = o.get_f()
        np.testing.assert_allclose(b.get_f(m), fo, rtol=0, atol=tol * np.abs(fo).max())


def test_resonance_sweep_finds_the_driven_pipe_mode():
    """The paper's protocol (Sec. IV.A: a pipe driven by a ring in front of its end, damping D
    at the walls, the steady-state response at a probe against the source frequency): in a
    closed pipe the axisymmetric axial modes sit at omega_n = n pi c / L (closed form; a
    free-decay run of the same lattice finds them with the spectrum estimator), and the
    sweep's response peak must fall on the measured mode within 1%."""
    from paper_1705_01801_gb300 import lbw, sweep
    from lbw_workloads import embedding, node_coords
    n_r, n_t, n_z = 6, 8, 100
    c = 0.4
    spec = GridSpec(kind=KIND_CYLINDRICAL, n=(n_r, n_t, n_z), h=(1, 2 * math.pi / n_t, 1),
                    x0=(2, 0, 0), c=c, damping=0.98,
                    bc=(BC_BOUNCE, BC_BOUNCE, BC_PERIODIC, BC_PERIODIC, BC_BOUNCE, BC_BOUNCE),
                    prec=PREC_F32)
    ring = _ring(spec, 0, 0)
    probe = [2, 0, n_z // 10]
    g = lbw.Grid(spec)
    pl = []
    for j in range(n_t):
        X = embedding(spec, *node_coords(spec, 1, j, 1))
        pl.append([X[0], X[1], X[2], 1.5, 1.0])
    g.init(pl)
    g.set_probes([probe], 8000)
    g.step(8000)
    f, _ = g.spectrum(0, 8)
    theory = 2 * math.pi * c / n_z  # n = 2
    mode = f[np.argmin(np.abs(f - theory))]
    assert abs(mode - theory) < 2e-3 * theory
    omegas = np.linspace(mode * 0.85, mode * 1.15, 41)
    resp = sweep.resonance_curve(spec, ring, probe, omegas, steps=8000, tail=2000)
    peak = sweep.peak_frequency(omegas, resp)
    print(f"closed form {theory:.6f}, free-decay mode {mode:.6f}, sweep peak {peak:.6f} rad/step")
    assert abs(peak - mode) < 0.01 * mode
    assert resp.max() > 2 * resp.min()


# ---------------------------------------------------------------- the paper's pipe ---------

def _paper_pipe(damping, prec=PREC_F32):
    """The open-closed pipe of Sec. IV.A: 20 x 5 x 100 cells over r in [1, 25] (h_r = 1.2),
    z in [0, 100], c = 0.1; bounce-back with damping D at r = 25 and at the closed end z = 0,
    a free face at the open end z = 100.  The paper's free inner face at r = 1 grows without
    bound under the copy rule (on a curved inner wall it is a Robin condition with the
    destabilising sign), so the inner wall is rigid here, with the same D."""
    n = (20, 5, 100)
    return GridSpec(kind=KIND_CYLINDRICAL, n=n, h=(1.2, 2 * math.pi / n[1], 1.0), x0=(1.0, 0, 0),
                    c=0.1, damping=damping, prec=prec,
                    bc=(BC_BOUNCE, BC_BOUNCE, BC_PERIODIC, BC_PERIODIC, BC_BOUNCE, BC_FREE))


PAPER_PROBE = [1, 0, 10]  # r = 2.8, z = 10.5: the paper's probe at r = 3, z = z_max / 10


@pytest.mark.parametrize("kind", [0, 1], ids=["ring", "plate"])
def test_paper_pipe_sources_match_oracle(kind):
    """The paper's pipe with D = 0.65, driven by the ring (P at r_min, z = 0) or the plate
    (J'_z over the cross-section at z = 0): device and FP64 oracle agree."""
    from paper_1705_01801_gb300 import lbw
    spec = _paper_pipe(0.65, prec=PREC_F64)
    src = _ring(spec, 0, 0) if kind == 0 else _plate(spec, 0)
    g = lbw.Grid(spec)
    g.init(np.zeros((0, 5)))
    g.set_sources(src, kind=kind, amp=1.0, omega=0.0123)
    g.set_probes([PAPER_PROBE], 700)
    g.step(700)
    o = oracle.OracleGrid(spec)
    o.init(np.zeros((0, 5)))
    o.set_sources(src, kind=kind, amp=1.0, omega=0.0123)
    o.set_probes([PAPER_PROBE], 700)
    o.step(700)
    fo = o.get_f()
    np.testing.assert_allclose(g.get_f(), fo, rtol=0, atol=1e-11 * np.abs(fo).max())
    so = o.read_probes()
    np.testing.assert_allclose(g.read_probes(), so, rtol=0, atol=1e-10 * np.abs(so).max())


def test_paper_pipe_is_an_open_closed_pipe():
    """Free decay of the paper's pipe (lossless walls, a layer of pulses across the section near
    the closed end, the paper's probe): the lowest modes are the open-closed pipe's plane-wave
    family, odd multiples (1 : 3 : 5) of a quarter wave (Sec. IV.A), not the closed pipe's
    1 : 2 : 3, with the open end at L_e = L - cs^2 / c (the free face's end correction; the
    higher modes sit up to 2 % above, the end correction being frequency dependent); and the
    ring-source sweep of the paper's protocol (8400 steps, response = largest |P| at the probe
    over the last 2000) peaks on them within the sweep's resolution 2 pi / 8400."""
    from paper_1705_01801_gb300 import lbw, sweep
    from lbw_workloads import embedding, node_coords
    spec = _paper_pipe(1.0, prec=PREC_F64)
    g = lbw.Grid(spec)
    pl = []
    for i in range(1, spec.n[0], 3):  # nearly uniform across the section: the plane-wave modes
        for j in range(spec.n[1]):
            X = embedding(spec, *node_coords(spec, i, j, 3))
            pl.append([X[0], X[1], X[2], 2.5, 1.0])
    g.init(pl)
    T = 16384
    g.set_probes([PAPER_PROBE], T)
    g.step(T)
    f, _ = g.spectrum(0, 6, lowest=True, rel_power=1e-3)
    f = np.sort(np.asarray(f))
    L_e = spec.n[2] - spec.cs2 / spec.c
    quarter = [(2 * n + 1) * math.pi * spec.c / (2 * L_e) for n in range(3)]
    print("free-decay modes", np.round(f[:5], 6), "quarter-wave family", np.round(quarter, 6))
    np.testing.assert_allclose(f[:3], quarter, rtol=3e-2)
    np.testing.assert_allclose(f[1:3] / f[0], [3, 5], rtol=5e-2)
    omegas = np.linspace(0.0008, 0.0095, 175)
    resp = sweep.resonance_curve(spec.with_(prec=PREC_F32), _ring(spec, 0, 0), PAPER_PROBE, omegas,
                                 steps=8400, tail=2000, kind=0)
    res = 2 * math.pi / 8400
    for m in f[:3]:  # the response has a maximum inside [m - res, m + res], not at its edges
        win = np.nonzero(np.abs(omegas - m) <= res)[0]
        k = win[np.argmax(resp[win])]
        print(f"mode {m:.6f}: sweep peak {omegas[k]:.6f}")
        assert win[0] < k < win[-1], (m, omegas[win[0]], omegas[k], omegas[win[-1]])


@pytest.mark.parametrize("prec,tol", [(PREC_F64, 1e-11), (PREC_F32, 2e-5)], ids=["f64", "f32"])
def test_paper_radial_wave_matches_oracle(prec, tol):
    """The radial wave from the axis (Sec. IV.A) on the paper's lattice: 100 x 3 x 10 cells
    of 4.99 along r (from r = 3, so that the inner ghost node has r > 0), c = 0.6, the ring source sin(0.075 t) at r_min, cs2 = (c / h_r)^2 (the
    lattice speed along r; the default cs2 makes the wave 35 % too long there), 365 steps.
    Device and FP64 oracle agree, and the device's profile is the outgoing J0 / Y0 wave with
    k = omega / c (fit within 6 %, wavenumber within 2 %)."""
    from paper_1705_01801_gb300 import lbw
    from test_oracle_pins import PAPER_RADIAL, _bessel_fit
    h_r, r_min, T, om = PAPER_RADIAL["h_r"], PAPER_RADIAL["r_min"], 365, 0.075
    n = (PAPER_RADIAL["n1"], 3, 10)
    spec = GridSpec(kind=KIND_CYLINDRICAL, n=n, h=(h_r, 2 * math.pi / 3, h_r), x0=(r_min, 0, 0), c=0.6,
                    cs2=(0.6 / h_r) ** 2, prec=prec,
                    bc=(BC_FREE, BC_FREE, BC_PERIODIC, BC_PERIODIC, BC_PERIODIC, BC_PERIODIC))
    src = [[0, j, k] for j in range(n[1]) for k in range(n[2])]
    g = lbw.Grid(spec)
    try:
        g.init(np.zeros((0, 5)))
        g.set_sources(src, kind=0, amp=1.0, omega=om)
        g.step(T)
        P = g.get_P()
    finally:
        g.close()
    o = oracle.OracleGrid(spec.with_(prec=PREC_F64))
    o.init(np.zeros((0, 5)))
    o.set_sources(src, kind=0, amp=1.0, omega=om)
    o.step(T)
    Po = o.get_P()
    np.testing.assert_allclose(P, Po, rtol=0, atol=tol * np.abs(Po).max())
    r = r_min + (np.arange(n[0]) + 0.5) * h_r
    e0, _, _, kb = _bessel_fit(r, P[0, :, 0], om / 0.6, 10, 0.5 * 0.6 * T)
    print(f"\ndevice prec {prec}: J0/Y0 residual {e0:.4f}, best k / k {kb:.3f}")
    assert e0 < 0.06 and abs(kb - 1) < 0.02


def _pipe_free_decay(prec, steps):
    """The six lowest modes of the lossless paper pipe's free decay (a layer of pulses near the
    closed end, the paper's probe), and the probe series."""
    from paper_1705_01801_gb300 import lbw
    from lbw_workloads import embedding, node_coords
    spec = _paper_pipe(1.0, prec=prec)
    pl = []
    for i in range(1, spec.n[0], 3):
        for j in range(spec.n[1]):
            X = embedding(spec, *node_coords(spec, i, j, 3))
            pl.append([X[0], X[1], X[2], 2.5, 1.0])
    g = lbw.Grid(spec)
    try:
        g.init(pl)
        g.set_probes([PAPER_PROBE], steps)
        g.step(steps)
        f, _ = g.spectrum(0, 6, lowest=True, rel_power=1e-3)
        return np.sort(np.asarray(f)), g.read_probes()[0]
    finally:
        g.close()


@pytest.mark.parametrize("prec,tol", [(PREC_F32, 1e-5), (PREC_F16S, 5e-3)], ids=["f32", "f16"])
def test_paper_pipe_modes_in_reduced_storage(prec, tol):
    """At the paper's small wave speed (c = 0.1, so the forcing and the departures of the
    populations from w P are small against the stored values) and over 65 536 steps, the
    reduced storage forms give the FP64 run's six lowest modes of the open-closed pipe: FP32
    within 1e-5, the 16-bit form within the 0.5 % mode bound; the FP32 probe series stays
    within 1e-4 of the FP64 one (rounding of the coefficients and populations, no drift)."""
    steps = 65536
    f64, x64 = _pipe_free_decay(PREC_F64, steps)
    f, x = _pipe_free_decay(prec, steps)
    print(f"\nFP64 modes {np.round(f64, 6)}; prec {prec}: {np.round(f, 6)}, "
          f"series max |diff| {np.abs(x - x64).max():.2e}")
    assert len(f) == len(f64) == 6
    np.testing.assert_allclose(f, f64, rtol=tol)
    if prec == PREC_F32:
        assert np.abs(x - x64).max() <= 1e-4 * np.abs(x64).max()


def _paper_torus(prec=PREC_F64):
    """The torus of Sec. IV.C: R = 640, r < 409.6, 20 x 200 x 30 cells in (r, theta major,
    phi minor), bounce-back with D = 0.65 at r_max, periodic theta and phi.  Two changes: the
    inner face is rigid (the paper's free face grows without bound on a curved inner wall) and
    sits at r = 12 instead of 5.12, because with 20 cells of 20 units the ghost node of a face
    at 5.12 would lie at negative r, where the metric is undefined.  The paper does not state
    c: c = 2 (physical units per step, 0.1 cells of h_r per step)."""
    from lbw_workloads import BC_BOUNCE as BB, KIND_TOROIDAL
    n = (20, 200, 30)
    return GridSpec(kind=KIND_TOROIDAL, n=n, h=((409.6 - 12.0) / n[0], 2 * math.pi / n[1], 2 * math.pi / n[2]),
                    x0=(12.0, 0, 0), c=2.0, damping=0.65, geom=(640.0, 0, 0, 0), prec=prec,
                    bc=(BB, BB, BC_PERIODIC, BC_PERIODIC, BC_PERIODIC, BC_PERIODIC))


@pytest.mark.parametrize("source", ["major-ring", "small-ring", "point"])
def test_paper_torus_sources_match_oracle(source):
    """The three sources of Sec. IV.C on the paper's torus, device against the FP64 oracle:
    the ring along the major circle (r = r_min, all theta and phi), the small ring (r = r_min,
    theta = 0, all phi) and the off-axis point (mid radius, theta = 0, phi = pi / 2)."""
    from paper_1705_01801_gb300 import lbw
    spec = _paper_torus()
    n1, n2, n3 = spec.n
    src = {"major-ring": [[0, j, k] for j in range(n2) for k in range(n3)],
           "small-ring": [[0, 0, k] for k in range(n3)],
           "point": [[n1 // 2, 0, n3 // 4]]}[source]
    probe = [[n1 - 1, n2 // 2, 0], [n1 // 2, n2 // 4, n3 // 2]]  # (r_max, pi, 0) and an inner node
    g = lbw.Grid(spec)
    o = oracle.OracleGrid(spec)
    for grid in (g, o):
        grid.init(np.zeros((0, 5)))
        grid.set_sources(src, kind=0, amp=1.0, omega=0.07)
        grid.set_probes(probe, 300)
        grid.step(300)
    fo = o.get_f()
    np.testing.assert_allclose(g.get_f(), fo, rtol=0, atol=1e-11 * np.abs(fo).max())
    so = o.read_probes()
    np.testing.assert_allclose(g.read_probes(), so, rtol=0, atol=1e-10 * np.abs(so).max())


def test_probe_peak_reduction_matches_the_series():
    """The sweep's response, reduced on the device (largest |P| of each probe over the last
    `tail` samples), equals the same reduction of the read-back series."""
    from paper_1705_01801_gb300 import lbw
    specs, _ = ensemble(3, seed=14, r_range=(9, 12), theta_range=(33, 40), z_range=(18, 24), prec=PREC_F64)
    b = lbw.Batch(specs)
    b.init([np.zeros((0, 5))] * 3)
    b.set_sources(np.array([[[2, 0, 1]]] * 3), [0.05, 0.1, 0.2], kind=0, amp=1.0)
    q = np.array([[[3, 5, 7], [1, 2, 10]]] * 3, dtype=np.int32)
    b.set_probes(q, 300)
    b.step(300)
    series = b.read_probes()
    for tail in (1, 77, 300):
        np.testing.assert_array_equal(b.probe_peak(tail), np.abs(series[:, :, -tail:]).max(axis=2))
    with pytest.raises(lbw.LbwError) as e:
        b.probe_peak(301)
    assert e.value.status == lbw.LBW_EINVAL
