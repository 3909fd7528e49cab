"""The paper's Bessel horn (Sec. IV.B) on the device: the pipe-versus-horn comparison of the
axial normal modes, against the FP64 oracle on small horns and against Webster's horn
equation at the paper's horn length (Zmax = 750) and flare exponents lam = 0.1, 0.2, and the
driven resonance sweep of a horn."""
import math

import numpy as np
import pytest

import oracle
from lbw_workloads import PREC_F32, PREC_F64, bessel_horn, ensemble_excitation
from modes import bessel_horn_wavenumbers

pytestmark = pytest.mark.gpu

SMALL = (4, 8, 64)  # r x theta x z cells of the small horns


def _axisymmetric_start(spec):
    """Post-collision populations f^eq(rho, 0) of a radially uniform Gaussian P(z) near the
    q3 = 0 end, rho = sqrt(g) P with sqrt(g) from the oracle's geometry (input data only)."""
    n1, n2, n3 = spec.n
    o = oracle.OracleGrid(spec)
    sg = np.array([[o.geometry(q1, 0, q3)[0] for q1 in range(n1)] for q3 in range(n3)])
    o.close()
    z = np.arange(n3) + 0.5
    rho = sg[:, :, None] * np.exp(-0.5 * ((z - 0.15 * n3) / 3.0) ** 2)[:, None, None] * np.ones(n2)
    w = np.array([1 - 3 * spec.cs2] + [spec.cs2 / 2] * 6)
    return w[:, None, None, None] * rho[None]


@pytest.mark.parametrize("lam", [0.0, 0.2, 0.4])
@pytest.mark.parametrize("prec,tol", [(PREC_F64, 1e-9), (PREC_F32, 2e-5)], ids=["f64", "f32"])
def test_horn_modes_match_oracle(lam, prec, tol):
    """The same start on both sides, 8000 steps: the probe series agree to FP64 rounding (FP64)
    or 2e-4 of its peak (FP32 storage), and the device's lowest-peak spectrum
    (lbw_spectrum_lowest) finds the oracle estimator's four lowest modes within tol."""
    from paper_1705_01801_gb300 import lbw
    spec = bessel_horn(lam, n=SMALL, prec=prec)
    f0 = _axisymmetric_start(spec)
    probe = [[spec.n[0] // 2, 0, 2]]
    steps = 8000
    o = oracle.OracleGrid(spec.with_(prec=PREC_F64))
    o.set_f(f0)
    o.set_probes(probe, steps)
    o.step(steps)
    xo = o.read_probes()[0]
    g = lbw.Grid(spec)
    g.set_f(f0)
    g.set_probes(probe, steps)
    g.step(steps)
    xg = g.read_probes()[0]
    assert np.abs(xg - xo).max() <= (1e-10 if prec == PREC_F64 else 2e-4) * np.abs(xo).max()
    fo, _ = oracle.spectrum(xo, 4, thresh=1e-3, lowest=True)
    fg, _ = g.spectrum(0, 4, lowest=True, rel_power=1e-3)
    g.close()
    assert len(fg) == len(fo) == 4
    np.testing.assert_allclose(fg, fo, rtol=tol)


def test_paper_horns_follow_webster():
    """Sec. IV.B at the paper's horn length: Zmax = 750, horns of flare lam = 0.1 and 0.2 and
    the straight pipe (lam = 0) over 0 < z < 640, 16 x 32 cells across, advanced together as
    one ensemble.  Webster's horn equation fixes the ratio of each horn mode to the same pipe
    mode (the lattice dispersion cancels in it): the four lowest axial modes must match it
    within 1e-3 (the flare lowers the fundamental by 1.3% and 2.4%)."""
    from paper_1705_01801_gb300 import lbw
    lams = (0.0, 0.1, 0.2)
    L, zmax, steps = 640, 750.0, 80000
    specs = [bessel_horn(lam, n=(16, 32, L), z_gap=zmax - L, prec=PREC_F32) for lam in lams]
    exc = [ensemble_excitation(s) for s in specs]
    b = lbw.Batch(specs)
    try:
        b.init([p for p, _ in exc])
        b.set_probes(np.stack([q for _, q in exc]), steps)
        b.step(steps)
        f, _, cnt = b.spectrum(4, lowest=True, rel_power=1e-3)
    finally:
        b.close()
    assert np.all(cnt == 4)
    n_pi_L = np.arange(1, 5) * math.pi / L
    assert np.all(np.abs(f[0] / (specs[0].c * n_pi_L) - 1) < 2e-3)
    for m, lam in enumerate(lams[1:], start=1):
        webster = np.asarray(bessel_horn_wavenumbers(lam, zmax - L, zmax, 4)) / n_pi_L
        print(f"lam {lam}: lattice horn / pipe {np.round(f[m] / f[0], 5)}, Webster {np.round(webster, 5)}")
        assert np.all(np.abs(f[m] / f[0] - webster) < 1e-3)


def test_resonance_sweep_of_a_horn():
    """The paper's driven protocol on a horn (lam = 0.4): a ring source of axial momentum
    J'_z near the narrow end (a pressure-imposing ring would clamp P there and flatten the
    resonance of so thin a horn), damping 0.98 at the walls, the steady-state response against
    the source frequency.  The lossless horn's free-decay fundamental sits within 0.3% of
    Webster's c k_1, and the damped horn's response peak falls on it within 1%."""
    from paper_1705_01801_gb300 import lbw, sweep
    lam = 0.4
    spec = bessel_horn(lam, n=SMALL, prec=PREC_F32)
    n1, n2, n3 = spec.n
    g = lbw.Grid(spec)
    g.set_f(_axisymmetric_start(spec))
    g.set_probes([[n1 // 2, 0, 2]], 8000)
    g.step(8000)
    mode = g.spectrum(0, 1, lowest=True, rel_power=1e-3)[0][0]
    g.close()
    zmax = spec.geom[0]
    webster = spec.c * bessel_horn_wavenumbers(lam, zmax - n3, zmax, 1)[0]
    assert abs(mode / webster - 1) < 3e-3
    ring = [[n1 // 2, j, 1] for j in range(n2)]
    omegas = np.linspace(mode * 0.85, mode * 1.15, 41)
    resp = sweep.resonance_curve(spec.with_(damping=0.98), ring, [n1 // 2, 0, n3 - 3], omegas,
                                 steps=8000, tail=2000, kind=1)
    peak = sweep.peak_frequency(omegas, resp)
    print(f"Webster {webster:.6f}, horn free-decay fundamental {mode:.6f}, sweep peak {peak:.6f} rad/step")
    assert abs(peak - mode) < 0.01 * mode
    assert resp.max() > 2 * resp.min()
