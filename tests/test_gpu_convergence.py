"""Second-order convergence of the device sweep in curvilinear coordinates (Sec. IV.A, the
convergence study of Fig. Convergence): the lowest axisymmetric mode of a closed annular
cylinder, resolved with 1, 2, 4 and 8 cells per unit length, against its closed form."""
import math

import numpy as np
import pytest

from lbw_workloads import (BC_ANTIBOUNCE, BC_BOUNCE, BC_PERIODIC, KIND_CYLINDRICAL, PREC_F32,
                           PREC_F64, GridSpec)
from modes import annulus_radial, annulus_wavenumbers

pytestmark = pytest.mark.gpu

A_IN, R_OUT, LENGTH, C0 = 3.0, 15.0, 16.0, 0.4  # physical inner / outer radius, length, speed


def _cylinder(s, prec):
    """s cells per unit length in r and z; the lattice speed c / h stays C0, so the time step
    shrinks with the cells (c = C0 / s per step)."""
    n_r, n_z, n_t = int((R_OUT - A_IN) * s), int(LENGTH * s), 8
    return GridSpec(kind=KIND_CYLINDRICAL, n=(n_r, n_t, n_z), h=(1 / s, 2 * math.pi / n_t, 1 / s),
                    x0=(A_IN, 0, 0), c=C0 / s, prec=prec,
                    bc=(BC_BOUNCE, BC_ANTIBOUNCE, BC_PERIODIC, BC_PERIODIC, BC_ANTIBOUNCE,
                        BC_ANTIBOUNCE))


def _mode_error(s, prec):
    """Relative error of the measured frequency of the (m = 0, radial 0, axial 1) mode, whose
    closed form is omega = c sqrt(k^2 + (pi / L)^2) with k the annulus root (rigid inner wall,
    Dirichlet outer wall and caps)."""
    from paper_1705_01801_gb300 import lbw
    spec = _cylinder(s, prec)
    n_r, n_t, n_z = spec.n
    k = annulus_wavenumbers(0, A_IN, R_OUT, 1)[0]
    r = A_IN + (np.arange(n_r) + 0.5) / s
    z = (np.arange(n_z) + 0.5) / s
    P0 = np.sin(math.pi * z / LENGTH)[:, None, None] * annulus_radial(0, k, A_IN, r)[None, :, None] \
        * np.ones(n_t)
    sqrt_g = r * spec.h[0] * spec.h[1] * spec.h[2]  # r h_r h_theta h_z
    w = np.array([1 - 3 * spec.cs2] + [spec.cs2 / 2] * 6)
    steps = 1500 * s
    g = lbw.Grid(spec)
    try:
        g.set_f(w[:, None, None, None] * (sqrt_g[None, :, None] * P0)[None])
        g.set_probes([[n_r // 3, 0, n_z // 3]], steps)
        g.step(steps)
        f, a = g.spectrum(0, 3)
    finally:
        g.close()
    omega = f[np.argmax(a)]
    return omega / (spec.c * math.hypot(k, math.pi / LENGTH)) - 1


@pytest.mark.parametrize("prec", [PREC_F64, PREC_F32], ids=["f64", "f32"])
def test_mode_error_falls_as_h_squared(prec):
    """The error shrinks four-fold per halving of the cell (fitted order 2 +- 0.15; the paper
    fits 2.1 +- 0.08 on its pipe) and is below 2.5e-5 at 8 cells per unit."""
    scales = [1, 2, 4, 8]
    err = np.array([_mode_error(s, prec) for s in scales])
    order = -np.polyfit(np.log(scales), np.log(np.abs(err)), 1)[0]
    print(f"errors {err}, fitted order {order:.3f}")
    assert abs(order - 2) < 0.15
    assert abs(err[-1]) < 2.5e-5
