"""Closed-form normal modes used as pins (scipy Bessel functions; test infrastructure).

Annulus a < r < R with a rigid inner wall (dP/dr = 0 at r = a) and a Dirichlet outer wall
(P = 0 at r = R): P = R_m(k r) cos(m theta) cos(omega t), omega = c k, where
R_m(k r) = J_m(k r) Y_m'(k a) - Y_m(k r) J_m'(k a) and k solves R_m(k R) = 0
(separation of variables of the wave equation in cylindrical coordinates, as in the
paper's appendix "Radial modes of the pipe").
"""
import numpy as np
from scipy.optimize import brentq
from scipy.special import jv, jvp, yv, yvp


def roots(fun, lo, hi, n_grid=20000):
    xs = np.linspace(lo, hi, n_grid)
    v = fun(xs)
    out = []
    for i in range(n_grid - 1):
        if np.isfinite(v[i]) and np.isfinite(v[i + 1]) and v[i] * v[i + 1] < 0:
            out.append(brentq(fun, xs[i], xs[i + 1], xtol=1e-14))
    return out


def annulus_radial(m, k, a, r):
    return jv(m, k * r) * yvp(m, k * a) - yv(m, k * r) * jvp(m, k * a)


def annulus_wavenumbers(m, a, R, count=3):
    f = lambda k: annulus_radial(m, k, a, R)
    ks = roots(f, 1e-4 / R, 40.0 / R)
    return ks[:count]


def pipe_zeros(m, count=3):
    f = lambda x: (m + 1) * jv(m, x) - x * jv(m + 1, x)
    return roots(f, 1e-3, 30.0)[:count]


def bessel_horn_wavenumbers(lam, z_a, z_b, count=4):
    """Axial wavenumbers of Webster's horn equation (the plane-wave limit of the wave equation
    in a duct) for the paper's Bessel horn, cross-section area S ~ s^2 = Zc^(-2 lam) with
    Zc = Zmax - z, between rigid ends at Zc = z_a and Zc = z_b (dP/dz = 0).  In Zc the
    equation P'' - (2 lam / Zc) P' + k^2 P = 0 has the solutions Zc^nu C_nu(k Zc) with
    nu = lam + 1/2 (C a cylinder function), whose derivative is k Zc^nu C_(nu-1)(k Zc);
    rigid ends therefore need J_(nu-1)(k z_a) Y_(nu-1)(k z_b) - Y_(nu-1)(k z_a) J_(nu-1)(k z_b)
    = 0.  lam = 0 gives the pipe, k = n pi / (z_b - z_a)."""
    o = lam - 0.5
    f = lambda k: jv(o, k * z_a) * yv(o, k * z_b) - yv(o, k * z_a) * jv(o, k * z_b)
    span = z_b - z_a
    return roots(f, 1e-3 / span, (count + 1.5) * np.pi / span)[:count]


def webster_wavenumbers(s, ds, length, count=4):
    """Axial wavenumbers of Webster's horn equation P'' + 2 (s'/s) P' + k^2 P = 0 (cross-section
    area ~ s(z)^2) between rigid ends at z = 0 and z = length (P' = 0), for any flare s(z) with
    derivative ds(z): shooting from z = 0 with P = 1, P' = 0 and bracketing the roots of P'(length)
    in k (scipy's adaptive Runge-Kutta at 1e-11 relative tolerance)."""
    from scipy.integrate import solve_ivp

    def end_slope(k):
        rhs = lambda z, y: [y[1], -2.0 * ds(z) / s(z) * y[1] - k * k * y[0]]
        return solve_ivp(rhs, (0.0, length), [1.0, 0.0], rtol=1e-11, atol=1e-12).y[1, -1]

    ks = np.linspace(1e-3 / length, (count + 1.5) * np.pi / length, 60 * (count + 2))
    v = [end_slope(k) for k in ks]
    out = []
    for i in range(len(ks) - 1):
        if v[i] * v[i + 1] < 0:
            out.append(brentq(end_slope, ks[i], ks[i + 1], xtol=1e-13))
    return out[:count]
