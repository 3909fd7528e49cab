"""FP64 CPU oracle of the curvilinear wave lattice-Boltzmann method (arXiv:1705.01801).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this package.  It
shares no code with the CUDA path (``paper_1705_01801_gb300``); neither imports the other.

* ``lbw_oracle.c``  -- the time step in plain C loops (FP64), compiled here with gcc.
* ``spectrum.py``   -- the mode-frequency estimator in numpy (FP64).

Parity status of each function is listed in ``PINS`` below; every entry is pinned by a
``-m "not gpu"`` test against something other than the oracle itself.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

from .spectrum import spectrum  # noqa: F401

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lbw_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_SO = os.path.join(_OUT_DIR, "liblbw_oracle.so")
_lock = threading.Lock()
_lib = None

# what pins each oracle function (tests/test_oracle_pins.py)
PINS = {
    "geometry": "embedding Jacobian (metric), divergence identity (Christoffel), sympy-free",
    "step/cartesian": "flat-space wave speed c for c != cs, conservation, order-2 convergence",
    "step/annulus": "Bessel annulus closed form (rigid inner, Dirichlet outer) within 0.2%",
    "step/cylinder": "annulus x sin(n pi z / L) closed form within 0.2%",
    "step/trumpet,torus": "finite-difference solve of the wave equation, order-2 agreement; "
                          "Bessel and exponential horns' axial modes vs Webster's horn equation",
    "step/linear operator": "spectral radius <= 1 and eigen-angles vs spectrum estimator",
    "spectrum": "synthetic sinusoids with known frequencies",
    "face/free": "open-closed pipe: quarter-wave modes (2n+1) pi c / (2 L_e), L - 1 < L_e <= L, "
                 "L_e = L - 1/2 at c = cs; flat and cylindrical q3 faces alike",
    "face/damping D": "impedance reflection (c - beta) / (c + beta), beta = cs2 (1 - D) / (1 + D): "
                      "mode decay per round trip on q1 and q3 walls",
    "source/plate J'_z": "dipole plane waves at speed c, amplitude C / (cs2 + c) at c = cs, "
                         "uniform across a pipe (sqrt g)",
    "source/ring P": "radiated profile fits J0 / Y0 of the radial Bessel equation, also on the "
                     "radial-wave lattice of Sec. IV.A as printed (cs2 matched to c / h_r)",
}


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (OpenMP over nodes) into oracle/_build."""
    with _lock:
        if (not force and os.path.exists(_SO)
                and os.path.getmtime(_SO) >= os.path.getmtime(_SRC)):
            return _SO
        os.makedirs(_OUT_DIR, exist_ok=True)
        tmp = _SO + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-std=c11", _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _SO)
        return _SO


def lib():
    global _lib
    if _lib is None:
        L = ctypes.CDLL(build())
        vp, dp, ip = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int32)
        L.lbwo_create.restype = vp
        L.lbwo_create.argtypes = [ip, dp]
        L.lbwo_destroy.argtypes = [vp]
        L.lbwo_geometry.argtypes = [vp, ctypes.c_double, ctypes.c_double, ctypes.c_double, dp]
        L.lbwo_embed.argtypes = [vp, ctypes.c_double, ctypes.c_double, ctypes.c_double, dp]
        L.lbwo_init.argtypes = [vp, dp, ctypes.c_int]
        L.lbwo_step.argtypes = [vp, ctypes.c_longlong]
        L.lbwo_set_probes.argtypes = [vp, ip, ctypes.c_int, ctypes.c_longlong]
        L.lbwo_read_probes.restype = ctypes.c_longlong
        L.lbwo_read_probes.argtypes = [vp, dp]
        L.lbwo_get_f.argtypes = [vp, dp]
        L.lbwo_set_f.argtypes = [vp, dp]
        L.lbwo_get_P.argtypes = [vp, dp]
        L.lbwo_set_sources.argtypes = [vp, ip, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                       ctypes.c_double]
        _lib = L
    return _lib


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _ip(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))


class OracleGrid:
    """One lattice advanced by the FP64 oracle.  ``spec`` is a ``lbw_workloads.GridSpec``."""

    def __init__(self, spec):
        self.spec = spec
        ints = np.array([spec.kind, *spec.n, *spec.bc, spec.profile,
                         getattr(spec, "equilibrium", 0)], dtype=np.int32)
        dbls = np.array([*spec.h, *spec.x0, spec.c, spec.cs2, spec.damping, *spec.geom],
                        dtype=np.float64)
        assert ints.size == 12 and dbls.size == 13
        self._L = lib()
        self._h = self._L.lbwo_create(_ip(ints), _dp(dbls))
        self.n = tuple(spec.n)
        self.nn = int(np.prod(self.n))
        self._probes = 0
        self._cap = 0

    def close(self):
        if self._h:
            self._L.lbwo_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def geometry(self, u1, u2, u3):
        out = np.zeros(10)
        self._L.lbwo_geometry(self._h, u1, u2, u3, _dp(out))
        return out

    def embed(self, u1, u2, u3):
        X = np.zeros(3)
        self._L.lbwo_embed(self._h, u1, u2, u3, _dp(X))
        return X

    def init(self, pulses):
        p = np.ascontiguousarray(np.asarray(pulses, dtype=np.float64).reshape(-1, 5))
        self._L.lbwo_init(self._h, _dp(p), p.shape[0])

    def step(self, n):
        self._L.lbwo_step(self._h, int(n))

    def set_probes(self, q, cap):
        q = np.ascontiguousarray(np.asarray(q, dtype=np.int32).reshape(-1, 3))
        self._probes, self._cap = q.shape[0], int(cap)
        self._L.lbwo_set_probes(self._h, _ip(q), q.shape[0], int(cap))

    def read_probes(self):
        out = np.zeros((max(self._probes, 1), max(self._cap, 1)))
        n = self._L.lbwo_read_probes(self._h, _dp(out))
        return out[: self._probes, :n]

    def set_sources(self, q, kind=0, amp=1.0, omega=0.0):
        """Harmonic sources at lattice nodes q (n x 3): kind 0 imposes P = amp sin(omega t),
        kind 1 imposes J'_z = amp sin(omega t), at the end of every time step t (reading R8 of
        lbw_oracle.c)."""
        q = np.ascontiguousarray(np.asarray(q, dtype=np.int32).reshape(-1, 3))
        self._L.lbwo_set_sources(self._h, _ip(q), q.shape[0], int(kind), float(amp), float(omega))

    def get_f(self):
        """Post-collision populations, shape (7, N3, N1, N2)."""
        out = np.zeros(7 * self.nn)
        self._L.lbwo_get_f(self._h, _dp(out))
        return out.reshape(7, self.n[2], self.n[0], self.n[1])

    def set_f(self, f):
        a = np.ascontiguousarray(np.asarray(f, dtype=np.float64).reshape(-1))
        assert a.size == 7 * self.nn
        self._L.lbwo_set_f(self._h, _dp(a))

    def get_P(self):
        """P = rho / sqrt(g), shape (N3, N1, N2)."""
        out = np.zeros(self.nn)
        self._L.lbwo_get_P(self._h, _dp(out))
        return out.reshape(self.n[2], self.n[0], self.n[1])
