"""Thin ctypes binding of liblbw.so (include/lbw.h), same names as the C ABI.

Argument marshalling only: every step of the method runs in the CUDA kernels of the
library.  There is no CPU fallback; if the library cannot be built or loaded, ``lib()``
raises.  PyTorch is used only to hand the library a CUDA stream (``torch_stream()``).
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import build as _build

LBW_OK, LBW_EINVAL, LBW_ENOMEM, LBW_ECUDA, LBW_EUNSTABLE, LBW_ETIMEOUT, LBW_ESTATE = range(7)
STATUS_NAMES = ["LBW_OK", "LBW_EINVAL", "LBW_ENOMEM", "LBW_ECUDA", "LBW_EUNSTABLE",
                "LBW_ETIMEOUT", "LBW_ESTATE"]

# every symbol the header declares (checked by tests/test_abi.py)
EXPORTS = ["lbw_create_grid", "lbw_init", "lbw_step", "lbw_probe", "lbw_probe_read",
           "lbw_spectrum", "lbw_spectrum_lowest", "lbw_spectrum_series", "lbw_spectrum_series_static", "lbw_get_field", "lbw_get_populations",
           "lbw_set_populations", "lbw_step_count", "lbw_inject_wait_timeout", "lbw_destroy", "lbw_last_error", "lbw_source",
           "lbw_batch_create", "lbw_batch_init", "lbw_batch_probe", "lbw_batch_step", "lbw_batch_source",
           "lbw_batch_probe_read", "lbw_batch_probe_peak", "lbw_batch_spectrum", "lbw_batch_spectrum_lowest", "lbw_batch_get_populations",
           "lbw_batch_tune", "lbw_batch_set_shape", "lbw_batch_info", "lbw_batch_destroy",
           "lbw_mlp_create", "lbw_mlp_param_count", "lbw_mlp_get_params", "lbw_mlp_set_params",
           "lbw_mlp_forward", "lbw_mlp_predict_bf16", "lbw_mlp_grad", "lbw_mlp_adam_step",
           "lbw_mlp_train", "lbw_mlp_destroy"]


class lbw_grid_desc(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("n", ctypes.c_int32 * 3), ("h", ctypes.c_double * 3),
                ("x0", ctypes.c_double * 3), ("c", ctypes.c_double), ("tau", ctypes.c_double),
                ("cs2", ctypes.c_double), ("damping", ctypes.c_double),
                ("geom", ctypes.c_double * 4), ("horn_profile", ctypes.c_int32),
                ("bc", ctypes.c_int32 * 6), ("prec", ctypes.c_int32),
                ("geom_mode", ctypes.c_int32), ("equilibrium", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


class lbw_pulse(ctypes.Structure):
    _fields_ = [("x", ctypes.c_double * 3), ("sigma", ctypes.c_double), ("amp", ctypes.c_double)]


class LbwError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES[status] if 0 <= status < 7 else status}: {msg}")
        self.status = status


_lock = threading.Lock()
_lib = None


def lib():
    """Build (if stale) and load the in-tree library; raises if that is impossible."""
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(_build.build())
            vp, i32, i64, dp = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.POINTER(ctypes.c_double)
            ip = ctypes.POINTER(ctypes.c_int32)
            fp = ctypes.POINTER(ctypes.c_float)
            st = ctypes.c_int
            sig = {
                "lbw_create_grid": (st, [ctypes.POINTER(lbw_grid_desc), vp, ctypes.POINTER(vp)]),
                "lbw_init": (st, [vp, ctypes.POINTER(lbw_pulse), i32]),
                "lbw_step": (st, [vp, i64]),
                "lbw_probe": (st, [vp, ip, i32, i64]),
                "lbw_source": (st, [vp, ip, i32, i32, ctypes.c_double, ctypes.c_double]),
                "lbw_batch_source": (st, [vp, ip, i32, i32, ctypes.c_double, dp]),
                "lbw_probe_read": (st, [vp, dp, i64, ctypes.POINTER(i64)]),
                "lbw_spectrum": (st, [vp, i32, i32, dp, dp, ip]),
                "lbw_spectrum_lowest": (st, [vp, i32, i32, ctypes.c_double, dp, dp, ip]),
                "lbw_spectrum_series": (st, [dp, i64, i32, i32, vp, dp, dp, ip]),
                "lbw_spectrum_series_static": (st, [vp, i64, i32, vp, dp, dp, ip]),
                "lbw_get_field": (st, [vp, dp]),
                "lbw_get_populations": (st, [vp, dp]),
                "lbw_set_populations": (st, [vp, dp]),
                "lbw_step_count": (st, [vp, ctypes.POINTER(i64)]),
                "lbw_inject_wait_timeout": (st, [vp]),
                "lbw_destroy": (None, [vp]),
                "lbw_last_error": (ctypes.c_char_p, []),
                "lbw_batch_create": (st, [ctypes.POINTER(lbw_grid_desc), i32, vp, ctypes.POINTER(vp)]),
                "lbw_batch_init": (st, [vp, ctypes.POINTER(lbw_pulse), ip]),
                "lbw_batch_probe": (st, [vp, ip, i32, i64]),
                "lbw_batch_step": (st, [vp, i64]),
                "lbw_batch_probe_read": (st, [vp, dp, ctypes.POINTER(i64)]),
                "lbw_batch_probe_peak": (st, [vp, i64, dp]),
                "lbw_batch_spectrum": (st, [vp, i32, dp, dp, ip]),
                "lbw_batch_spectrum_lowest": (st, [vp, i32, ctypes.c_double, dp, dp, ip]),
                "lbw_batch_get_populations": (st, [vp, i32, dp]),
                "lbw_batch_tune": (st, [vp, i32, ctypes.c_char_p, ctypes.c_char_p, i32]),
                "lbw_batch_set_shape": (st, [vp, i32, i32, i32]),
                "lbw_batch_info": (st, [vp, ctypes.POINTER(i64), ip, ip, ip]),
                "lbw_batch_destroy": (None, [vp]),
                "lbw_mlp_create": (st, [i32, i32, i32, i32, ctypes.c_uint64, vp, ctypes.POINTER(vp)]),
                "lbw_mlp_param_count": (st, [vp, ctypes.POINTER(i64)]),
                "lbw_mlp_get_params": (st, [vp, fp]),
                "lbw_mlp_set_params": (st, [vp, fp]),
                "lbw_mlp_forward": (st, [vp, fp, i32, fp]),
                "lbw_mlp_predict_bf16": (st, [vp, fp, i32, fp]),
                "lbw_mlp_grad": (st, [vp, fp, fp, i32, fp, fp]),
                "lbw_mlp_adam_step": (st, [vp, fp, ctypes.c_float]),
                "lbw_mlp_train": (st, [vp, fp, fp, i32, ip, i32, i32, ctypes.c_float, fp]),
                "lbw_mlp_destroy": (None, [vp]),
            }
            for name, (res, args) in sig.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
        return _lib


def library_path() -> str:
    return _build.SO


def _check(status):
    if status != LBW_OK:
        raise LbwError(status, lib().lbw_last_error().decode())


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _ip(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))


def torch_stream():
    """Handle of torch's current CUDA stream (torch only provides the stream)."""
    import torch
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def make_desc(spec) -> lbw_grid_desc:
    """lbw_grid_desc from a ``lbw_workloads.GridSpec``."""
    d = lbw_grid_desc()
    d.kind = spec.kind
    for a in range(3):
        d.n[a] = int(spec.n[a])
        d.h[a] = float(spec.h[a])
        d.x0[a] = float(spec.x0[a])
    d.c = spec.c
    d.tau = 0.5
    d.cs2 = spec.cs2
    d.damping = spec.damping
    for k in range(4):
        d.geom[k] = float(spec.geom[k])
    d.horn_profile = spec.profile
    for k in range(6):
        d.bc[k] = int(spec.bc[k])
    d.prec = spec.prec
    d.geom_mode = int(getattr(spec, "geom_mode", 0))
    d.equilibrium = int(getattr(spec, "equilibrium", 0))
    d.reserved = 0
    return d


def lbw_create_grid(desc: lbw_grid_desc, stream=None):
    out = ctypes.c_void_p()
    _check(lib().lbw_create_grid(ctypes.byref(desc), stream, ctypes.byref(out)))
    return out


def lbw_init(grid, pulses):
    p = np.asarray(pulses, dtype=np.float64).reshape(-1, 5)
    arr = (lbw_pulse * max(1, p.shape[0]))()
    for k in range(p.shape[0]):
        arr[k].x[0], arr[k].x[1], arr[k].x[2], arr[k].sigma, arr[k].amp = p[k]
    _check(lib().lbw_init(grid, arr, p.shape[0]))


def lbw_step(grid, n):
    _check(lib().lbw_step(grid, int(n)))


def lbw_probe(grid, q, capacity):
    q = np.ascontiguousarray(np.asarray(q, dtype=np.int32).reshape(-1, 3))
    _check(lib().lbw_probe(grid, _ip(q), q.shape[0], int(capacity)))


def lbw_source(grid, q, kind, amp, omega):
    q = np.ascontiguousarray(np.asarray(q, dtype=np.int32).reshape(-1, 3))
    _check(lib().lbw_source(grid, _ip(q), q.shape[0], int(kind), float(amp), float(omega)))


def lbw_probe_read(grid, n_probes, cap):
    out = np.zeros((max(1, n_probes), max(1, cap)))
    n = ctypes.c_int64()
    _check(lib().lbw_probe_read(grid, _dp(out), max(1, cap), ctypes.byref(n)))
    return out[:n_probes, : n.value]


def lbw_spectrum(grid, probe, k):
    f = np.zeros(k)
    a = np.zeros(k)
    n = ctypes.c_int32()
    _check(lib().lbw_spectrum(grid, int(probe), int(k), _dp(f), _dp(a), ctypes.byref(n)))
    return f[: n.value], a[: n.value]


def lbw_spectrum_lowest(grid, probe, k, rel_power=1e-3):
    f = np.zeros(k)
    a = np.zeros(k)
    n = ctypes.c_int32()
    _check(lib().lbw_spectrum_lowest(grid, int(probe), int(k), float(rel_power), _dp(f), _dp(a),
                                     ctypes.byref(n)))
    return f[: n.value], a[: n.value]


def lbw_spectrum_series(x, k, stream=None):
    x = np.ascontiguousarray(np.atleast_2d(np.asarray(x, dtype=np.float64)))
    ns, T = x.shape
    f = np.zeros((ns, k))
    a = np.zeros((ns, k))
    n = np.zeros(ns, dtype=np.int32)
    _check(lib().lbw_spectrum_series(_dp(x), T, ns, int(k), stream, _dp(f), _dp(a), _ip(n)))
    return [(f[j, : n[j]], a[j, : n[j]]) for j in range(ns)]


def lbw_spectrum_series_static(dev_ptr, T, k, stream=None):
    """Spectrum of T doubles already in device memory at dev_ptr, using the library's fixed
    workspace (no device allocation); returns (freq, amp)."""
    f = np.zeros(k)
    a = np.zeros(k)
    n = ctypes.c_int32()
    _check(lib().lbw_spectrum_series_static(ctypes.c_void_p(dev_ptr), int(T), int(k), stream,
                                            _dp(f), _dp(a), ctypes.byref(n)))
    return f[: n.value], a[: n.value]


def lbw_get_field(grid, shape):
    out = np.zeros(int(np.prod(shape)))
    _check(lib().lbw_get_field(grid, _dp(out)))
    return out.reshape(shape)


def lbw_get_populations(grid, nn):
    out = np.zeros(7 * nn)
    _check(lib().lbw_get_populations(grid, _dp(out)))
    return out


def lbw_set_populations(grid, f):
    a = np.ascontiguousarray(np.asarray(f, dtype=np.float64).reshape(-1))
    _check(lib().lbw_set_populations(grid, _dp(a)))


def lbw_step_count(grid):
    n = ctypes.c_int64()
    _check(lib().lbw_step_count(grid, ctypes.byref(n)))
    return n.value


def lbw_inject_wait_timeout(grid):
    _check(lib().lbw_inject_wait_timeout(grid))


def lbw_destroy(grid):
    lib().lbw_destroy(grid)


def lbw_last_error():
    return lib().lbw_last_error().decode()


class Grid:
    """Convenience owner of one lbw_grid (a ``lbw_workloads.GridSpec`` in, numpy out)."""

    def __init__(self, spec, stream=None):
        self.spec = spec
        self.n = tuple(int(v) for v in spec.n)
        self.nn = int(np.prod(self.n))
        self._h = lbw_create_grid(make_desc(spec), stream)
        self._nprobe = 0
        self._cap = 0

    def close(self):
        if self._h:
            lbw_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def handle(self):
        return self._h

    def init(self, pulses):
        lbw_init(self._h, pulses)

    def step(self, n):
        lbw_step(self._h, n)

    def set_sources(self, q, kind=0, amp=1.0, omega=0.0):
        lbw_source(self._h, q, kind, amp, omega)

    def set_probes(self, q, cap):
        q = np.asarray(q, dtype=np.int32).reshape(-1, 3)
        lbw_probe(self._h, q, cap)
        self._nprobe, self._cap = q.shape[0], int(cap)

    def read_probes(self):
        return lbw_probe_read(self._h, self._nprobe, self._cap)

    def spectrum(self, probe=0, k=8, lowest=False, rel_power=1e-3):
        """k strongest peaks, or with `lowest` the k lowest-frequency peaks whose power is at
        least rel_power of the strongest; (freq rad/step, amp), sorted by frequency."""
        if lowest:
            return lbw_spectrum_lowest(self._h, probe, k, rel_power)
        return lbw_spectrum(self._h, probe, k)

    def get_P(self):
        """P, shape (N3, N1, N2)."""
        return lbw_get_field(self._h, (self.n[2], self.n[0], self.n[1]))

    def get_f(self):
        """Post-collision populations as doubles, shape (7, N3, N1, N2)."""
        return lbw_get_populations(self._h, self.nn).reshape(7, self.n[2], self.n[0], self.n[1])

    def set_f(self, f):
        lbw_set_populations(self._h, f)

    def step_count(self):
        return lbw_step_count(self._h)


class Batch:
    """Owner of one lbw_batch: a list of ``lbw_workloads.GridSpec`` in, numpy out."""

    def __init__(self, specs, stream=None):
        self.specs = list(specs)
        n = len(self.specs)
        descs = (lbw_grid_desc * n)(*[make_desc(s) for s in self.specs])
        out = ctypes.c_void_p()
        _check(lib().lbw_batch_create(descs, n, stream, ctypes.byref(out)))
        self._h = out
        self.n = n
        self._per = 0
        self._cap = 0

    def close(self):
        if self._h:
            lib().lbw_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def tune(self, trial_steps=3, cache_path=None):
        rep = ctypes.create_string_buffer(8192)
        _check(lib().lbw_batch_tune(self._h, int(trial_steps),
                                    cache_path.encode() if cache_path else None, rep, 8192))
        return rep.value.decode()

    def set_shape(self, tile_rows, seg_planes, ctas_per_sm):
        """Launch shape chosen by the caller (tile_rows 0: full-row tiles)."""
        _check(lib().lbw_batch_set_shape(self._h, int(tile_rows), int(seg_planes), int(ctas_per_sm)))

    def info(self):
        t, by, lz, cps = ctypes.c_int64(), ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
        _check(lib().lbw_batch_info(self._h, ctypes.byref(t), ctypes.byref(by), ctypes.byref(lz),
                                    ctypes.byref(cps)))
        return {"nodes": t.value, "tile_rows": by.value, "seg_planes": lz.value,
                "ctas_per_sm": cps.value}

    def init(self, pulses_per_member):
        counts = np.array([len(np.asarray(p).reshape(-1, 5)) for p in pulses_per_member], np.int32)
        allp = np.concatenate([np.asarray(p, np.float64).reshape(-1, 5) for p in pulses_per_member])
        arr = (lbw_pulse * max(1, len(allp)))()
        for k, row in enumerate(allp):
            arr[k].x[0], arr[k].x[1], arr[k].x[2], arr[k].sigma, arr[k].amp = row
        _check(lib().lbw_batch_init(self._h, arr, _ip(counts)))

    def set_probes(self, q, cap):
        q = np.ascontiguousarray(np.asarray(q, np.int32).reshape(self.n, -1, 3))
        _check(lib().lbw_batch_probe(self._h, _ip(q), q.shape[1], int(cap)))
        self._per, self._cap = q.shape[1], int(cap)

    def set_sources(self, q, omegas, kind=0, amp=1.0):
        """q: n x per_member x 3 source nodes; omegas: one angular frequency per member."""
        q = np.ascontiguousarray(np.asarray(q, np.int32).reshape(self.n, -1, 3))
        om = np.ascontiguousarray(np.asarray(omegas, np.float64).reshape(self.n))
        _check(lib().lbw_batch_source(self._h, _ip(q), q.shape[1], int(kind), float(amp), _dp(om)))

    def step(self, n):
        _check(lib().lbw_batch_step(self._h, int(n)))

    def read_probes(self):
        out = np.zeros((self.n, max(1, self._per), max(1, self._cap)))
        n = ctypes.c_int64()
        _check(lib().lbw_batch_probe_read(self._h, _dp(out), ctypes.byref(n)))
        return out[:, : self._per, : n.value]

    def probe_peak(self, tail):
        """Largest |P| of every member's probes over the last `tail` samples, (n, per_member)."""
        out = np.zeros(self.n * max(1, self._per))
        _check(lib().lbw_batch_probe_peak(self._h, int(tail), _dp(out)))
        return out.reshape(self.n, max(1, self._per))

    def spectrum(self, k=8, lowest=False, rel_power=1e-3):
        """Per member the k strongest peaks, or (lowest) the k lowest-frequency peaks with at
        least rel_power of the strongest's power; frequencies sorted, rad / step."""
        f = np.zeros((self.n, k))
        a = np.zeros((self.n, k))
        c = np.zeros(self.n, np.int32)
        if lowest:
            _check(lib().lbw_batch_spectrum_lowest(self._h, int(k), float(rel_power), _dp(f), _dp(a), _ip(c)))
        else:
            _check(lib().lbw_batch_spectrum(self._h, int(k), _dp(f), _dp(a), _ip(c)))
        return f, a, c

    def get_f(self, member):
        s = self.specs[member]
        nn = int(np.prod(s.n))
        out = np.zeros(7 * nn)
        _check(lib().lbw_batch_get_populations(self._h, int(member), _dp(out)))
        return out.reshape(7, s.n[2], s.n[0], s.n[1])


def _fp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_float))


class MLP:
    """Owner of one lbw_mlp (numpy float32 in / out)."""

    def __init__(self, in_dim, hidden=256, depth=4, out_dim=8, seed=0, stream=None):
        out = ctypes.c_void_p()
        _check(lib().lbw_mlp_create(int(in_dim), int(hidden), int(depth), int(out_dim),
                                    ctypes.c_uint64(seed), stream, ctypes.byref(out)))
        self._h = out
        self.in_dim, self.out_dim = int(in_dim), int(out_dim)
        n = ctypes.c_int64()
        _check(lib().lbw_mlp_param_count(self._h, ctypes.byref(n)))
        self.nparam = n.value

    def close(self):
        if self._h:
            lib().lbw_mlp_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def get_params(self):
        p = np.zeros(self.nparam, np.float32)
        _check(lib().lbw_mlp_get_params(self._h, _fp(p)))
        return p

    def set_params(self, p):
        p = np.ascontiguousarray(np.asarray(p, np.float32))
        assert p.size == self.nparam
        _check(lib().lbw_mlp_set_params(self._h, _fp(p)))

    def forward(self, x):
        x = np.ascontiguousarray(np.asarray(x, np.float32))
        y = np.zeros((x.shape[0], self.out_dim), np.float32)
        _check(lib().lbw_mlp_forward(self._h, _fp(x), x.shape[0], _fp(y)))
        return y

    def predict_bf16(self, x):
        x = np.ascontiguousarray(np.asarray(x, np.float32))
        y = np.zeros((x.shape[0], self.out_dim), np.float32)
        _check(lib().lbw_mlp_predict_bf16(self._h, _fp(x), x.shape[0], _fp(y)))
        return y

    def grad(self, x, t):
        x = np.ascontiguousarray(np.asarray(x, np.float32))
        t = np.ascontiguousarray(np.asarray(t, np.float32))
        g = np.zeros(self.nparam, np.float32)
        loss = np.zeros(1, np.float32)
        _check(lib().lbw_mlp_grad(self._h, _fp(x), _fp(t), x.shape[0], _fp(g), _fp(loss)))
        return float(loss[0]), g

    def adam_step(self, g, lr):
        g = np.ascontiguousarray(np.asarray(g, np.float32))
        _check(lib().lbw_mlp_adam_step(self._h, _fp(g), ctypes.c_float(lr)))

    def train(self, x, t, order, batch, lr):
        x = np.ascontiguousarray(np.asarray(x, np.float32))
        t = np.ascontiguousarray(np.asarray(t, np.float32))
        order = np.ascontiguousarray(np.asarray(order, np.int32))
        steps = order.size // batch
        loss = np.zeros(max(1, steps), np.float32)
        _check(lib().lbw_mlp_train(self._h, _fp(x), _fp(t), x.shape[0], _ip(order), steps, int(batch),
                                   ctypes.c_float(lr), _fp(loss)))
        return loss[:steps]
