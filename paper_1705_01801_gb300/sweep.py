"""Resonance sweep: the paper's driven-source protocol (Sec. IV: a harmonic ring, plate or
point source, the steady-state pressure at a probe recorded against the source frequency).

One ensemble of identical lattices, one source frequency per member, advanced together by the
batched kernels (lbw_batch_*); the response is the largest |P| at the probe over the last
`tail` time steps, reduced on the device (lbw_batch_probe_peak).  All stepping and reduction
runs in the library's kernels; this module only assembles arrays (and refines the peak of the
response curve by a parabola through three of its points).
"""
from __future__ import annotations

import numpy as np

from . import lbw


def resonance_curve(spec, source_q, probe_q, omegas, steps: int, tail: int, kind: int = 0,
                    amp: float = 1.0):
    """Steady-state response max |P(probe)| over the last `tail` of `steps` time steps for
    each angular frequency in `omegas` (rad / step), the field starting at rest."""
    omegas = np.asarray(omegas, np.float64)
    n = len(omegas)
    source_q = np.asarray(source_q, np.int32).reshape(-1, 3)
    b = lbw.Batch([spec] * n)
    try:
        b.init([np.zeros((0, 5))] * n)
        b.set_sources(np.broadcast_to(source_q, (n,) + source_q.shape), omegas, kind=kind, amp=amp)
        b.set_probes(np.broadcast_to(np.asarray(probe_q, np.int32).reshape(1, 1, 3), (n, 1, 3)), steps)
        b.step(steps)
        peak = b.probe_peak(tail)[:, 0]
    finally:
        b.close()
    return peak


def peak_frequency(omegas, response):
    """Frequency of the largest response, refined by a parabola through its neighbours."""
    omegas = np.asarray(omegas, np.float64)
    k = int(np.argmax(response))
    if 0 < k < len(omegas) - 1:
        y0, y1, y2 = response[k - 1], response[k], response[k + 1]
        den = y0 - 2 * y1 + y2
        d = 0.5 * (y0 - y2) / den if den != 0 else 0.0
        return omegas[k] + d * (omegas[k + 1] - omegas[k])
    return omegas[k]
