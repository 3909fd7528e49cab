"""Mode-frequency estimator of a probe series, FP64 numpy.  TEST INFRASTRUCTURE ONLY.

The paper reads resonances off driven sweeps (Sec. IV.A, Fig. Fig.Frequencies; Sec. IV.C,
Fig. FreqTorus); for a pulse-excited run the same normal modes are the peaks of the probe
signal's spectrum.  The estimator, in order:

1. subtract the series mean;
2. Hann window w_t = 1/2 - 1/2 cos(2 pi t / (T - 1)), t = 0..T-1;
3. zero-pad to M = the smallest power of two >= pad * T and take |DFT|^2 at bins 0..M/2;
4. local maxima j in [1, M/2 - 1] with P[j] > P[j-1], P[j] >= P[j+1] and
   P[j] >= thresh * max_{j>=1} P[j]; keep the k largest (ties: lower j first), then sort them
   by frequency;
5. refine each: parabola through log P at j-1, j, j+1 gives j + delta; then a fixed number of
   golden-section iterations maximise |sum_t w_t x_t e^{-i omega t}|^2 on
   [omega_j - 2 pi / M, omega_j + 2 pi / M], omega_j = 2 pi (j + delta) / M;
6. amplitude = 2 |X(omega)| / sum_t w_t.

Frequencies are in radians per time step.
"""
from __future__ import annotations

import numpy as np

GOLDEN = 0.6180339887498949


def _dtft_power(xw: np.ndarray, omega: float) -> float:
    t = np.arange(xw.size, dtype=np.float64)
    re = np.sum(xw * np.cos(omega * t))
    im = -np.sum(xw * np.sin(omega * t))
    return re * re + im * im


def spectrum(x, k: int = 8, pad: int = 4, thresh: float = 1e-3, iters: int = 40,
             lowest: bool = False):
    """Return (freq[n_found], amp[n_found]) of the k strongest spectral peaks of x, or with
    `lowest` of the k lowest-frequency peaks whose power is at least thresh of the largest."""
    x = np.asarray(x, dtype=np.float64)
    T = x.size
    if T < 4:
        return np.zeros(0), np.zeros(0)
    x = x - x.mean()
    t = np.arange(T, dtype=np.float64)
    w = 0.5 - 0.5 * np.cos(2.0 * np.pi * t / (T - 1))
    xw = w * x
    M = 1
    while M < pad * T:
        M *= 2
    P = np.abs(np.fft.rfft(xw, M)) ** 2
    pmax = P[1:].max()
    if not pmax > 0.0:
        return np.zeros(0), np.zeros(0)
    cand = [j for j in range(1, M // 2)
            if P[j] > P[j - 1] and P[j] >= P[j + 1] and P[j] >= thresh * pmax]
    cand.sort(key=(lambda j: j) if lowest else (lambda j: (-P[j], j)))
    cand = sorted(cand[:k])
    sw = w.sum()
    freqs, amps = [], []
    for j in cand:
        la, lb, lc = np.log(P[j - 1]), np.log(P[j]), np.log(P[j + 1])
        den = la - 2.0 * lb + lc
        delta = 0.5 * (la - lc) / den if den < 0.0 else 0.0
        om = 2.0 * np.pi * (j + delta) / M
        half = 2.0 * np.pi / M
        a, b = om - half, om + half
        for _ in range(iters):
            c = b - GOLDEN * (b - a)
            d = a + GOLDEN * (b - a)
            if _dtft_power(xw, c) > _dtft_power(xw, d):
                b = d
            else:
                a = c
        om = 0.5 * (a + b)
        freqs.append(om)
        amps.append(2.0 * np.sqrt(_dtft_power(xw, om)) / sw)
    return np.array(freqs), np.array(amps)
