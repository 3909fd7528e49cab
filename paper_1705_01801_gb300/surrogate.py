"""Surrogate from trumpet geometry to its lowest mode frequencies.

The batched lattice-Boltzmann ensemble (lbw_batch_*) measures, for every member, the spectrum
of the sum of its probes (a ring of pulses at one rigid corner, a ring of probes at the other,
so the axisymmetric modes dominate); its `n_modes` lowest-frequency peaks above a power
threshold are the targets.  A multilayer perceptron (lbw_mlp_*: device forward / backward / Adam
kernels, BF16-weight inference) maps normalised geometry features to those frequencies.  The
lattice-Boltzmann runs remain the reference: `measure` gives the values the surrogate
is trained on and checked against.  All arithmetic runs in the library's kernels; this module
only assembles arrays.
"""
from __future__ import annotations

import math
import time

import numpy as np

import lbw_workloads as W

from . import lbw

FEATURE_NAMES = ["R_outer / 100", "L / 512", "a(L) / a(0)", "alpha L", "n_theta / 96",
                 "r_in / R_outer", "b / (a0 + b)"]


def features(spec: W.GridSpec) -> np.ndarray:
    """Normalised geometry of an exponential-flare trumpet member."""
    n1, n2, n3 = spec.n
    r_in = spec.x0[0]
    R = r_in + n1 * spec.h[0]
    L = n3 * spec.h[2]
    a0, b, al = spec.geom[:3]
    ratio = (a0 + b * math.exp(al * L)) / (a0 + b)
    return np.array([R / 100.0, L / 512.0, ratio, al * L, n2 / 96.0, r_in / R, b / (a0 + b)],
                    dtype=np.float32)


def measure(specs, steps: int, n_modes: int = 8, rel_power: float = 1e-3, tune: bool = True):
    """Run the ensemble for `steps` time steps and return (freqs [n, n_modes], valid [n],
    seconds of device work).  Targets are the n_modes lowest-frequency spectral peaks (rad /
    step) whose power is at least rel_power of the member's strongest peak (window side lobes
    stay below it); members with fewer such peaks are marked invalid."""
    import torch
    b = lbw.Batch(specs)
    if tune:
        b.tune(trial_steps=2)
    exc = [W.ensemble_excitation(s) for s in specs]
    b.init([e[0] for e in exc])
    b.set_probes(np.stack([e[1] for e in exc]), steps)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    b.step(steps)
    f, a, cnt = b.spectrum(n_modes, lowest=True, rel_power=rel_power)
    seconds = time.perf_counter() - t0
    valid = cnt >= n_modes
    out = np.where(valid[:, None], f, 0.0)
    b.close()
    return out, valid, seconds


class Surrogate:
    """Standardised inputs and outputs around lbw.MLP networks (4 weight layers, 256 wide):
    one network for all modes, or (per_mode) one network per mode, so that the smooth lowest
    modes do not share capacity with the higher ones, whose order changes where mode families
    cross."""

    def __init__(self, in_dim: int = len(FEATURE_NAMES), out_dim: int = 8, hidden: int = 256,
                 depth: int = 4, seed: int = 0, per_mode: bool = False):
        self.per_mode = per_mode
        if per_mode:
            self.nets = [lbw.MLP(in_dim, hidden=hidden, depth=depth, out_dim=1, seed=seed * out_dim + k)
                         for k in range(out_dim)]
        else:
            self.nets = [lbw.MLP(in_dim, hidden=hidden, depth=depth, out_dim=out_dim, seed=seed)]
        self.mx = self.sx = self.my = self.sy = None

    def fit(self, X, Y, steps: int = 4000, batch: int = 64, lr: float = 1e-3, seed: int = 0,
            decay_chunks: int = 20):
        """Adam on the standardised log-frequencies; the learning rate follows a cosine decay
        from lr, held constant over each of decay_chunks equal runs of steps (1: constant).
        Returns the minibatch loss curve of every network, shape (networks, steps)."""
        X = np.asarray(X, np.float64)
        Y = np.log(np.asarray(Y, np.float64))  # frequencies are positive and span decades
        self.mx, self.sx = X.mean(0), X.std(0) + 1e-12
        self.my, self.sy = Y.mean(0), Y.std(0) + 1e-12
        Xn = ((X - self.mx) / self.sx).astype(np.float32)
        Yn = ((Y - self.my) / self.sy).astype(np.float32)
        rng = np.random.default_rng(seed)  # minibatch order drawn here, passed to the kernels
        per_epoch = max(1, len(Xn) // batch)
        order = np.concatenate([rng.permutation(len(Xn))[: per_epoch * batch]
                                for _ in range(math.ceil(steps / per_epoch))])[: steps * batch]
        chunks = max(1, min(decay_chunks, steps))
        curves = []
        for k, net in enumerate(self.nets):
            T = np.ascontiguousarray(Yn[:, k:k + 1] if self.per_mode else Yn)
            curve = []
            for c in range(chunks):
                lo, hi = steps * c // chunks, steps * (c + 1) // chunks
                rate = lr * 0.5 * (1.0 + math.cos(math.pi * c / chunks)) if chunks > 1 else lr
                curve.append(net.train(Xn, T, order[lo * batch:hi * batch], batch, rate))
            curves.append(np.concatenate(curve))
        return np.stack(curves)

    def predict(self, X, bf16: bool = True):
        Xn = ((np.asarray(X, np.float64) - self.mx) / self.sx).astype(np.float32)
        Yn = np.concatenate([net.predict_bf16(Xn) if bf16 else net.forward(Xn) for net in self.nets], axis=1)
        return np.exp(Yn.astype(np.float64) * self.sy + self.my)


class SurrogateEnsemble:
    """k independently initialised surrogates answering together.  The answer is their mean in
    log-frequency; the spread between them (largest standard deviation of log f over the
    modes) measures how far a query lies from what the training data pins down.  Queries whose
    spread exceeds a calibrated threshold fall back to the lattice-Boltzmann ensemble, which
    stays the judge of the error: a fallback answer is the LBM's own."""

    def __init__(self, k: int = 4, **kw):
        self.members = [Surrogate(seed=s, **kw) for s in range(k)]
        self.threshold = np.inf

    def fit(self, X, Y, **kw):
        return [m.fit(X, Y, seed=i, **kw) for i, m in enumerate(self.members)]

    def predict(self, X, bf16: bool = True):
        """(mean frequencies [n, modes], spread [n])."""
        logp = np.log(np.stack([m.predict(X, bf16) for m in self.members]))
        return np.exp(logp.mean(0)), logp.std(0).max(1)

    def calibrate(self, X, Y, target: float):
        """Largest spread threshold at which the accepted queries of (X, Y) keep a mean relative
        error <= target; returns the fraction accepted."""
        pred, spread = self.predict(X)
        err = (np.abs(pred - Y) / Y).mean(1)
        order = np.argsort(spread)
        mean_err = np.cumsum(err[order]) / np.arange(1, len(err) + 1)
        ok = np.nonzero(mean_err <= target)[0]
        if len(ok) == 0:
            self.threshold = -np.inf
            return 0.0
        last = ok[-1]
        self.threshold = spread[order[last]]
        return (last + 1) / len(err)

    def answer(self, specs, X, steps: int, n_modes: int = 8):
        """Frequencies for every query: the ensemble's mean where its spread is within the
        threshold, the LBM's measurement (``measure``) elsewhere.  Returns (freqs, fell_back
        mask, seconds of surrogate work, seconds of LBM work)."""
        t0 = time.perf_counter()
        pred, spread = self.predict(X)
        sur_s = time.perf_counter() - t0
        back = spread > self.threshold
        lbm_s = 0.0
        if back.any():
            sub = [s for s, b in zip(specs, back) if b]
            f, valid, lbm_s = measure(sub, steps=steps, n_modes=n_modes, tune=False)
            pred[back] = np.where(valid[:, None], f, np.nan)
        return pred, back, sur_s, lbm_s
