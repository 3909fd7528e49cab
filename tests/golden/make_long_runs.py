"""Write the FP64 oracle's full-length runs of two benchmark lattices into tests/golden/.

Only the oracle (``oracle/``) and the seeded input generators (``lbw_workloads``) are used, so
every stored value comes from the plain CPU implementation of the paper's step.  Each file
holds, for the workload's own seeded pulses and probes:

* the k = 8 strongest spectral peaks of the summed probe series (the estimator of
  ``oracle.spectrum``: Hann window, zero padding to 4 T, parabolic and golden-section
  refinement), frequency in rad / step and amplitude;
* P = rho / sqrt(g) at 256 seeded lattice nodes after each checkpoint step count.

Usage (repo root; OpenMP threads = host cores):

    python tests/golden/make_long_runs.py cylinder   # 128 x 128 x 256, 20 000 steps
    python tests/golden/make_long_runs.py torus      # 192 x 1024 x 256, 500 steps

The cylinder runs the benchmark's full 20 000 steps; the torus runs 500 of its 50 000, the
length the oracle finishes in about half an hour on eight host cores.
"""
from __future__ import annotations

import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import lbw_workloads as W  # noqa: E402
import oracle  # noqa: E402

RUNS = {
    "cylinder": (20000, [1000, 2000, 5000, 10000, 20000]),
    "torus": (500, [100, 250, 500]),
}
N_SAMPLES = 256
SAMPLE_SEED = 77
K_PEAKS = 8


def sample_nodes(spec, count=N_SAMPLES, seed=SAMPLE_SEED):
    """count distinct seeded lattice nodes (q1, q2, q3), uniform over the lattice."""
    rng = np.random.default_rng(seed)
    flat = rng.choice(spec.nodes, size=count, replace=False)
    n1, n2 = spec.n[0], spec.n[1]
    q2 = flat % n2
    q1 = (flat // n2) % n1
    q3 = flat // (n1 * n2)
    return np.stack([q1, q2, q3], 1).astype(np.int64)


def path_for(name):
    steps, _ = RUNS[name]
    return os.path.join(HERE, f"{name}_{steps}_steps_f64.txt")


def run(name):
    steps, checkpoints = RUNS[name]
    wl = W.workload(name)
    spec = wl.spec.with_(prec=W.PREC_F64)
    nodes = sample_nodes(spec)
    g = oracle.OracleGrid(spec)
    g.init(wl.pulses)
    g.set_probes(wl.probes, steps)
    t0 = time.perf_counter()
    done, fields = 0, []
    for cp in checkpoints:
        g.step(cp - done)
        done = cp
        P = g.get_P()  # (N3, N1, N2)
        fields.append((cp, P[nodes[:, 2], nodes[:, 0], nodes[:, 1]].copy()))
        print(f"{name}: {cp} steps, {time.perf_counter() - t0:.0f} s", flush=True)
    series = g.read_probes()
    freq, amp = oracle.spectrum(series.sum(0), K_PEAKS)
    wall = time.perf_counter() - t0
    with open(path_for(name), "w") as fh:
        fh.write(f"# FP64 oracle, workload {name} ({wl.notes}), {steps} time steps, "
                 f"{wl.probes.shape[0]} probes, seeded pulses of lbw_workloads.workload('{name}')\n")
        fh.write(f"# written by tests/golden/make_long_runs.py in {wall:.0f} s on "
                 f"{os.environ.get('OMP_NUM_THREADS', os.cpu_count())} host threads\n")
        fh.write(f"peaks {len(freq)}  # freq (rad/step) amp, summed probe series, k = {K_PEAKS}\n")
        for f, a in zip(freq, amp):
            fh.write(f"{float(f)!r} {float(a)!r}\n")
        fh.write(f"samples {len(nodes)} seed {SAMPLE_SEED}  # q1 q2 q3\n")
        for q in nodes:
            fh.write(f"{q[0]} {q[1]} {q[2]}\n")
        for cp, vals in fields:
            fh.write(f"field {cp}  # P at the sampled nodes after {cp} steps\n")
            for v in vals:
                fh.write(f"{float(v)!r}\n")


def load(name):
    """(steps, peaks (n x 2), nodes (256 x 3), {step: P values}) of a stored run."""
    steps, _ = RUNS[name]
    with open(path_for(name)) as fh:
        lines = [l.split("#")[0].strip() for l in fh]
    lines = [l for l in lines if l]
    i, peaks, nodes, fields = 0, None, None, {}
    while i < len(lines):
        head = lines[i].split()
        if head[0] == "peaks":
            n = int(head[1])
            peaks = np.array([[float(x) for x in lines[i + 1 + j].split()] for j in range(n)])
            i += n + 1
        elif head[0] == "samples":
            n = int(head[1])
            nodes = np.array([[int(x) for x in lines[i + 1 + j].split()] for j in range(n)])
            i += n + 1
        elif head[0] == "field":
            cp = int(head[1])
            fields[cp] = np.array([float(lines[i + 1 + j]) for j in range(len(nodes))])
            i += len(nodes) + 1
        else:
            raise ValueError(f"bad line {lines[i]!r}")
    return steps, peaks, nodes, fields


if __name__ == "__main__":
    for name in sys.argv[1:] or list(RUNS):
        run(name)
