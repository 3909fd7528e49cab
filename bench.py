"""Benchmark of the fused curvilinear wave-LBM sweep on GB300.

One benchmark step = one run of the whole hot path on the torus workload (r 192 x theta 1024
x phi 256 = 50,331,648 nodes, R / a = 3, FP32 storage, one seeded Gaussian pulse): 2000 time
steps of the fused stream + collide kernel with 64 probes recorded every step, then the device
spectrum of the summed probes.  Metric: MLUPS = nodes x time steps / seconds / 1e6 (whole
job, all ranks).

  value  device-timed: the initial state is rebuilt (untimed) before every step, then
         CUDA events on the library's stream bracket lbw_step + lbw_spectrum.
  e2e    the same run through the public C ABI from host buffers: lbw_init (host pulses),
         lbw_probe (host probe nodes), lbw_step, lbw_probe_read (series to host) and
         lbw_spectrum, all inside the timed region.
The torus's working set (two population buffers, 2.82 GB in FP32) is 22 times the 129 MB L2,
so no flush is needed between steps.  --workload selects the other lattices (their own time
step counts unless --lbm-steps is given); --impl reference times the FP64 CPU oracle on the
same workload.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import lbw_workloads as W  # noqa: E402

# time steps per benchmark step: the torus runs a stated 2000 (its full 50 000-step run takes
# 24 s per step on the GPU); the other workloads run their own full length
BENCH_TIME_STEPS = {"torus": 2000}
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(x: float, device=None) -> float:
    """The largest x over the ranks of the default process group (x itself without one): the
    whole job takes as long as its slowest rank."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_mlups(nodes: int, time_steps: int, world_size: int, seconds: float) -> float:
    """Lattice updates of all ranks (one replica each) per second, in millions."""
    return nodes * time_steps * world_size / seconds / 1e6


def _peaks():
    try:
        with open(PEAKS_FILE) as fh:
            p = json.load(fh)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.lines = []
        if self.proc is not None:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except Exception:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [l for l in out.splitlines() if l.strip()]

    def summary(self):
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in getattr(self, "lines", []):
            v = [x.strip() for x in l.split(",")]
            if len(v) < 9:
                continue
            try:
                sm.append(float(v[1]))
                mx = max(mx, float(v[2]))
            except ValueError:
                continue
            for n, flag in zip(names, v[5:9]):
                if flag.lower() in ("active", "0x1", "1"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx or None,
                "reasons": sorted(reasons), "samples": len(sm)}


WORKLOAD = "torus"
PREC_OVERRIDE = None
SHAPE = None
GEOM_MODE = 0


def workload():
    """The benchmark workload (torus by default; --workload / --prec select another)."""
    wl = W.workload(WORKLOAD, SHAPE)
    if PREC_OVERRIDE is not None:
        wl.spec = wl.spec.with_(prec=PREC_OVERRIDE)
    wl.spec = wl.spec.with_(geom_mode=GEOM_MODE)
    return wl


def cpu_baseline(spec, pulses, probes, budget_s=15.0):
    """The FP64 oracle, as it stands, on a bounded sample of the same workload: the full
    lattice for as many time steps as fit in ~budget_s seconds of host time."""
    import oracle
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    g = oracle.OracleGrid(spec)
    g.init(pulses)
    g.set_probes(probes, 1 << 16)
    t0 = time.perf_counter()
    g.step(1)
    t1 = time.perf_counter() - t0
    n = max(1, int(budget_s / max(t1, 1e-6)) - 1)
    t0 = time.perf_counter()
    g.step(n)
    dt = time.perf_counter() - t0
    mlups = spec.nodes * n / dt / 1e6
    return {"value": mlups, "unit": "MLUPS", "cores": cores, "kind": "oracle",
            "sample": f"full {spec.n[0]}x{spec.n[1]}x{spec.n[2]} lattice, {n} time steps "
                      f"({dt:.1f} s) of the FP64 C oracle, OpenMP over nodes"}


ENSEMBLE_STEPS = 512


def run_ensemble(args):
    """The batched form: seeded trumpets of uneven sizes (r, theta in [32, 96], z in [128, 512])
    advanced together by the persistent ensemble kernel (shape from the library's autotuner,
    untimed), each benchmark step = the time steps plus every member's spectrum."""
    import torch
    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_1705_01801_gb300 import lbw
    prec = PREC_OVERRIDE if PREC_OVERRIDE is not None else W.PREC_F32
    specs, _ = W.ensemble(args.members, seed=5, prec=prec)
    nodes = sum(s.nodes for s in specs)
    lbm_steps = args.lbm_steps if args.lbm_steps is not None else ENSEMBLE_STEPS
    stream = torch.cuda.Stream()
    sh = lbw.ctypes.c_void_p(stream.cuda_stream)
    b = lbw.Batch(specs, stream=sh)
    if args.launch:
        rows, planes, ctas = (int(v) for v in args.launch.split(","))
        b.set_shape(rows, planes, ctas)
        tune_report = f"set by={rows} lz={planes} cps={ctas}"
    else:
        tune_report = b.tune(trial_steps=2).strip().splitlines()[-1]
    exc = [W.ensemble_excitation(s) for s in specs]
    pulses = [e[0] for e in exc]
    probes_q = np.stack([e[1] for e in exc])

    def device_step():
        b.init(pulses)
        b.set_probes(probes_q, lbm_steps)
        stream.synchronize()
        ev0, ev1, ev2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        ev0.record(stream)
        b.step(lbm_steps)
        ev1.record(stream)
        f, a, cnt = b.spectrum(8)
        ev2.record(stream)
        ev2.synchronize()
        return ev0.elapsed_time(ev2), ev0.elapsed_time(ev1)

    for _ in range(args.warmup):
        device_step()
    torch.cuda.synchronize()
    tot, stp = [], []
    with ClockSampler(local) as clk:
        for _ in range(args.steps):
            t, s_ = device_step()
            tot.append(t)
            stp.append(s_)
    my_ms = max_over_ranks(sum(tot), device="cuda")
    value = whole_job_mlups(nodes, lbm_steps * args.steps, ws, my_ms / 1e3)
    elem = {W.PREC_F64: 8, W.PREC_F32: 4, W.PREC_F16S: 2, W.PREC_BF16S: 2}[prec]
    kernel_ms = sum(stp) / (args.steps * lbm_steps)
    achieved = nodes * 14 * elem / (kernel_ms / 1e3) / 1e9
    peak, peak_kind = _peaks()

    # end to end through the C ABI with host buffers: pulses and probe nodes in, series and
    # spectra out
    t0 = time.perf_counter()
    for _ in range(args.steps):
        b.init(pulses)
        b.set_probes(probes_q, lbm_steps)
        b.step(lbm_steps)
        series = b.read_probes()
        f, a, cnt = b.spectrum(8)
    torch.cuda.synchronize()
    e2e_s = max_over_ranks(time.perf_counter() - t0, device="cuda")
    e2e_value = whole_job_mlups(nodes, lbm_steps * args.steps, ws, e2e_s)
    h2d = sum(np.asarray(p).nbytes for p in pulses) + probes_q.astype(np.int32).nbytes
    d2h = series.nbytes + 2 * 8 * 8 * len(specs)
    b.close()
    sequential = None
    if args.vs_sequential > 0:
        # the same members one after another, each its own lattice on the single-lattice path
        sub = specs[: args.vs_sequential]
        grids = [lbw.Grid(s_, stream=sh) for s_ in sub]
        for g_, p_ in zip(grids, pulses):
            g_.init(p_)
            g_.step(8)
        stream.synchronize()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        for g_ in grids:
            g_.step(lbm_steps)
        ev1.record(stream)
        ev1.synchronize()
        seq_ms = ev0.elapsed_time(ev1)
        sub_nodes = sum(s_.nodes for s_ in sub)
        seq = sub_nodes * lbm_steps / (seq_ms / 1e3) / 1e6
        sequential = {"members": len(sub), "mlups": seq,
                      "batched_step_mlups": nodes * lbm_steps * args.steps / (sum(stp) / 1e3) / 1e6}
        sequential["batched_over_sequential"] = sequential["batched_step_mlups"] / seq
        for g_ in grids:
            g_.close()
    if rank != 0:
        if ws > 1:
            torch.distributed.destroy_process_group()
        return 0
    base = None
    if not args.no_cpu_baseline and ws == 1:
        base = cpu_baseline(specs[0], pulses[0], probes_q[0], budget_s=15.0)
        base["sample"] = "member 0 of the ensemble: " + base["sample"]
    M = 1
    while M < 4 * lbm_steps:
        M *= 2
    launches = args.steps * (lbm_steps + len(specs) * (2 + int(math.log2(M)) + 5))
    line = {
        "metric": "MLUPS", "value": value, "unit": "MLUPS", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": my_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": {W.PREC_F64: "f64", W.PREC_F32: "f32", W.PREC_F16S: "f16 storage / f32 math",
                  W.PREC_BF16S: "bf16 storage / f32 math"}[prec], "data": "synthetic",
        "config": {"workload": f"ensemble of {len(specs)} seeded trumpets (r, theta in [32, 96], "
                               f"z in [128, 512]), {lbm_steps} time steps + per-member spectrum "
                               "per step, 8 probes per member",
                   "nodes": nodes, "time_steps_per_step": lbm_steps, "shape": tune_report,
                   "l2": f"working set {2 * 7 * nodes * elem / 1e9:.1f} GB vs 129 MB L2",
                   "parallelism": f"replicas x{ws}"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak,
                     "traffic": profiled_ensemble_traffic(nodes) if prec == W.PREC_F32 else None,
                     "kernel": "ensemble step kernel",
                     "peak_source": peak_kind, "bytes_per_node": 14 * elem,
                     "kernel_us": kernel_ms * 1e3},
        "cpu_baseline": base,
        "e2e": {"value": e2e_value, "unit": "MLUPS", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        "clocks": clk.summary(),
        "gpu_launches": launches,
    }
    if sequential is not None:
        line["vs_sequential"] = sequential
    if args.surrogate > 0:
        line["surrogate"] = surrogate_report(specs, args.surrogate)
    print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()
    return 0


def surrogate_report(specs, steps):
    """Mode targets of every member from the batched LBM (steps time steps), 4-layer 256-wide
    MLPs trained on the first 80% of the members (device kernels, FP32, cosine-decayed Adam),
    BF16-weight inference on the rest: one network for the lowest 8 mode frequencies, and one
    network per mode.  Reports the held-out mean relative error per mode, how many of the
    lowest modes the per-mode networks give within 0.5 %, the error of predicting the training
    mean, and the per-geometry time of the LBM and of the surrogate."""
    from paper_1705_01801_gb300 import surrogate as S
    freqs, valid, lbm_s = S.measure(specs, steps=steps, tune=True)
    X = np.stack([S.features(s) for s in specs])[valid]
    Y = freqs[valid]
    ntr = int(0.8 * len(X))
    out = {"members": len(specs), "valid": int(valid.sum()), "time_steps": steps,
           "held_out": int(len(X) - ntr), "training_steps": 20000}
    for name, per_mode in (("joint", False), ("per_mode", True)):
        sur = S.Surrogate(hidden=256, depth=4, seed=0, per_mode=per_mode)
        t0 = time.perf_counter()
        sur.fit(X[:ntr], Y[:ntr], steps=20000, batch=32, lr=1e-3)
        train_s = time.perf_counter() - t0
        t0 = time.perf_counter()
        pred = sur.predict(X[ntr:])
        sur_s = time.perf_counter() - t0
        err = np.abs(pred - Y[ntr:]) / Y[ntr:]
        per = err.mean(0)
        within = int(np.argmax(np.append(per, 1.0) > 0.005))
        out[name] = {"mean_rel_err": float(err.mean()),
                     "mean_rel_err_per_mode": [round(float(x), 4) for x in per],
                     "lowest_modes_within_0.5pct": within, "train_s": train_s,
                     "surrogate_s_per_geometry": sur_s / max(1, len(X) - ntr),
                     "speedup": (lbm_s / len(specs)) / (sur_s / max(1, len(X) - ntr))}
    base = np.abs(np.exp(np.log(Y[:ntr]).mean(0)) - Y[ntr:]) / Y[ntr:]
    out["mean_predictor_rel_err"] = float(base.mean())
    out["lbm_s_per_geometry"] = lbm_s / len(specs)
    return out


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    if WORKLOAD == "ensemble":  # the oracle advances one member at a time: member 0
        prec = PREC_OVERRIDE if PREC_OVERRIDE is not None else W.PREC_F32
        spec = W.ensemble(args.members, seed=5, prec=prec)[0][0]
        pulses_, probes_ = W.ensemble_excitation(spec)
        label = f"ensemble member 0 ({args.members} seeded trumpets)"
    else:
        wl = workload()
        spec, pulses_, probes_ = wl.spec, wl.pulses, wl.probes
        label = WORKLOAD
    import oracle
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    g = oracle.OracleGrid(spec)
    g.init(pulses_)
    g.set_probes(probes_, 1 << 16)
    g.step(1)
    t0 = time.perf_counter()
    g.step(1)
    t1 = time.perf_counter() - t0
    per_step = max(1, int(8.0 / max(t1, 1e-6)))  # ~8 s of host work per benchmark step
    for _ in range(args.warmup):
        g.step(1)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        g.step(per_step)
        times.append(time.perf_counter() - t0)
    total = sum(times)
    mlups = spec.nodes * per_step * args.steps / total / 1e6
    line = {
        "impl": "reference", "metric": "MLUPS", "value": mlups, "unit": "MLUPS", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": f"{label} {spec.n[0]}x{spec.n[1]}x{spec.n[2]}, "
                               f"{per_step} time steps per benchmark step (bounded sample)",
                   "nodes": spec.nodes},
        "cpu_baseline": {"value": mlups, "unit": "MLUPS", "cores": cores, "kind": "oracle",
                         "sample": f"{per_step} time steps of the full lattice per step"},
        "e2e": {"value": mlups, "unit": "MLUPS", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--lbm-steps", type=int, default=None,
                    help="time steps per benchmark step (default: 2000 for the torus, the "
                         "workload's full length otherwise, 512 for the ensemble)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", default="torus",
                    choices=["cylinder", "disk", "trumpet", "torus", "ensemble"])
    ap.add_argument("--members", type=int, default=512,
                    help="ensemble members (--workload ensemble)")
    ap.add_argument("--surrogate", type=int, default=0, metavar="T",
                    help="ensemble: measure every member's spectrum over T time steps, train the "
                         "MLP surrogate on 80%% of the members and report its held-out error and "
                         "speed against the ensemble run")
    ap.add_argument("--vs-sequential", type=int, default=0, metavar="M",
                    help="ensemble: also time the first M members advanced one after another as "
                         "single lattices (the plain path) and report both rates")
    ap.add_argument("--vs-f64", action="store_true",
                    help="after the timed region, rerun the workload with FP64 storage on the "
                         "GPU and report the field and mode-frequency deviations")
    ap.add_argument("--prec", default=None, choices=["f64", "f32", "f16s", "bf16s"],
                    help="storage override (default: the workload's own)")
    ap.add_argument("--shape", default=None, metavar="N1,N2,N3",
                    help="resize the workload's lattice (smaller profiling captures)")
    ap.add_argument("--launch", default=None, metavar="ROWS,PLANES,CTAS",
                    help="ensemble: this launch shape (lbw_batch_set_shape; rows 0 = full-row "
                         "tiles) instead of the autotuner's")
    ap.add_argument("--geom", default="auto", choices=["auto", "table", "analytic"],
                    help="geometry source of the step kernel (lbw_geom_mode)")
    args = ap.parse_args()
    global WORKLOAD, PREC_OVERRIDE, SHAPE, GEOM_MODE
    WORKLOAD = args.workload
    if args.shape:
        SHAPE = tuple(int(v) for v in args.shape.split(","))
    GEOM_MODE = {"auto": W.GEOM_AUTO, "table": W.GEOM_TABLE, "analytic": W.GEOM_ANALYTIC}[args.geom]
    if args.prec:
        PREC_OVERRIDE = {"f64": W.PREC_F64, "f32": W.PREC_F32, "f16s": W.PREC_F16S,
                         "bf16s": W.PREC_BF16S}[args.prec]
    if args.impl == "reference":
        return run_reference(args)
    if WORKLOAD == "ensemble":
        return run_ensemble(args)

    import torch
    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_1705_01801_gb300 import lbw

    wl = workload()
    spec = wl.spec
    lbm_steps = args.lbm_steps if args.lbm_steps is not None else BENCH_TIME_STEPS.get(WORKLOAD, wl.steps)
    stream = torch.cuda.Stream()
    sh = lbw.ctypes.c_void_p(stream.cuda_stream)
    grid = lbw.Grid(spec, stream=sh)
    nprobe = wl.probes.shape[0]

    def device_step(timed_events=None):
        # initial state rebuilt outside the timed region; probes restarted
        grid.init(wl.pulses)
        grid.set_probes(wl.probes, lbm_steps)
        stream.synchronize()
        ev0, ev1, ev2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        ev0.record(stream)
        grid.step(lbm_steps)
        ev1.record(stream)
        f, a = grid.spectrum(-1, 8)
        ev2.record(stream)
        ev2.synchronize()
        return ev0.elapsed_time(ev2), ev0.elapsed_time(ev1), f

    def barrier():
        if ws > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    # ---- device-timed value
    for _ in range(args.warmup):
        device_step()
    gpu_index = local
    if os.environ.get("CUDA_VISIBLE_DEVICES"):
        try:
            gpu_index = int(os.environ["CUDA_VISIBLE_DEVICES"].split(",")[local])
        except ValueError:
            pass
    barrier()
    tot_ms, step_ms, freqs = [], [], None
    with ClockSampler(gpu_index) as clk:
        for _ in range(args.steps):
            t, s, freqs = device_step()
            tot_ms.append(t)
            step_ms.append(s)
    barrier()
    my_ms = max_over_ranks(sum(tot_ms), device="cuda")
    value = whole_job_mlups(spec.nodes, lbm_steps * args.steps, ws, my_ms / 1e3)

    # ---- roofline of the fused step kernel (algorithmic bytes: 7 loads + 7 stores)
    elem = {W.PREC_F64: 8, W.PREC_F32: 4, W.PREC_F16S: 2, W.PREC_BF16S: 2}[spec.prec]
    bytes_per_node = 14 * elem
    kernel_ms = sum(step_ms) / (args.steps * lbm_steps)
    achieved = spec.nodes * bytes_per_node / (kernel_ms / 1e3) / 1e9
    peak, peak_kind = _peaks()
    traffic = profiled_traffic(WORKLOAD, spec) if SHAPE is None and GEOM_MODE != W.GEOM_ANALYTIC else None

    # ---- end to end through the C ABI with host buffers
    host_pulses = np.ascontiguousarray(wl.pulses)
    host_probes = np.ascontiguousarray(wl.probes.astype(np.int32))
    L = lbw.lib()

    def e2e_step():
        lbw.lbw_init(grid.handle, host_pulses)
        lbw.lbw_probe(grid.handle, host_probes, lbm_steps)
        lbw.lbw_step(grid.handle, lbm_steps)
        series = lbw.lbw_probe_read(grid.handle, nprobe, lbm_steps)
        f, a = lbw.lbw_spectrum(grid.handle, -1, 8)
        return series, f

    for _ in range(max(1, args.warmup // 2)):
        e2e_step()
    barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        series, _ = e2e_step()
    torch.cuda.synchronize()
    e2e_s = max_over_ranks(time.perf_counter() - t0, device="cuda")
    e2e_value = whole_job_mlups(spec.nodes, lbm_steps * args.steps, ws, e2e_s)
    h2d = host_pulses.nbytes + host_probes.nbytes
    d2h = nprobe * lbm_steps * 8 + 8 * 8 * 2

    # kernel launches of this library inside the timed region: per step the fused kernels
    # plus the spectrum (stats, window, log2 M Stockham passes, power, max, candidates,
    # select, refine)
    M = 1
    while M < 4 * lbm_steps:
        M *= 2
    spectrum_launches = 2 + int(math.log2(M)) + 5
    launches = args.steps * (lbm_steps + spectrum_launches)

    accuracy = None
    if args.vs_f64 and rank == 0:
        accuracy = f64_deviation(lbw, wl, lbm_steps, grid, sh)
    if rank != 0:
        if ws > 1:
            torch.distributed.destroy_process_group()
        return 0
    base = None
    if not args.no_cpu_baseline and ws == 1:
        base = cpu_baseline(spec, wl.pulses, wl.probes)
    line = {
        "metric": "MLUPS", "value": value, "unit": "MLUPS", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": my_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": {W.PREC_F64: "f64", W.PREC_F32: "f32", W.PREC_F16S: "f16 storage / f32 math",
                  W.PREC_BF16S: "bf16 storage / f32 math"}[spec.prec], "data": "synthetic",
        "config": {"workload": f"{wl.notes}, {spec.nodes:,} nodes, {lbm_steps} time steps + "
                               f"spectrum per step, {nprobe} probes, {pulse_label(wl)}",
                   "nodes": spec.nodes, "time_steps_per_step": lbm_steps, "c": spec.c,
                   "r_in": spec.x0[0],
                   "geometry": ["auto (table)", "table", "analytic"][spec.geom_mode],
                   "l2": l2_note(2 * 7 * spec.nodes * elem),
                   "parallelism": f"replicas x{ws}"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic,
                     "kernel": "fused step kernel", "peak_source": peak_kind,
                     "bytes_per_node": bytes_per_node, "kernel_us": kernel_ms * 1e3},
        "cpu_baseline": base,
        "e2e": {"value": e2e_value, "unit": "MLUPS", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        "clocks": clk.summary(),
        "gpu_launches": launches,
        "spectrum_peaks": [round(float(x), 6) for x in freqs] if freqs is not None else None,
    }
    if accuracy is not None:
        line["vs_f64"] = accuracy
    print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()
    return 0


def f64_deviation(lbw, wl, lbm_steps, grid, stream_handle, k=8):
    """The same run with FP64 storage and arithmetic on the GPU (the FP64 kernels match the FP64
    oracle to 1e-11 on the parity grids) as the reference at full size: relative L2 of the
    final P field, and for each of the k strongest spectral peaks (rad / step) of the FP64
    run's summed probes the relative deviation of the nearest of the 2k strongest peaks of
    this run (the error of each mode's frequency, whatever the ranking of nearly equal peaks)."""
    spec64 = wl.spec.with_(prec=W.PREC_F64)
    ref = lbw.Grid(spec64, stream=stream_handle)
    out = {}
    try:
        runs = []
        for g, kk in ((grid, 2 * k), (ref, k)):
            g.init(wl.pulses)
            g.set_probes(wl.probes, lbm_steps)
            g.step(lbm_steps)
            f, _ = g.spectrum(-1, kk)
            runs.append((np.sort(np.asarray(f)), g.get_P()))
        (fa, Pa), (fb, Pb) = runs
        out["field_rel_l2"] = float(np.linalg.norm(Pa - Pb) / np.linalg.norm(Pb))
        if len(fa) and len(fb):
            dev = np.array([np.min(np.abs(fa - x)) / x for x in fb])
            out["mode_freq_max_rel"] = float(dev.max())
            out["mode_freq_rel"] = [float(f"{x:.2e}") for x in dev]
        out["modes_compared"] = int(len(fb))
        out["peaks_f64"] = [round(float(x), 7) for x in fb]
        out["time_steps"] = lbm_steps
    finally:
        ref.close()
    return out


PROFILES = {
    ("torus", W.PREC_F32): os.path.join(ROOT, "profiles", "step_tma_kernel_torus_192x1024x256_f32.md"),
    ("cylinder", W.PREC_F32): os.path.join(ROOT, "profiles", "step_tma_kernel_cylinder_128x128x256_f32.md"),
}
ENSEMBLE_PROFILE = os.path.join(ROOT, "profiles", "batch_row_kernel_ensemble_32_trumpets_f32.md")


def source_hash(name):
    import hashlib
    p = os.path.join(ROOT, "paper_1705_01801_gb300", "csrc", name)
    with open(p, "rb") as fh:
        return hashlib.sha256(fh.read()).hexdigest()[:16]


def lbw_kernel_hash():
    return source_hash("lbw_step.cu")


def _profile_fields(path):
    fields = {}
    with open(path) as fh:
        for line in fh:
            if ":" in line and not line.startswith(("#", "|", " ")):
                k, v = line.split(":", 1)
                fields[k.strip()] = v.strip()
    return fields


def pulse_label(wl):
    """What the initial field is, from the workload's own pulse list."""
    n = len(wl.pulses)
    phased = bool(np.any(np.abs(wl.pulses[:, 4]) != 1.0))
    kind = "random-phase " if phased else ""
    return f"{n} {kind}Gaussian pulse{'s' if n != 1 else ''} (sigma {wl.pulses[0, 3]:g} cells)"


def l2_note(working_set_bytes):
    """Working set against the 129 MB L2: the benchmark does not flush L2 between steps, which
    is valid only when the population buffers do not fit in it."""
    ratio = working_set_bytes / 129e6
    if ratio >= 4.0:
        return (f"working set {working_set_bytes / 1e6:.0f} MB = {ratio:.1f}x the 129 MB L2 "
                "(no flush between steps)")
    return (f"working set {working_set_bytes / 1e6:.0f} MB = only {ratio:.1f}x the 129 MB L2: "
            "part of it stays L2-resident between time steps")


def profiled_traffic(workload_name, spec):
    """DRAM bytes per launch of the step kernel from the committed ncu summary of this workload
    and storage, or None when there is none or the kernel source changed since the counters
    were taken."""
    try:
        fields = _profile_fields(PROFILES[(workload_name, spec.prec)])
        if fields.get("step_source_sha256_16") != lbw_kernel_hash():
            return None
        return int(fields["traffic_bytes_per_launch"])
    except Exception:
        return None


def profiled_ensemble_traffic(nodes):
    """DRAM bytes per launch of the FP32 ensemble kernel: the committed ncu summary's bytes per
    node (a 32-member capture of the same member distribution) times the ensemble's nodes, or
    None when the ensemble source changed since the counters were taken."""
    try:
        fields = _profile_fields(ENSEMBLE_PROFILE)
        if fields.get("batch_source_sha256_16") != source_hash("lbw_batch.cu"):
            return None
        return int(round(float(fields["traffic_bytes_per_node"]) * nodes))
    except Exception:
        return None


if __name__ == "__main__":
    sys.exit(main())
