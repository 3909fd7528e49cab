"""Parity at the benchmark workloads' full sizes, in the launch configuration the benchmark
times: the 256 x 256 x 512 trumpet (FP32 and FP16 storage) and the 192 x 1024 x 256 torus
(FP32 and BF16 storage), one device step from a shared state against one FP64 oracle step at
every node; the 512-trumpet ensemble on sampled members; the 128 x 128 disk over its full
4000 steps; a 512 x 1024 x 768 cylinder, whose 2.8e9 populations per buffer pass 2^31, in its
far corner against a small oracle lattice over that corner."""
import numpy as np
import pytest

import lbw_workloads as W
import oracle

pytestmark = pytest.mark.gpu

W_D3Q7 = np.array([0.25] + [0.125] * 6)  # weights at cs^2 = 1/4


def _shared_state(spec, seed):
    """Random populations (7, N3, N1, N2) that the storage type holds exactly: FP32 values,
    or w_i h_i with h_i = k / 64, |k| <= 64, for the 16-bit forms (they store h_i = f_i / w_i;
    k / 64 needs at most 7 significand bits)."""
    rng = np.random.default_rng(seed)
    shape = (7, spec.n[2], spec.n[0], spec.n[1])
    if spec.prec == W.PREC_F32:
        return rng.standard_normal(shape, dtype=np.float32).astype(np.float64)
    h = rng.integers(-64, 65, size=shape).astype(np.float64) / 64.0
    return h * W_D3Q7[:, None, None, None]


# storage rounding of one step's result: half an ulp of FP32 (with the FP32 arithmetic),
# FP16 (11 significand bits) and BF16 (8)
RTOL = {W.PREC_F32: 0.0, W.PREC_F16S: 2.0 ** -11, W.PREC_BF16S: 2.0 ** -8}


@pytest.mark.parametrize("name,prec", [("trumpet", W.PREC_F32), ("trumpet", W.PREC_F16S),
                                       ("torus", W.PREC_F32), ("torus", W.PREC_BF16S)],
                         ids=["trumpet-f32", "trumpet-f16", "torus-f32", "torus-bf16"])
def test_one_step_full_size(name, prec):
    from paper_1705_01801_gb300 import lbw
    spec = {"trumpet": W.trumpet, "torus": W.torus}[name](prec=prec)
    f = _shared_state(spec, seed=11)
    g = lbw.Grid(spec)
    try:
        g.set_f(f)
        g.step(1)
        fg = g.get_f()
    finally:
        g.close()
    o = oracle.OracleGrid(spec)
    o.set_f(f)
    del f
    o.step(1)
    fo = o.get_f()
    o.close()
    scale = np.abs(fo).max()
    np.testing.assert_allclose(fg, fo, rtol=RTOL[prec], atol=1e-6 * scale)


def test_ensemble_full_size_sampled_members():
    """The 512-trumpet ensemble with the autotuned launch shape, three steps from the
    benchmark's excitation; members 0, 255 and 511 against the oracle run of each member."""
    from paper_1705_01801_gb300 import lbw
    specs, _ = W.ensemble(512, seed=5)
    exc = [W.ensemble_excitation(s) for s in specs]
    b = lbw.Batch(specs)
    try:
        b.tune(trial_steps=2)
        b.init([e[0] for e in exc])
        b.step(3)
        got = {m: b.get_f(m) for m in (0, 255, 511)}
    finally:
        b.close()
    for m, fg in got.items():
        o = oracle.OracleGrid(specs[m])
        o.init(exc[m][0])
        o.step(3)
        fo = o.get_f()
        o.close()
        np.testing.assert_allclose(fg, fo, rtol=0, atol=2e-5 * np.abs(fo).max())


def test_disk_full_run_matches_oracle():
    """The 128 x 128 FP64 disk in full: 4000 steps from the benchmark's pulse, the four probe
    series within 1e-10 of their peak, the final populations within 1e-10 of the oracle's
    largest, and the spectrum of the summed probes equal to the oracle estimator's."""
    from paper_1705_01801_gb300 import lbw
    w = W.workload("disk")
    g = lbw.Grid(w.spec)
    o = oracle.OracleGrid(w.spec)
    try:
        for grid in (g, o):
            grid.init(w.pulses)
            grid.set_probes(w.probes, w.steps)
            grid.step(w.steps)
        xg, xo = g.read_probes(), o.read_probes()
        assert xg.shape == xo.shape == (len(w.probes), w.steps)
        assert np.abs(xg - xo).max() <= 1e-10 * np.abs(xo).max()
        fo = o.get_f()
        np.testing.assert_allclose(g.get_f(), fo, rtol=0, atol=1e-10 * np.abs(fo).max())
        fg_sum, _ = g.spectrum(-1, 4)
        fo_sum, _ = oracle.spectrum(xo.sum(0), 4)
        np.testing.assert_allclose(fg_sum, fo_sum, rtol=1e-8)
    finally:
        g.close()
        o.close()


@pytest.mark.parametrize("prec,tol", [(W.PREC_F32, 1e-5), (W.PREC_F64, 1e-11)], ids=["f32", "f64"])
def test_lattice_beyond_2_31_populations(prec, tol):
    """Index arithmetic past 2^31 populations (and past 2^32 bytes) per buffer: a 512 x 1024 x
    768 cylinder (402,653,184 nodes, 2,818,572,288 populations; 11.3 GB per FP32 buffer,
    22.5 GB in FP64) with two pulses in its far corner, one on the very last node (the last
    rows, columns and planes, where the offsets are largest), four steps.  The field a step moves spreads two cells at most,
    so the corner block of 44 rows x 1024 columns x 32 planes must equal an oracle lattice of
    that block (same radii and heights, same faces on the far sides; the pulse is below 1e-11
    at the block's near faces), and a probe in the very last node must record the same
    series."""
    from paper_1705_01801_gb300 import lbw
    spec = W.cylinder(n_r=512, n_theta=1024, n_z=768, prec=prec)
    r0, z0 = 468, 736
    assert 7 * spec.n[0] * spec.n[1] * spec.n[2] > 2 ** 31
    small = spec.with_(n=(spec.n[0] - r0, spec.n[1], spec.n[2] - z0), prec=W.PREC_F64,
                       x0=(spec.x0[0] + r0 * spec.h[0], spec.x0[1], spec.x0[2] + z0 * spec.h[2]))
    last = [spec.n[0] - 1, spec.n[1] - 1, spec.n[2] - 1]
    pl = [[*W.embedding(spec, *W.node_coords(spec, *q)), 3.0, a] for q, a in (([500, 1000, 758], 1.0), (last, -0.5))]
    near = [500, 1000, 760]
    steps = 4
    g = lbw.Grid(spec)
    try:
        g.init(pl)
        g.set_probes([last, near], steps)
        g.step(steps)
        P = g.get_P()[z0:, r0:, :].copy()
        series = g.read_probes()
    finally:
        g.close()
    o = oracle.OracleGrid(small)
    o.init(pl)
    o.set_probes([[q[0] - r0, q[1], q[2] - z0] for q in (last, near)], steps)
    o.step(steps)
    Po = o.get_P()
    so = o.read_probes()
    o.close()
    scale = np.abs(Po).max()
    assert scale > 0.05  # the pulse is inside the block
    np.testing.assert_allclose(P, Po, rtol=0, atol=tol * scale)
    np.testing.assert_allclose(series, so, rtol=0, atol=tol * np.abs(so).max())

