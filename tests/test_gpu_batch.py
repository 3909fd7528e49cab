"""Ensembles of uneven lattices advanced by the persistent batched kernel, against the FP64
oracle member by member, plus the autotuner and its cache."""
import numpy as np
import pytest

import oracle
from lbw_workloads import PREC_BF16S, PREC_F16S, PREC_F32, PREC_F64, ensemble, ensemble_excitation

pytestmark = pytest.mark.gpu


def _small_ensemble(prec, n=5):
    # uneven sizes (q2 extents not multiples of 32, ragged q1 tiles), short enough for the oracle
    specs, _ = ensemble(n, seed=11, r_range=(9, 21), theta_range=(33, 70), z_range=(18, 40),
                        prec=prec)
    return specs


@pytest.mark.parametrize("prec,tol", [(PREC_F64, 1e-11), (PREC_F32, 2e-5)], ids=["f64", "f32"])
def test_members_match_oracle(prec, tol):
    from paper_1705_01801_gb300 import lbw
    specs = _small_ensemble(prec)
    exc = [ensemble_excitation(s, sigma=2.5) for s in specs]
    b = lbw.Batch(specs)
    b.init([e[0] for e in exc])
    b.set_probes(np.stack([e[1] for e in exc]), 150)
    b.step(150)
    series = b.read_probes()
    for m, s in enumerate(specs):
        o = oracle.OracleGrid(s)
        o.init(exc[m][0])
        o.set_probes(exc[m][1], 150)
        o.step(150)
        fo = o.get_f()
        np.testing.assert_allclose(b.get_f(m), fo, rtol=0, atol=tol * np.abs(fo).max())
        so = o.read_probes()
        np.testing.assert_allclose(series[m], so, rtol=0, atol=tol * 10 * np.abs(so).max())


def test_member_equals_single_lattice_run():
    """A member and the same lattice run alone (possibly by another kernel, in another
    rounding order) agree to FP32 rounding."""
    from paper_1705_01801_gb300 import lbw
    specs = _small_ensemble(PREC_F32, n=3)
    exc = [ensemble_excitation(s, sigma=2.5) for s in specs]
    b = lbw.Batch(specs)
    b.init([e[0] for e in exc])
    b.step(70)
    for m, s in enumerate(specs):
        g = lbw.Grid(s)
        g.init(exc[m][0])
        g.step(70)
        fg = g.get_f()
        np.testing.assert_allclose(b.get_f(m), fg, rtol=0, atol=2e-5 * np.abs(fg).max())


def test_member_spectra_match_oracle_estimator():
    from paper_1705_01801_gb300 import lbw
    specs = _small_ensemble(PREC_F64, n=3)
    exc = [ensemble_excitation(s, sigma=2.5) for s in specs]
    b = lbw.Batch(specs)
    b.init([e[0] for e in exc])
    b.set_probes(np.stack([e[1] for e in exc]), 1500)
    b.step(1500)
    f, a, cnt = b.spectrum(4)
    for m, s in enumerate(specs):
        o = oracle.OracleGrid(s)
        o.init(exc[m][0])
        o.set_probes(exc[m][1], 1500)
        o.step(1500)
        fo, _ = oracle.spectrum(o.read_probes().sum(0), 4)
        assert cnt[m] == len(fo)
        np.testing.assert_allclose(f[m, : cnt[m]], fo, rtol=1e-8)


def test_autotuner_chooses_and_caches(tmp_path):
    from paper_1705_01801_gb300 import lbw
    specs = _small_ensemble(PREC_F32, n=4)
    cache = str(tmp_path / "tune.jsonl")
    b = lbw.Batch(specs)
    rep = b.tune(trial_steps=2, cache_path=cache)
    assert "chosen" in rep and rep.count("ms=") >= 9
    shape = b.info()
    b2 = lbw.Batch(specs)
    rep2 = b2.tune(trial_steps=2, cache_path=cache)
    assert "cached" in rep2 and b2.info() == shape
    # a tuned ensemble still computes the same numbers
    exc = [ensemble_excitation(s, sigma=2.5) for s in specs]
    b.init([e[0] for e in exc])
    b.step(20)
    o = oracle.OracleGrid(specs[0])
    o.init(exc[0][0])
    o.step(20)
    fo = o.get_f()
    np.testing.assert_allclose(b.get_f(0), fo, rtol=0, atol=2e-5 * np.abs(fo).max())


def _edge_members(prec):
    """Members that exercise the padded tile kernel's edges: q2 extents below, at and above
    one 64-column tile (ragged and odd ones included, so the periodic wrap runs through the
    ghost columns), and q1 extents with (n1 - 1) a multiple of 4 or 7 (tiles shifted to start
    at q1 = -1 so no halo row sits on a face)."""
    from lbw_workloads import ensemble_member, trumpet_params
    sizes = [(8, 33, 20), (9, 64, 18), (15, 100, 22), (29, 47, 19), (22, 128, 17)]
    out = []
    for k, (n1, n2, n3) in enumerate(sizes):
        a0, b_, al = trumpet_params(100 + k, n1, n3)
        out.append(ensemble_member(n1, n2, n3, a0, b_, al, prec=prec))
    return out


@pytest.mark.parametrize("prec,tol", [(PREC_F64, 1e-11), (PREC_F32, 2e-5)], ids=["f64", "f32"])
def test_edge_shapes_match_oracle(prec, tol):
    from paper_1705_01801_gb300 import lbw
    specs = _edge_members(prec)
    exc = [ensemble_excitation(s, sigma=2.5) for s in specs]
    b = lbw.Batch(specs)
    b.init([e[0] for e in exc])
    b.set_probes(np.stack([e[1] for e in exc]), 120)
    b.step(120)
    series = b.read_probes()
    for m, s in enumerate(specs):
        o = oracle.OracleGrid(s)
        o.init(exc[m][0])
        o.set_probes(exc[m][1], 120)
        o.step(120)
        fo = o.get_f()
        np.testing.assert_allclose(b.get_f(m), fo, rtol=0, atol=tol * np.abs(fo).max())
        so = o.read_probes()
        np.testing.assert_allclose(series[m], so, rtol=0, atol=tol * 10 * np.abs(so).max())


@pytest.mark.parametrize("prec,unit", [(PREC_F16S, 2.0 ** -11), (PREC_BF16S, 2.0 ** -8)],
                         ids=["f16", "bf16"])
def test_sixteen_bit_members_error_bound(prec, unit):
    """16-bit storage in the ensemble: field error against the FP64 oracle within 3 u sqrt(S),
    the bound the single-lattice precision tests use."""
    import math
    from paper_1705_01801_gb300 import lbw
    specs = _edge_members(prec)
    exc = [ensemble_excitation(s, sigma=2.5) for s in specs]
    b = lbw.Batch(specs)
    b.init([e[0] for e in exc])
    steps = 200
    b.step(steps)
    for m, s in enumerate(specs):
        o = oracle.OracleGrid(s)
        o.init(exc[m][0])
        o.step(steps)
        fo, fg = o.get_f(), b.get_f(m)
        rel = np.linalg.norm(fg - fo) / np.linalg.norm(fo)
        assert rel <= 3 * unit * math.sqrt(steps), (m, rel)


def test_lowest_peaks_match_oracle_estimator():
    """lbw_batch_spectrum_lowest against the oracle estimator's lowest-frequency selection."""
    from paper_1705_01801_gb300 import lbw
    specs = _small_ensemble(PREC_F64, n=3)
    exc = [ensemble_excitation(s, sigma=2.5) for s in specs]
    b = lbw.Batch(specs)
    b.init([e[0] for e in exc])
    b.set_probes(np.stack([e[1] for e in exc]), 1500)
    b.step(1500)
    f, a, cnt = b.spectrum(5, lowest=True, rel_power=1e-2)
    for m, s in enumerate(specs):
        o = oracle.OracleGrid(s)
        o.init(exc[m][0])
        o.set_probes(exc[m][1], 1500)
        o.step(1500)
        fo, _ = oracle.spectrum(o.read_probes().sum(0), 5, thresh=1e-2, lowest=True)
        assert cnt[m] == len(fo)
        np.testing.assert_allclose(f[m, : cnt[m]], fo, rtol=1e-8)


def _row_members(prec):
    """Members for full-row tiles: odd and even q2 extents (an odd one ends each row with a
    phantom node), a narrow row (tiles of 16 rows), a q1 extent whose tiles start at q1 = -1
    ((n1 - 1) a multiple of the 7 rows of a 64-wide row) and a 100-wide row (3-row tiles)."""
    from lbw_workloads import ensemble_member, trumpet_params
    sizes = [(8, 33, 20), (15, 64, 18), (15, 100, 22), (29, 47, 19), (13, 10, 9), (22, 95, 17)]
    seeds = [200, 201, 202, 203, 204, 305]  # flares the library accepts at c = 0.4
    return [ensemble_member(n1, n2, n3, *trumpet_params(sd, n1, n3), prec=prec)
            for (n1, n2, n3), sd in zip(sizes, seeds)]


def _ensemble_vs_oracle(b, specs, exc, steps, tol):
    series = b.read_probes()
    for m, s in enumerate(specs):
        o = oracle.OracleGrid(s)
        o.init(exc[m][0])
        o.set_probes(exc[m][1], steps)
        o.step(steps)
        fo = o.get_f()
        np.testing.assert_allclose(b.get_f(m), fo, rtol=0, atol=tol * np.abs(fo).max())
        so = o.read_probes()
        np.testing.assert_allclose(series[m], so, rtol=0, atol=tol * 10 * np.abs(so).max())


@pytest.mark.parametrize("prec,tol", [(PREC_F64, 1e-11), (PREC_F32, 2e-5)], ids=["f64", "f32"])
def test_full_row_tiles_match_oracle(prec, tol):
    """The full-row ensemble kernel (tile_rows 0: whole rows per tile, the q2 wrap inside
    the tile) against the oracle member by member, 120 steps, several q3 segments."""
    from paper_1705_01801_gb300 import lbw
    specs = _row_members(prec)
    exc = [ensemble_excitation(s, sigma=2.5) for s in specs]
    b = lbw.Batch(specs)
    try:
        b.set_shape(0, 8, 2 if prec == PREC_F32 else 1)  # FP64 tiles fill the shared memory of an SM
        assert b.info()["tile_rows"] == 0
        b.init([e[0] for e in exc])
        b.set_probes(np.stack([e[1] for e in exc]), 120)
        b.step(120)
        _ensemble_vs_oracle(b, specs, exc, 120, tol)
    finally:
        b.close()


def test_shape_switch_mid_run_keeps_the_run():
    """60 steps on full-row tiles, then 60 on 64-column tiles (which read the ghost columns the
    full-row kernel does not keep; the switch rebuilds them): the same run as the oracle's."""
    from paper_1705_01801_gb300 import lbw
    specs = _row_members(PREC_F64)
    exc = [ensemble_excitation(s, sigma=2.5) for s in specs]
    b = lbw.Batch(specs)
    try:
        b.set_shape(0, 16, 1)
        b.init([e[0] for e in exc])
        b.set_probes(np.stack([e[1] for e in exc]), 120)
        b.step(60)
        b.set_shape(7, 32, 1)
        b.step(60)
        _ensemble_vs_oracle(b, specs, exc, 120, 1e-11)
    finally:
        b.close()


def test_set_shape_rejects_what_the_ensemble_cannot_run():
    from paper_1705_01801_gb300 import lbw
    from lbw_workloads import ensemble_member, trumpet_params
    wide = [ensemble_member(12, 128, 10, *trumpet_params(5, 12, 10), prec=PREC_F32)]  # 2-row tiles only
    b = lbw.Batch(wide)
    try:
        for shape in ((0, 16, 2), (5, 16, 2), (7, 0, 2), (7, 16, 0), (7, 16, 64)):
            with pytest.raises(lbw.LbwError) as e:
                b.set_shape(*shape)
            assert e.value.status == lbw.LBW_EINVAL
        b.set_shape(4, 16, 1)
        assert b.info()["tile_rows"] == 4
    finally:
        b.close()
