"""Ensembles of uneven lattices advanced by the persistent batched kernel, against the FP64
oracle member by member, plus the autotuner and its cache."""
import numpy as np
import pytest

import oracle
from lbw_workloads import PREC_F32, PREC_F64, ensemble, ensemble_excitation

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
    """Same register-pipelined per-node code: a member and the same lattice run alone agree
    to FP32 rounding."""
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
        np.testing.assert_allclose(b.get_f(m), fg, rtol=0, atol=1e-6 * np.abs(fg).max())


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
