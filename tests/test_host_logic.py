"""Host-side helpers that need no GPU: the sweep's peak refinement, the surrogate's
geometry features, the ensemble excitation and the benchmark's profile bookkeeping."""
import math

import numpy as np
import pytest

import lbw_workloads as W


def test_peak_frequency_refines_a_sampled_resonance():
    from paper_1705_01801_gb300 import sweep
    w0, gamma = 0.0251, 0.0004
    omegas = np.linspace(0.8 * w0, 1.2 * w0, 41)
    resp = 1.0 / np.sqrt((omegas ** 2 - w0 ** 2) ** 2 + (gamma * omegas) ** 2)  # driven oscillator
    peak = sweep.peak_frequency(omegas, resp)
    step = omegas[1] - omegas[0]
    assert abs(peak - w0) < 0.1 * step
    # a maximum on the edge of the band is returned as is
    assert sweep.peak_frequency(omegas[:10], resp[:10]) == omegas[9]


def test_surrogate_features_of_a_member():
    from paper_1705_01801_gb300 import surrogate as S
    n_r, n_t, n_z = 40, 64, 256
    a0, b, al = W.trumpet_params(3, n_r, n_z)
    spec = W.ensemble_member(n_r, n_t, n_z, a0, b, al)
    f = S.features(spec)
    r_in = spec.x0[0]
    R = r_in + n_r
    assert f.shape == (len(S.FEATURE_NAMES),)
    assert f[0] == pytest.approx(R / 100.0)
    assert f[1] == pytest.approx(n_z / 512.0)
    assert f[2] == pytest.approx((a0 + b * math.exp(al * n_z)) / (a0 + b), rel=1e-6)
    assert f[4] == pytest.approx(n_t / 96.0)
    assert f[5] == pytest.approx(r_in / R)


def test_ensemble_excitation_is_axisymmetric_and_inside():
    specs, _ = W.ensemble(6, seed=4)
    for s in specs:
        pulses, probes = W.ensemble_excitation(s)
        assert pulses.shape == (12, 5)
        radii = np.hypot(pulses[:, 0], pulses[:, 1])
        assert np.ptp(radii) < 1e-9 * radii.max()  # one ring
        assert (probes >= 0).all() and (probes < np.array(s.n)).all()
        assert len({tuple(p[[0, 2]]) for p in probes}) == 1  # one corner ring of probes


def test_profiled_traffic_follows_the_kernel_source(monkeypatch):
    """bench.py reports ncu DRAM traffic only while the kernel source still hashes to the
    value recorded with the counters; the ensemble's bytes per node scale with its nodes."""
    import bench
    import lbw_workloads as W
    spec = W.workload("cylinder").spec
    step = bench._profile_fields(bench.PROFILES[("cylinder", W.PREC_F32)])
    ens = bench._profile_fields(bench.ENSEMBLE_PROFILE)
    real = {"lbw_step.cu": step["step_source_sha256_16"],
            "lbw_batch.cu": ens["batch_source_sha256_16"]}
    monkeypatch.setattr(bench, "source_hash", lambda name: real[name])
    assert bench.profiled_traffic("cylinder", spec) == int(step["traffic_bytes_per_launch"])
    assert bench.profiled_traffic("cylinder", spec.with_(prec=W.PREC_F16S)) is None
    assert bench.profiled_traffic("disk", W.workload("disk").spec) is None
    per_node = float(ens["traffic_bytes_per_node"])
    assert bench.profiled_ensemble_traffic(1000) == round(per_node * 1000)
    monkeypatch.setattr(bench, "source_hash", lambda name: "0" * 16)
    assert bench.profiled_traffic("cylinder", spec) is None
    assert bench.profiled_ensemble_traffic(1000) is None



def test_committed_profiles_match_the_kernel_sources():
    """The committed ncu summaries were taken on the kernel sources as they stand, so the
    benchmark lines of the torus (the headline), the cylinder and the ensemble carry measured
    DRAM traffic; a kernel edit without retaken counters fails here."""
    import bench
    import lbw_workloads as W
    for name in ("torus", "cylinder"):
        spec = W.workload(name).spec
        fields = bench._profile_fields(bench.PROFILES[(name, W.PREC_F32)])
        assert fields["step_source_sha256_16"] == bench.lbw_kernel_hash(), name
        traffic = bench.profiled_traffic(name, spec)
        assert traffic == int(fields["traffic_bytes_per_launch"])
        # within a few percent of the 56 B per node that one launch moves at least in part
        assert 0.75 < traffic / (56 * spec.nodes) < 1.1, (name, traffic)
    ens = bench._profile_fields(bench.ENSEMBLE_PROFILE)
    assert ens["batch_source_sha256_16"] == bench.source_hash("lbw_batch.cu")
