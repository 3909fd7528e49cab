"""The no-allocation spectrum entry point against the allocating one.

lbw_spectrum_series_static serves callers that must not allocate device memory: its workspace
is a fixed array inside the library.  The test hands it series that already sit in device
memory and compares its peaks with lbw_spectrum_series on the same data, on two calls in a
row (the fixed workspace keeps the previous call's contents), within the tolerances of the
other spectrum tests (1e-8 relative in frequency, 1e-7 in amplitude).
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _series(T, seed):
    rng = np.random.default_rng(seed)
    t = np.arange(T)
    om = rng.uniform(0.01, 0.3, 3)
    return (np.cos(om[0] * t + 0.2) + 0.5 * np.cos(om[1] * t + 1.0) + 0.25 * np.cos(om[2] * t)
            + 0.01 * rng.standard_normal(T))


def test_static_workspace_spectrum_matches_allocating_entry_point():
    import torch
    from paper_1705_01801_gb300 import lbw
    k = 4
    for call, T in enumerate((6000, 16384)):  # two calls in a row, the second at the maximum T
        x = _series(T, 100 + call)
        d_x = torch.tensor(x, dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        fs, as_ = lbw.lbw_spectrum_series_static(d_x.data_ptr(), T, k)
        (fr, ar), = lbw.lbw_spectrum_series(x, k)
        assert len(fs) == len(fr) > 0
        np.testing.assert_allclose(fs, fr, rtol=1e-8)
        np.testing.assert_allclose(as_, ar, rtol=1e-7)


def test_static_workspace_rejects_series_beyond_its_size():
    import torch
    from paper_1705_01801_gb300 import lbw
    d_x = torch.zeros(16385, dtype=torch.float64, device="cuda")
    with pytest.raises(lbw.LbwError) as e:
        lbw.lbw_spectrum_series_static(d_x.data_ptr(), 16385, 4)
    assert e.value.status == lbw.LBW_EINVAL and "16384" in str(e.value)
