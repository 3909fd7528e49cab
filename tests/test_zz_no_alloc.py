"""The no-allocation spectrum entry point against the allocating one.

lbw_spectrum_series_static serves callers that must not allocate device memory: its workspace
is a fixed array inside the library.  The test hands it series that already sit in device
memory and compares its peaks with lbw_spectrum_series on the same data, on two calls in a
row (the fixed workspace keeps the previous call's contents), within the tolerances of the
other spectrum tests (1e-8 relative in frequency, 1e-7 in amplitude).  It also reads the
device's default stream-ordered memory pool (the pool the allocating entry points draw from)
around the fixed-workspace calls: they must not raise its high-water mark, while the
allocating call afterwards must, which shows that the measurement sees allocations.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

# CUmemPool_attribute values of the driver API (cuda.h)
_USED_MEM_CURRENT, _USED_MEM_HIGH = 7, 8


def _series(T, seed):
    rng = np.random.default_rng(seed)
    t = np.arange(T)
    om = rng.uniform(0.01, 0.3, 3)
    return (np.cos(om[0] * t + 0.2) + 0.5 * np.cos(om[1] * t + 1.0) + 0.25 * np.cos(om[2] * t)
            + 0.01 * rng.standard_normal(T))


class _DefaultPool:
    """High-water mark of the current device's default memory pool, through the driver API."""

    def __init__(self):
        import torch
        self.cu = ctypes.CDLL("libcuda.so.1")
        dev = ctypes.c_int(0)
        assert self.cu.cuDeviceGet(ctypes.byref(dev), torch.cuda.current_device()) == 0
        self.pool = ctypes.c_void_p()
        assert self.cu.cuDeviceGetDefaultMemPool(ctypes.byref(self.pool), dev) == 0

    def _get(self, attr):
        v = ctypes.c_uint64(0)
        assert self.cu.cuMemPoolGetAttribute(self.pool, attr, ctypes.byref(v)) == 0
        return v.value

    def reset_high(self):
        zero = ctypes.c_uint64(0)  # resets the high-water mark to the current use
        assert self.cu.cuMemPoolSetAttribute(self.pool, _USED_MEM_HIGH, ctypes.byref(zero)) == 0

    def used(self):
        return self._get(_USED_MEM_CURRENT)

    def high(self):
        return self._get(_USED_MEM_HIGH)


def test_static_workspace_spectrum_matches_allocating_entry_point():
    import torch
    from paper_1705_01801_gb300 import lbw
    k = 4
    pool = _DefaultPool()
    for call, T in enumerate((6000, 16384)):  # two calls in a row, the second at the maximum T
        x = _series(T, 100 + call)
        d_x = torch.tensor(x, dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        before = pool.used()
        pool.reset_high()
        fs, as_ = lbw.lbw_spectrum_series_static(d_x.data_ptr(), T, k)
        assert pool.high() <= before, "the fixed-workspace call allocated from the pool"
        pool.reset_high()
        (fr, ar), = lbw.lbw_spectrum_series(x, k)
        assert pool.high() > before, "the allocating call was not seen by the pool counter"
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
