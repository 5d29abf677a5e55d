"""The FP32 reciprocal of the step kernels (1/rho in u = j / rho, Eq. 22)
against the correctly rounded 1/x.

The kernels take the hardware reciprocal estimate r0 and one Newton-Raphson
step r1 = r0 + r0 (1 - x r0) with fused multiply-adds.  If x r0 = 1 - e,
the step's exact value is (1/x)(1 - e^2): with |e| near 2^-23 that is within
about 2^-46 of 1/x, so one rounding leaves r1 at most 1 ulp from the
correctly rounded result, and equal to it except where 1/x lies within
about 2^-46 (relative) of a rounding boundary.

The correctly rounded FP32 reference is 1/x in FP64 rounded to FP32: for a
24-bit x, 1/x is never within 2^-53 (relative) of an FP32 rounding
midpoint without being exactly on one (its distance from any 25-bit
number is a nonzero integer over 2^k x, at least about 2^-49 relative), so
the two roundings agree with one.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

MAX_ULP = 1   # the bound stated above


def _ulp_distance(a: np.ndarray, b: np.ndarray) -> np.ndarray:
    # same-sign finite floats: distance of their bit patterns
    ia = np.abs(a).view(np.int32).astype(np.int64)
    ib = np.abs(b).view(np.int32).astype(np.int64)
    assert np.array_equal(np.signbit(a), np.signbit(b))
    return np.abs(ia - ib)


def _device_recip(x: np.ndarray) -> np.ndarray:
    import torch
    import paper_1905_05110_gb300 as vp
    xd = torch.from_numpy(x).cuda()
    yd = torch.empty_like(xd)
    vp.vplbm_eval_recip_f32(xd.data_ptr(), yd.data_ptr(), x.size, torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    return yd.cpu().numpy()


def _check(x: np.ndarray):
    y = _device_recip(x)
    ref = (1.0 / x.astype(np.float64)).astype(np.float32)
    d = _ulp_distance(y, ref)
    return int(d.max()), float(np.mean(d == 0))


def test_recip_every_float_of_the_density_range(gpu_library):
    # every FP32 value in [0.5, 2): 2^24 inputs, the densities of the flows
    lo = np.array(0.5, dtype=np.float32).view(np.int32)
    hi = np.array(2.0, dtype=np.float32).view(np.int32)
    x = np.arange(lo, hi, dtype=np.int32).view(np.float32)
    assert x.size == 1 << 24
    worst, exact = _check(x)
    assert worst <= MAX_ULP
    assert exact > 0.999


def test_recip_log_spaced_wide_range_and_negatives(gpu_library):
    # normal inputs whose reciprocals are normal too (the reciprocal flushes
    # subnormals to zero), both signs, log-uniform over 2^-125 .. 2^125
    rng = np.random.default_rng(5)
    mag = np.exp2(rng.uniform(-125.0, 125.0, size=1 << 20)).astype(np.float32)
    sign = np.where(rng.random(mag.size) < 0.5, -1.0, 1.0).astype(np.float32)
    x = np.concatenate([mag * sign, np.float32(2.0) ** np.arange(-125, 126, dtype=np.float32)])
    worst, exact = _check(x)
    assert worst <= MAX_ULP
    assert exact > 0.999
    # powers of two are exact
    p2 = x[-251:]
    assert np.array_equal(_device_recip(p2), (1.0 / p2.astype(np.float64)).astype(np.float32))


def test_recip_rejects_bad_arguments(gpu_library):
    import torch
    import paper_1905_05110_gb300 as vp
    buf = torch.zeros(16, dtype=torch.float32, device="cuda")
    with pytest.raises(vp.VplbmError) as ei:
        vp.vplbm_eval_recip_f32(buf.data_ptr() + 2, buf.data_ptr(), 4)
    assert ei.value.status == 1
    with pytest.raises(vp.VplbmError):
        vp.vplbm_eval_recip_f32(0, buf.data_ptr(), 4)
    vp.vplbm_eval_recip_f32(0, 0, 0)   # nothing to do
