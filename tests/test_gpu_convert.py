"""The binary64 <-> binary32 conversions of the FP32-certified levels
(integer routines, katz_convert_f64_f32) against the hardware conversions:
rounding to nearest with ties to even, carries into the exponent, subnormal
results and underflow to zero, and exact widening."""
from __future__ import annotations

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
K = pytest.importorskip("paper_1807_03847_gb300")


def _cases():
    rng = np.random.default_rng(7)
    vals = [0.0, 1.0, 0.5, 2.0 ** -126, 2.0 ** -149, 2.0 ** -150, 1.5 * 2.0 ** -150, 2.0 ** -151, 2.0 ** -1000,
            np.nextafter(0.0, 1.0), 1.0 - 2.0 ** -25, 1.0 - 2.0 ** -24, 3.4e38, 3.5e38, 1e300]
    f = rng.random(20000).astype(np.float32).astype(np.float64)
    f = np.concatenate([f, np.ldexp(f, rng.integers(-160, 2, f.size))])
    # exact halfway points between neighbouring floats (ties), and one ulp of
    # binary64 to either side of them
    up = np.nextafter(f.astype(np.float32), np.float32(np.inf)).astype(np.float64)
    mid = (f + up) / 2
    vals += list(f) + list(mid) + list(np.nextafter(mid, 0.0)) + list(np.nextafter(mid, np.inf))
    vals += list(np.exp(rng.uniform(np.log(1e-60), 0.0, 40000)))
    # subnormal binary32 range, ties included
    sub = np.arange(0, 2 ** 12, dtype=np.float64) * 2.0 ** -149
    vals += list(sub) + list(sub + 2.0 ** -150) + list(np.nextafter(sub + 2.0 ** -150, 0.0))
    a = np.array(vals, np.float64)
    return a[np.isfinite(a) & (a >= 0)]


def test_rounding_matches_the_hardware():
    x = torch.from_numpy(_cases()).cuda()
    out, back = K.katz_convert_f64_f32(x)
    want = x.float()
    assert torch.equal(out.view(torch.int32), want.view(torch.int32))
    assert torch.equal(back.view(torch.int64), want.double().view(torch.int64))


def test_arguments_are_checked():
    x = torch.zeros(4, dtype=torch.float64)
    with pytest.raises((K.KatzError, AssertionError)):
        K.katz_convert_f64_f32(x)
