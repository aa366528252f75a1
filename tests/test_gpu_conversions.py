"""The integer FP64 <-> FP32 conversions of the CG vector kernels (rounding to nearest, ties to
even, by the IEEE 754 formats) against the hardware conversions: random bit patterns over the
whole range, values at every rounding boundary (ties, half-ulps, the overflow edge, the normal /
subnormal edge of binary32), zeros, infinities, NaNs and binary32 subnormals."""
import numpy as np
import pytest

from gpu_helpers import topo_lib, torch_cuda

pytestmark = pytest.mark.gpu


def _doubles(rng):
    bits = rng.integers(0, 2**64, size=1 << 20, dtype=np.uint64)
    d = [bits.view(np.float64)]
    # doubles near the binary32 grid: a float plus multiples of a quarter of its ulp (ties included)
    f = np.ldexp(rng.standard_normal(1 << 16), rng.integers(-149, 127, size=1 << 16)).astype(np.float32)
    f = f[np.isfinite(f) & (f != 0)]
    ulp = np.spacing(np.abs(f)).astype(np.float64)
    for k in (-3, -2, -1, 1, 2, 3):
        d.append(f.astype(np.float64) + k * ulp / 4)
    # binary32 subnormal / normal edge and the overflow edge
    edge = np.array([2.0**-126, 2.0**-149, 2.0**-150, 1.5 * 2.0**-150, 2.0**-151, 2.0**-127,
                     (2 - 2.0**-23) * 2.0**127, (2 - 2.0**-24) * 2.0**127, 2.0**128, 2.0**-1074,
                     0.0, np.inf, np.nan, 1.0, 1.0 + 2.0**-24, 1.0 + 3 * 2.0**-24])
    d.append(np.concatenate([edge, -edge]))
    return np.concatenate(d)


def test_integer_conversions_match_the_hardware():
    torch = torch_cuda()
    topo = topo_lib()
    rng = np.random.default_rng(71)
    d = _doubles(rng)
    fbits = rng.integers(0, 2**32, size=d.size, dtype=np.uint64).astype(np.uint32)
    fbits[:4096] = np.arange(4096, dtype=np.uint32)  # subnormals
    fbits[4096:8192] = np.arange(4096, dtype=np.uint32) | np.uint32(0x80000000)
    f = fbits.view(np.float32)
    bad = topo.check_conversions(torch.as_tensor(d, device="cuda"),
                                 torch.as_tensor(f, device="cuda"))
    assert bad == (0, 0)
