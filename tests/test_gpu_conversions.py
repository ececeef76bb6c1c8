"""The FP64 <-> FP32 conversions of the FP32-mixed kernels (built from the
bit patterns with integer operations) against IEEE 754 conversions done by
numpy on the host: rounding to nearest with ties to even, the rounding
remainder, the exact widening, and the special values."""
import numpy as np
import pytest

from paper_2606_18927_gb300 import dg
from gpu_helpers import torch_cuda

pytestmark = pytest.mark.gpu


def _inputs():
    rng = np.random.default_rng(2024)
    n = 1 << 20
    # random magnitudes over most of the FP32 normal range, both signs
    mant = rng.uniform(1.0, 2.0, n)
    expo = rng.integers(-120, 120, n)
    d = np.ldexp(mant, expo) * rng.choice([-1.0, 1.0], n)
    # exact ties and near-ties: a float plus half an FP32 unit (and one FP64 unit either side)
    f0 = rng.uniform(1.0, 2.0, 4096).astype(np.float32).astype(np.float64)
    half = np.ldexp(1.0, -24)
    ties = np.concatenate([f0 + half, f0 + half + np.ldexp(1.0, -52), f0 + half - np.ldexp(1.0, -52),
                           -(f0 + half)])
    # values that round up across a power of two, the largest float and zero
    edge = np.array([np.nextafter(2.0, 0.0), np.nextafter(1.0, 0.0), -np.nextafter(4.0, 0.0), 0.0, -0.0,
                     float(np.finfo(np.float32).max), float(np.finfo(np.float32).tiny), 1.0, -1.5, 1e-3, 71.42857])
    return np.concatenate([d, ties, edge])


def test_round_to_nearest_and_remainder():
    torch = torch_cuda()
    d = _inputs()
    g = d.astype(np.float32)
    f, rem, gd = dg.convert_fp32(torch.from_numpy(d).cuda(), torch.from_numpy(g).cuda())
    f = f.cpu().numpy(); rem = rem.cpu().numpy(); gd = gd.cpu().numpy()
    ref = d.astype(np.float32)
    assert np.array_equal(f.view(np.uint32), ref.view(np.uint32))
    # the remainder d - f (exact in FP64): its 29 bits kept to 23, an error
    # below 64 units of d's last place (2^-46 |d|)
    r_ref = d - ref.astype(np.float64)
    big = np.abs(d) > 1e-20
    ulp = np.spacing(np.abs(d))
    assert np.all(np.abs(rem[big] - r_ref[big]) < 64 * ulp[big])
    assert np.all(np.abs(rem[big] - r_ref[big]) <= np.ldexp(1.0, -46) * np.abs(d[big]))
    assert np.abs(f.astype(np.float64)[big] + rem[big] - d[big]).max() <= np.ldexp(1.0, -46) * np.abs(d[big]).max()
    # widening is exact
    assert np.array_equal(gd.view(np.uint64), g.astype(np.float64).view(np.uint64))


def test_special_values():
    torch = torch_cuda()
    d = np.array([np.inf, -np.inf, np.nan, 1e300, -1e300, 1e-300, -1e-300, 0.0, -0.0])
    g = np.array([np.inf, -np.inf, np.nan, 1e-45, -1e-45, 0.0, -0.0, 3.0, -2.5], dtype=np.float32)
    f, rem, gd = dg.convert_fp32(torch.from_numpy(d).cuda(), torch.from_numpy(g).cuda())
    f = f.cpu().numpy(); rem = rem.cpu().numpy(); gd = gd.cpu().numpy()
    assert f[0] == np.inf and f[1] == -np.inf and np.isnan(f[2])
    assert f[3] == np.inf and f[4] == -np.inf
    # below the FP32 normal range: signed zero
    assert f[5] == 0.0 and not np.signbit(f[5]) and f[6] == 0.0 and np.signbit(f[6])
    assert f[7] == 0.0 and np.signbit(f[8])
    assert np.all(rem[[0, 1, 2, 7, 8]] == 0.0)
    assert gd[0] == np.inf and gd[1] == -np.inf and np.isnan(gd[2])
    # FP32 subnormals give signed zero
    assert gd[3] == 0.0 and np.signbit(gd[4])
    assert gd[7] == 3.0 and gd[8] == -2.5
