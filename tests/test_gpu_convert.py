"""Integer-unit precision conversions (fdst_convert) against the IEEE 754
conversions NumPy performs on the host: double -> float rounded to nearest
(ties to even) and float -> double bit for bit, the double-float split within
2^-48 |x| with |lo| below one unit of hi, the join equal to the FP64 sum of
the two parts. Inputs: seeded normals scaled over 60 decades, random bit
patterns, and the edge values of the ranges (zero, subnormals, the largest
float and the values rounding past it, ties, infinities)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _inputs():
    rng = np.random.default_rng(2024)
    a = rng.standard_normal(300_000) * 10.0 ** rng.uniform(-30, 30, 300_000)
    bits = rng.integers(0, 2 ** 63, 100_000, dtype=np.uint64)
    bits |= rng.integers(0, 2, 100_000, dtype=np.uint64) << np.uint64(63)
    b = bits.view(np.float64)
    edge = np.array([0.0, -0.0, 1.0, -1.0, 3.4028234663852886e38, 3.4028235677973366e38, -3.4028235677973366e38,
                     3.402823567797337e38, 1.1754943508222875e-38, 5.877471754111438e-39, 1e-40, 1e-46, 1e-300,
                     1e300, np.inf, -np.inf, 2.0 ** -74, 2.0 ** -75, 1 + 2.0 ** -24, 1 + 2.0 ** -23 + 2.0 ** -24,
                     1 - 2.0 ** -25, -(1 + 3 * 2.0 ** -24), 2.0 ** 127, 2.0 ** 128, (2 - 2.0 ** -23) * 2.0 ** 127])
    x = np.concatenate([a, b, edge])
    return x[~np.isnan(x)]


def test_f64_to_f32_nearest_bit_exact():
    import paper_1712_00403_gb300 as fd
    x = _inputs()
    src = torch.tensor(x, device="cuda")
    dst = torch.empty(x.size, dtype=torch.float32, device="cuda")
    fd.convert(fd.CONVERT_F64_TO_F32, src, dst)
    torch.cuda.synchronize()
    with np.errstate(over="ignore"):
        ref = x.astype(np.float32)
    assert np.array_equal(dst.cpu().numpy().view(np.uint32), ref.view(np.uint32))


def test_f32_to_f64_exact():
    import paper_1712_00403_gb300 as fd
    with np.errstate(over="ignore"):
        f = _inputs().astype(np.float32)
    src = torch.tensor(f, device="cuda")
    dst = torch.empty(f.size, dtype=torch.float64, device="cuda")
    fd.convert(fd.CONVERT_F32_TO_F64, src, dst)
    torch.cuda.synchronize()
    assert np.array_equal(dst.cpu().numpy().view(np.uint64), f.astype(np.float64).view(np.uint64))


def test_split_and_join():
    import paper_1712_00403_gb300 as fd
    x = _inputs()
    x = x[np.isfinite(x) & (np.abs(x) < 3e38)]
    src = torch.tensor(x, device="cuda")
    pair = torch.empty(2 * x.size, dtype=torch.float32, device="cuda")
    fd.convert(fd.CONVERT_F64_TO_DF, src, pair)
    back = torch.empty(x.size, dtype=torch.float64, device="cuda")
    fd.convert(fd.CONVERT_DF_TO_F64, pair, back)
    torch.cuda.synchronize()
    p = pair.cpu().numpy().reshape(-1, 2).astype(np.float64)
    hi, lo = p[:, 0], p[:, 1]
    # double-float range (both parts normal floats): hi + lo within 2^-48 |x|, |lo| < ulp(hi)
    rng_ok = (np.abs(x) >= 2.0 ** -74) & (np.abs(x) < 2.0 ** 127)
    err = np.abs((hi + lo) - x)
    assert np.all(err[rng_ok] <= 2.0 ** -48 * np.abs(x[rng_ok]))
    assert np.all(np.abs(lo[rng_ok]) <= np.abs(hi[rng_ok]) * 2.0 ** -23)
    # zero stays zero
    assert np.all(hi[x == 0] == 0) and np.all(lo[x == 0] == 0)
    # join: the FP64 sum of the two parts, bit for bit
    assert np.array_equal(back.cpu().numpy().view(np.uint64), (hi + lo).view(np.uint64))
