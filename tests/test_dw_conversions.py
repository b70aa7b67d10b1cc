"""The integer-and-FP32 conversions the mixed path applies per cell (the
double-word split of FP64 values and the FP32 -> FP64 widening), run on the host
through the library's m1_dw_split / m1_f32_widen, against the IEEE conversions
numpy performs (round to nearest even).  The split must give exactly
hi = fl32(x) and lo = fl32(x - hi) for every FP64 value, including the ranges
that take the conversion call (|x| < 2^-74, |x| >= 2^127, subnormal, infinite
and NaN inputs), zeros of both signs, ties at the rounding bit and carries into
the exponent.  The device runs of the same functions are compared in
tests/test_gpu_elementwise.py."""
import numpy as np
import pytest

m1 = pytest.importorskip("paper_2208_14703_gb300.m1")


def reference_split(x):
    with np.errstate(over="ignore", invalid="ignore"):
        hi = x.astype(np.float32)
        lo = (x - hi.astype(np.float64)).astype(np.float32)
    return hi, lo


def same_bits(a, b, itype=np.uint32):
    """Equal bit patterns, any NaN matching any NaN."""
    na, nb = np.isnan(a), np.isnan(b)
    assert np.array_equal(na, nb)
    assert np.array_equal(a[~na].view(itype), b[~nb].view(itype))


def edge_doubles():
    f = np.float64
    xs = [0.0, -0.0, np.inf, -np.inf, np.nan, 5e-324, -5e-324, 2.2250738585072014e-308,
          np.finfo(np.float32).max, -np.finfo(np.float32).max, np.finfo(np.float32).tiny,
          2.0 ** -149, 2.0 ** -150, 1e300, -1e300, 1.0, -1.0, 1.0 / 3.0]
    for e in (-75, -74, -73, -1, 0, 1, 126, 127, 128):
        for m in (1.0, np.nextafter(1.0, 2.0), np.nextafter(2.0, 1.0)):
            xs += [m * f(2.0) ** e, -m * f(2.0) ** e]
    bits = []
    for e in (949, 950, 1023, 1148, 1149, 948, 1150):
        top = np.uint64(e) << np.uint64(52)
        for low in (0x0FFFFFFF, 0x10000000, 0x10000001, 0x1FFFFFFF, 0x30000000, 0x10000000 | (1 << 29),
                    (1 << 52) - 1, ((1 << 23) - 1) << 29 | 0x10000000, ((1 << 23) - 1) << 29 | 0x1FFFFFFF,
                    0x00007FFF, 0x00008000, 0x1FFF8000):
            bits.append(top | np.uint64(low))
    b = np.array(bits, dtype=np.uint64)
    return np.concatenate([np.array(xs, dtype=np.float64), b.view(np.float64), -b.view(np.float64)])


def random_doubles(seed, n=400_000):
    rng = np.random.default_rng(seed)
    b = rng.integers(0, 2 ** 63, size=n, dtype=np.uint64)
    b |= rng.integers(0, 2, size=n, dtype=np.uint64) << np.uint64(63)
    # half spread over all exponents, half over the FP32 range where the integer form runs
    e = rng.integers(880, 1170, size=n // 2, dtype=np.uint64)
    b[: n // 2] = (b[: n // 2] & np.uint64(0x800FFFFFFFFFFFFF)) | (e << np.uint64(52))
    # a quarter with the 29 dropped bits at or next to a tie
    q = slice(n // 2, 3 * n // 4)
    tie = rng.choice(np.array([0x0FFFFFFF, 0x10000000, 0x10000001], dtype=np.uint64), size=n // 4)
    b[q] = (b[q] & ~np.uint64(0x1FFFFFFF)) | tie
    return b.view(np.float64)


def test_dw_split_edges():
    x = edge_doubles()
    hi, lo = m1.dw_split(x)
    rhi, rlo = reference_split(x)
    same_bits(hi, rhi)
    same_bits(lo, rlo)


def test_dw_split_random_over_all_exponents():
    x = random_doubles(7)
    hi, lo = m1.dw_split(x)
    rhi, rlo = reference_split(x)
    same_bits(hi, rhi)
    same_bits(lo, rlo)
    fin = np.isfinite(x) & (np.abs(x) < 2.0 ** 127) & (np.abs(x) >= 2.0 ** -74)
    # the pair is normalised and carries x to about 48 bits
    assert np.all(np.abs(lo[fin]).astype(np.float64) <= np.spacing(np.abs(hi[fin])).astype(np.float64) / 2)
    err = np.abs(hi[fin].astype(np.float64) + lo[fin].astype(np.float64) - x[fin])
    assert np.all(err <= np.abs(x[fin]) * 2.0 ** -47)


def random_floats(seed, n=400_000):
    rng = np.random.default_rng(seed)
    b = rng.integers(0, 2 ** 32, size=n, dtype=np.uint64).astype(np.uint32)
    specials = np.array([0, 0x80000000, 1, 0x807FFFFF, 0x00800000, 0x7F7FFFFF, 0xFF7FFFFF,
                         0x7F800000, 0xFF800000, 0x7FC00000, 0x3F800000, 0xBF800001], dtype=np.uint32)
    return np.concatenate([specials, b]).view(np.float32)


def test_f32_widen_all_classes():
    x = random_floats(8)
    y = m1.f32_widen(x)
    with np.errstate(invalid="ignore"):
        ref = x.astype(np.float64)
    same_bits(y, ref, np.uint64)


def test_conversion_arguments():
    assert m1._lib.m1_dw_split(None, -1, None, None) == m1.ERR_INVALID_ARG
    assert m1._lib.m1_dw_split(None, 3, None, None) == m1.ERR_INVALID_ARG
    assert m1._lib.m1_dw_split(None, 0, None, None) == 0
    assert m1._lib.m1_f32_widen(None, 2, None) == m1.ERR_INVALID_ARG
    assert m1._lib.m1_f32_widen(None, 0, None) == 0
