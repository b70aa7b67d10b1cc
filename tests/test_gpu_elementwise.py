"""The kernels' inline per-element arithmetic on the device (m1_op_elementwise)
against correctly rounded results: numpy's IEEE division and square root on the host,
and for FP64 also CUDA's (torch on the same device), which agree bit for bit.

- FP64 reciprocal and square root (hardware estimate + one third-order
  correction): within 1 ulp of the correctly rounded result over positive
  normal arguments from 2^-1000 to 2^1000;
- FP32 approximate reciprocal and square root: within 2 ulps;
- the double-word split and the FP32 -> FP64 widening of the mixed path: bit for
  bit the IEEE conversions and the host runs of the same code
  (tests/test_dw_conversions.py), over every class of input."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
m1 = pytest.importorskip("paper_2208_14703_gb300.m1")


def ulp_distance(a, b, itype):
    """|a - b| in units in the last place, for finite values of one sign."""
    return np.abs(a.view(itype).astype(np.int64) - b.view(itype).astype(np.int64))


def positive_doubles(n, lo_exp, hi_exp, seed):
    rng = np.random.default_rng(seed)
    e = rng.uniform(lo_exp, hi_exp, n)
    x = np.exp2(np.floor(e)) * rng.uniform(1.0, 2.0, n)
    edges = np.array([1.0, 2.0, np.nextafter(1.0, 2.0), np.nextafter(2.0, 1.0), 3.0, 0.5, 1.5,
                      2.0 ** lo_exp, 2.0 ** hi_exp, 4.0, 9.0, 1e-300, 1e300])
    return np.concatenate([edges, x])


@pytest.mark.parametrize("fn, ref", [(m1.FN_RCP64, lambda t: 1.0 / t), (m1.FN_SQRT64, torch.sqrt)])
def test_fp64_rcp_sqrt_within_one_ulp(fn, ref):
    x = positive_doubles(2_000_000, -1000, 1000, seed=31 + fn)
    xd = torch.from_numpy(x).cuda()
    got = m1.op_elementwise(fn, xd).cpu().numpy()
    cuda_ref = ref(xd).cpu().numpy()
    host_ref = 1.0 / x if fn == m1.FN_RCP64 else np.sqrt(x)
    assert np.array_equal(cuda_ref.view(np.uint64), host_ref.view(np.uint64))
    d = ulp_distance(got, cuda_ref, np.int64)
    print(f"fn {fn}: max {d.max()} ulp, {np.mean(d == 0):.4f} correctly rounded")
    assert d.max() <= 1


@pytest.mark.parametrize("fn", [m1.FN_RCP32, m1.FN_SQRT32])
def test_fp32_approximations_within_two_ulps(fn):
    x = positive_doubles(2_000_000, -120, 120, seed=41 + fn).astype(np.float32)
    xd = torch.from_numpy(x).cuda()
    got = m1.op_elementwise(fn, xd).cpu().numpy()
    x64 = x.astype(np.float64)
    host_ref = (1.0 / x64 if fn == m1.FN_RCP32 else np.sqrt(x64)).astype(np.float32)
    cuda_ref = (1.0 / xd if fn == m1.FN_RCP32 else torch.sqrt(xd)).cpu().numpy()
    d = ulp_distance(got, host_ref, np.int32)
    print(f"fn {fn}: max {d.max()} ulp, {np.mean(d == 0):.4f} correctly rounded; torch's FP32 "
          f"operation matches the correctly rounded result on {np.mean(cuda_ref == host_ref):.6f}")
    assert d.max() <= 2


def test_dw_split_on_device_is_the_ieee_split():
    from test_dw_conversions import edge_doubles, random_doubles, reference_split, same_bits
    x = np.concatenate([edge_doubles(), random_doubles(51, 1_000_000)])
    got = m1.op_elementwise(m1.FN_DW_SPLIT, torch.from_numpy(x).cuda()).cpu().numpy()
    hi, lo = reference_split(x)
    same_bits(np.ascontiguousarray(got[:, 0]), hi)
    same_bits(np.ascontiguousarray(got[:, 1]), lo)
    hhi, hlo = m1.dw_split(x)          # the host run of the same code
    same_bits(np.ascontiguousarray(got[:, 0]), hhi)
    same_bits(np.ascontiguousarray(got[:, 1]), hlo)


def test_widen_on_device_is_exact():
    from test_dw_conversions import random_floats, same_bits
    x = random_floats(52, 1_000_000)
    got = m1.op_elementwise(m1.FN_WIDEN, torch.from_numpy(x).cuda()).cpu().numpy()
    with np.errstate(invalid="ignore"):
        ref = x.astype(np.float64)
    same_bits(got, ref, np.uint64)
