// Double-word FP32 arithmetic ("float-float"): a value is the unevaluated sum
// hi + lo of two FP32 numbers with |lo| <= ulp(hi) / 2, about 48 bits of
// significand.  The operations follow the double-word algorithms analysed by
// Joldes, Muller & Popescu, "Tight and rigorous error bounds for basic building
// blocks of double-word arithmetic", ACM TOMS 44(2), 2017, built on the
// error-free transforms TwoSum (Knuth), Fast2Sum (Dekker) and TwoProd by a fused
// multiply-add.  Relative error bounds, with u = 2^-24: sum of two double words
// (their accurate algorithm) 3u^2 + 13u^3; product of two double words (the FMA
// algorithm) 5u^2; product by an FP32 number 2u^2; sum with an FP32 number 2u^2.
// The reciprocal and square root here are one Newton-Raphson correction of the
// correctly rounded FP32 result, computed with these operations (relative error
// a few u^2).
//
// GB300 runs FP32 at 64 times its FP64 rate, so a computation needing about 48
// bits costs fewer FP32 issue slots as double words than FP64 slots: the
// mixed-precision defect uses this when its tolerance allows (m1_kernels.cu).
#pragma once
#include <cstring>
#include <cuda_runtime.h>

#include "m1_device.cuh"   // float_of_bits, bits_of_float, widen

namespace m1 {

struct DW {
    float hi, lo;
};

// A cell's state (E, Fx, Fy, T) and opacities as double words, and the
// per-slot double-word copies the mixed path's defect reads (fine level: the
// iterate v, the right-hand side b, the opacities).
struct alignas(32) DW4 {
    DW E, Fx, Fy, T;
};
struct alignas(16) DW2 {
    DW sa, ss;
};
struct DwLevel {
    DW4* v;
    DW4* b;
    DW2* sig;
};

__device__ __forceinline__ DW two_sum(float a, float b)
{
    const float s = a + b;
    const float bb = s - a;
    return DW{ s, (a - (s - bb)) + (b - bb) };
}

// |a| >= |b| (or a = 0)
__device__ __forceinline__ DW fast_two_sum(float a, float b)
{
    const float s = a + b;
    return DW{ s, b - (s - a) };
}

__device__ __forceinline__ DW two_prod(float a, float b)
{
    const float p = a * b;
    return DW{ p, fmaf(a, b, -p) };
}

__host__ __device__ __forceinline__ DW dw_from(double x)
{
    const float h = (float)x;
    return DW{ h, (float)(x - (double)h) };
}

// dw_from as a call, for the values dw_split's integer form does not cover:
// kept out of line so that the compiler branches around it instead of
// evaluating it for every value and selecting.
static __host__ __device__ __noinline__ DW dw_from_call(double x) { return dw_from(x); }

// The pair dw_from(x) by integer and FP32 operations on the bit pattern of x.
// GB300 issues FP64 instructions, the conversions between FP64 and FP32 among
// them, at 1/64 of the FP32 rate, and the three conversions of dw_from bound
// the kernels that split every cell of a level.  With x = M 2^(e-1075), M the
// 53-bit significand and e the biased exponent: hi = M rounded to nearest-even
// at bit 29 (a carry into the exponent field is the correct rounding),
// rebiased to FP32; lo = (M - hi's significand) 2^(e-1075), an integer of at
// most 29 bits, formed in FP32 as two exact 15-bit halves joined by one
// fused multiply-add (a single rounding to nearest) and scaled by the power
// of two, exact while it stays normal.  That holds for 2^-74 <= |x| < 2^127
// (e in [949, 1149]); zero is handled here too, and the other values call
// dw_from, so the result equals dw_from(x) for every x.
__host__ __device__ __forceinline__ DW dw_split(double x)
{
    unsigned long long b;
    memcpy(&b, &x, sizeof b);
    const unsigned sign = (unsigned)(b >> 32) & 0x80000000u;
    const unsigned long long a = b & 0x7fffffffffffffffull;
    if (a == 0) return DW{ float_of_bits(sign), 0.0f };
    const unsigned e = (unsigned)(a >> 52);
    if (e - 949u > 1149u - 949u) return dw_from_call(x);
    const unsigned long long q = (a + 0x0fffffffull + ((a >> 29) & 1ull)) >> 29;
    const bool up = q != (a >> 29);
    const unsigned low = (unsigned)a & 0x1fffffffu;
    const unsigned m = up ? 0x20000000u - low : low;        // |lo| in units of 2^(e-1075)
    const float scale = float_of_bits((e - 948u) << 23);     // 2^(e-1075)
    const float mag = fmaf(small_uint_to_float(m >> 15), 32768.0f * scale,
                           small_uint_to_float(m & 0x7fffu) * scale);
    const bool neg = (sign != 0) != up;
    return DW{ float_of_bits(((unsigned)q - (896u << 23)) | sign),
               float_of_bits(bits_of_float(mag) | (neg && m != 0 ? 0x80000000u : 0u)) };
}


__device__ __forceinline__ double dw_to_double(DW x) { return (double)x.hi + (double)x.lo; }

__device__ __forceinline__ DW4 dw4_from(double E, double Fx, double Fy, double T)
{
    return DW4{ dw_split(E), dw_split(Fx), dw_split(Fy), dw_split(T) };
}

__device__ __forceinline__ DW operator-(DW x) { return DW{ -x.hi, -x.lo }; }

__device__ __forceinline__ DW operator+(DW x, DW y)
{
    const DW s = two_sum(x.hi, y.hi);
    const DW t = two_sum(x.lo, y.lo);
    const DW v = fast_two_sum(s.hi, s.lo + t.hi);
    return fast_two_sum(v.hi, t.lo + v.lo);
}

__device__ __forceinline__ DW operator-(DW x, DW y) { return x + (-y); }

__device__ __forceinline__ DW operator+(DW x, float y)
{
    const DW s = two_sum(x.hi, y);
    return fast_two_sum(s.hi, x.lo + s.lo);
}

__device__ __forceinline__ DW operator*(DW x, DW y)
{
    const DW c = two_prod(x.hi, y.hi);
    const float t = fmaf(x.lo, y.hi, fmaf(x.hi, y.lo, x.lo * y.lo));
    return fast_two_sum(c.hi, c.lo + t);
}

__device__ __forceinline__ DW operator*(DW x, float y)
{
    const DW c = two_prod(x.hi, y);
    return fast_two_sum(c.hi, fmaf(x.lo, y, c.lo));
}

__device__ __forceinline__ bool operator>(DW x, float y) { return x.hi > y || (x.hi == y && x.lo > 0.f); }

// 1/x: r0 = the correctly rounded FP32 reciprocal of x.hi, then
// r = r0 + r0 e with e = 1 - x r0 formed in double words (|e| ~ u).
__device__ __forceinline__ DW dw_rcp(DW x)
{
    const float r0 = __frcp_rn(x.hi);
    const DW xr = x * r0;
    const DW e = DW{ 1.f, 0.f } - xr;
    return fast_two_sum(r0, r0 * e.hi);
}

// sqrt(a): s0 = the correctly rounded FP32 square root of a.hi, then
// s = s0 + (a - s0^2) / (2 s0), the difference formed exactly by TwoProd.
__device__ __forceinline__ DW dw_sqrt(DW a)
{
    const float s0 = __fsqrt_rn(a.hi);
    const DW p = two_prod(s0, s0);
    const float d = ((a.hi - p.hi) - p.lo) + a.lo;
    return fast_two_sum(s0, d * (0.5f * __frcp_rn(s0)));
}

}  // namespace m1
