// Device-side data structures and per-cell arithmetic of the implicit M1
// multigrid step (Bloch, Tremblin, Gonzalez & Audit, arXiv:2208.14703).
//
// Layout.  A level stores its states as arrays of Cell4 {E, Fx, Fy, T}
// (array-of-structures: one 32-byte vector load per cell in FP64, 16 bytes in
// FP32), row-major with index j*nx + i, and the opacities as Sig2 {sa, ss}.
// In 1D ny = 1 and Fy stays zero.
#pragma once
#include <cfloat>
#include <cstdint>
#include <cstring>
#include <cuda_runtime.h>

namespace m1 {

enum Bc { BC_PERIODIC = 0, BC_REFLECT = 1, BC_NEUMANN = 2, BC_INFLOW = 3 };
enum Kind { KIND_STATE = 0, KIND_DIFF = 1 };
enum Wall { WALL_W = 0, WALL_E = 1, WALL_S = 2, WALL_N = 3 };

// Relative slack of the admissibility test that decides whether a prolongated
// cell is damped (Algorithm 4): cells on the f = 1 boundary up to rounding are
// not damped.  Same value in FP32 would be below its precision; the FP32 path
// uses a slack scaled to its epsilon.
template <typename R> struct Slack;
template <> struct Slack<double> { static constexpr double v = 1e-12; };
template <> struct Slack<float> { static constexpr float v = 1e-6f; };

template <typename R> struct alignas(4 * sizeof(R)) Cell4 { R E, Fx, Fy, T; };
template <typename R> struct alignas(2 * sizeof(R)) Sig2 { R sa, ss; };

// Block size of the cell-parallel kernels (256 threads) and the tile shape of the
// no-allocation residual: 32 x 8 cells in 2D, 256 x 1 in 1D.
constexpr int kThreads = 256;
constexpr int kTx2 = 32, kTy2 = 8, kTx1 = 256;
// Warp strips of the stencil kernels: a warp's 32 lanes own 32 consecutive columns
// (kStripW = 30 output columns and one halo column on each side) and march up
// to kStripH rows (2D; one row in 1D).
constexpr int kStripW = 30, kStripH = 16, kStripWarps = 2;
// Blocks of a persistent strip launch: up to 16 resident 2-warp blocks per SM.
constexpr int kStripBlocks = 152 * 16;

// One grid level as the kernels see it.  Constants that depend on the time
// step (ax, bx, diag, cdt) are rewritten before every implicit step.
template <typename R>
struct Level {
    int dim, nx, ny, n;
    int bc[4];
    int tx, ty, tiles_x, tiles;   // 32 x 8 tiles of the no-allocation residual (else 0)
    int chunks;                   // 256-cell chunks (cell-parallel kernels)
    int part_off;                 // first norm partial of this instance (level 0)
    int prof_len;                 // stride of the inflow profile table
    int sx, sh, strips;           // warp strips: count along x, rows each, total
    int ring;                     // FP32 correction form: stage strip rows by cp.async
    R c, a_r, c_v;
    R ic2;                        // 1 / c^2
    R ax, ay, bx, by;             // c dt / h and dt / (2 h) per axis (y: 0 in 1D)
    R diag;                       // 1 + ax + ay
    R cdt;                        // c dt
    double vol;                   // cell volume h^d (norm weight)
    Cell4<R>* v;                  // restricted iterate v_l
    Cell4<R>* u[2];               // ping-pong iterate u_l
    Cell4<R>* f;                  // right-hand side (b at level 0, FAS rhs above)
    Cell4<R>* r;                  // residual (restricted from below / computed here)
    Cell4<R>* w;                  // base state of the correction form (mixed path), else null
    Cell4<R>* aw;                 // A(w) of the base state (correction form), else null
    Sig2<R>* sig;                 // opacities
    R* inflow;                    // [wall][E, Fx, Fy][prof_len] prescribed ghosts
};

// Device-resident control block of one implicit step: the cycle counter, the
// residual norms, the implicit pseudo-time step and the stop flag.  Every kernel
// of a captured V-cycle returns at once when `done` is set, so a CUDA graph of
// the cycle can be relaunched past convergence without changing the result.
struct Ctl {
    // parameters (written by the host before the step)
    double tol, grow, shrink, eps_i, eps_d, dtau0, dtau_min, dtau_max, theta_ex, theta_c;
    double res0_floor;            // stop at once if ||r_0|| <= res0_floor ||b||
    int max_cycles, hist_len;
    int dtau_rule;                // 0: |change| of the residual norm; 1: its decrease
    int active;                   // the instance takes part in the batch
    double dw_floor;              // mixed path: the defect of the cycles is formed in
                                  // double-word FP32 when tol ||r_0|| > dw_floor ||b||
    int defect_dw;                // (state) set by FIN_INIT from that rule
    // state
    double res0, res, res_prev, bnorm, dtau;
    int kappa, done, status, result_buf;
    int pending_r0;               // the next deferred norm is r_0 again (set by FIN_INIT)
    unsigned int newton_fail, damped;
    double* hist;                 // res_hist[kappa], length hist_len (device)
    double* dtau_hist;            // dtau used in cycle kappa, length hist_len
};

enum CtlStatus { CTL_OK = 0, CTL_NOT_CONVERGED = -4 };

// Completion count of a batch: every instance that sets its `done` flag adds
// one; `all_done` is set when the count reaches the number of active instances.
struct BatchCtl {
    int n_done, n_active, all_done, pad;
};

// A work list: items[0 .. *count) of (instance, strip or 256-cell chunk), read by
// persistent kernels (a fixed grid striding over the items), so the list can
// change between V-cycles without changing a captured graph.
struct WorkList {
    const int2* items;
    const int* count;
    int capacity;
};

// Blocks of a persistent launch: 4 resident CTAs on each of the 152 SMs.
constexpr int kPersistentBlocks = 152 * 4;

// ---------------------------------------------------------------------------
// FP32 <-> FP64 conversions without conversion instructions.  GB300 issues
// FP64 instructions, the conversions between FP64 and FP32 among them, at 1/64
// of the FP32 rate, and the FP64 kernels are bound by that pipe; these forms
// use integer and FP32 operations on the bit patterns and give exactly the
// IEEE results (round to nearest even).  Values outside the ranges they cover
// call the conversion out of line, so that the compiler branches around it
// instead of evaluating it for every value and selecting.
__host__ __device__ __forceinline__ float float_of_bits(unsigned u)
{
    float f;
    memcpy(&f, &u, sizeof f);
    return f;
}

__host__ __device__ __forceinline__ unsigned bits_of_float(float f)
{
    unsigned u;
    memcpy(&u, &f, sizeof u);
    return u;
}

// An integer 0 <= m < 2^23 as an FP32 number: 2^23 + m is exact in FP32 and
// the subtraction of 2^23 is exact.
__host__ __device__ __forceinline__ float small_uint_to_float(unsigned m)
{
    return float_of_bits(0x4b000000u | m) - 8388608.0f;
}

static __host__ __device__ __noinline__ double widen_call(float x) { return (double)x; }
static __host__ __device__ __noinline__ float narrow_call(double x) { return (float)x; }

// (double)x: for x normal or zero the exponent is rebiased by 1023 - 127 and
// the significand moved to the top of FP64's 52 bits; subnormals, infinities
// and NaN take the conversion.
__host__ __device__ __forceinline__ double widen(float x)
{
    const unsigned u = bits_of_float(x);
    const unsigned e = (u >> 23) & 0xffu;
    unsigned long long b = (unsigned long long)(u & 0x80000000u) << 32;
    if (e - 1u <= 253u)
        b |= ((unsigned long long)(e + 896u) << 52) | ((unsigned long long)(u & 0x7fffffu) << 29);
    else if ((u & 0x7fffffffu) != 0)
        return widen_call(x);
    double d;
    memcpy(&d, &b, sizeof d);
    return d;
}

// (float)x: with x = M 2^(e-1075) (M the 53-bit significand, e the biased
// exponent), M rounded to nearest-even at bit 29 (a carry into the exponent
// field is the correct rounding, up to infinity past FLT_MAX) and rebiased.
// Covers e in [897, 1150], the x whose FP32 rounding is normal or infinite;
// zero, subnormal results, infinities and NaN take the conversion.
__host__ __device__ __forceinline__ float narrow(double x)
{
    unsigned long long b;
    memcpy(&b, &x, sizeof b);
    const unsigned long long a = b & 0x7fffffffffffffffull;
    const unsigned e = (unsigned)(a >> 52);
    if (e - 897u > 1150u - 897u) return narrow_call(x);
    const unsigned long long q = (a + 0x0fffffffull + ((a >> 29) & 1ull)) >> 29;
    return float_of_bits(((unsigned)q - (896u << 23)) | ((unsigned)(b >> 32) & 0x80000000u));
}

// ---------------------------------------------------------------------------
// Reciprocal and square root of the per-cell arithmetic.
// FP64: a hardware estimate (PTX rcp.approx.ftz.f64, rsqrt.approx.ftz.f64;
// relative error near 2^-22 or better) refined by Newton-Raphson iteration, the
// textbook method for these functions: for r ~ 1/a, r <- r + r (1 - a r); for
// y ~ 1/sqrt(a), y <- y + (y/2)(1 - a y^2); each step squares the relative
// error, so two steps reach FP64 rounding (the result can differ from the
// correctly rounded one in the last bit).  The square root is s = a y with one
// correction s <- s + (y/2)(a - s^2).  Arguments are positive normal numbers.
// FP32: the approximate hardware operations (rcp.approx.ftz.f32,
// sqrt.approx.ftz.f32; about 1 ulp), the correction form keeping their error
// relative to the correction.
template <typename R> struct Fm;
template <> struct Fm<double> {
    // 1/a from the hardware estimate r0 with relative error e = 1 - a r0:
    // 1/a = r0 / (1 - e) = r0 (1 + e + e^2 + ...); keeping e^2 makes the error
    // third order in e, so one step reaches FP64 rounding.
    __device__ static __forceinline__ double rcp(double a)
    {
        double r;
        asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(a));
        const double e = fma(-a, r, 1.0);
        return fma(r, fma(e, e, e), r);
    }
    // sqrt(a) from the hardware estimate y of 1/sqrt(a): with s0 = a y and
    // t = 1 - s0 y (= 1 - a y^2), sqrt(a) = s0 (1 - t)^(-1/2)
    // = s0 (1 + t/2 + 3 t^2/8 + ...) (binomial series); the t^2 term makes the
    // error third order in t.
    __device__ static __forceinline__ double sqrt(double a)
    {
        double y;
        asm("rsqrt.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(a));
        const double s0 = a * y;
        const double t = fma(-s0, y, 1.0);
        return fma(s0 * t, fma(0.375, t, 0.5), s0);
    }
};
template <> struct Fm<float> {
    __device__ static __forceinline__ float rcp(float a)
    {
        float r;
        asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(a));
        return r;
    }
    __device__ static __forceinline__ float sqrt(float a)
    {
        float r;
        asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(a));
        return r;
    }
};

// ---------------------------------------------------------------------------
// FP64 comparisons from bit patterns: exact, off the FP64 pipe.
// x > 0 for an FP64 x from its bit pattern (sign clear, not zero, not NaN):
// the FP64 comparison would take an FP64-pipe slot.
__device__ __forceinline__ bool positive_f64(double x)
{
    const long long b = __double_as_longlong(x);
    return b > 0 && b <= 0x7ff0000000000000LL;
}

// x > 1 and x == 0 for an FP64 x from its bit pattern (NaN compares false, as in
// the FP64 comparisons these replace).
__device__ __forceinline__ bool gt_one_f64(double x)
{
    const long long b = __double_as_longlong(x);
    return b > 0x3ff0000000000000LL && b <= 0x7ff0000000000000LL;
}

__device__ __forceinline__ bool is_zero_f64(double x)
{
    return (__double_as_longlong(x) << 1) == 0;
}

// ---------------------------------------------------------------------------
// Per-cell arithmetic.

// M1 closure (Section 2.1, Eq. (5)) in the algebraically equivalent form
//   s = sqrt(4 - 3 f^2),  (1 - chi)/2 = (s - 1)/3,  (3 chi - 1)/(2 f^2) = 3/(2 + s),
//   P = (s - 1)/3 E I + 3/(2 + s) F F^T / (c^2 E),
// which needs no unit vector n and is smooth at F = 0.  f^2 is clamped to 1.
template <typename R>
__device__ __forceinline__ void closure(R E, R Fx, R Fy, R inv_c2, R& Pxx, R& Pxy, R& Pyy)
{
    const R iE = Fm<R>::rcp(E);
    const R fx = Fx * iE, fy = Fy * iE;
    // 4 - 3 f^2 with f^2 = |F/E|^2 / c^2 clamped to 1
    R a = fma(fma(fy, fy, fx * fx), R(-3) * inv_c2, R(4));
    if constexpr (sizeof(R) == 8) a = gt_one_f64(a) ? a : R(1);   // off the FP64 pipe
    else a = a > R(1) ? a : R(1);
    const R s = Fm<R>::sqrt(a);
    const R Eiso = E * fma(s, R(1) / R(3), R(-1) / R(3));
    const R q = Fm<R>::rcp(R(2) + s) * (R(3) * inv_c2);
    // E q (F/E)(F/E)^T = q (F/E) F^T
    const R qx = q * fx, qy = q * fy;
    Pxx = fma(qx, Fx, Eiso);
    Pxy = qx * Fy;
    Pyy = fma(qy, Fy, Eiso);
}

// Largest tau >= 0 with u + tau d admissible (E > 0, T > 0, |F| <= c E): the
// smallest positive root of |F + tau dF|^2 = c^2 (E + tau dE)^2 and the linear
// E and T bounds; +inf when none applies.
template <typename R>
__device__ __forceinline__ R max_admissible_step(const Cell4<R>& u, const Cell4<R>& d, R c)
{
    const R inf = R(INFINITY);
    R tau = inf;
    if (d.E < R(0)) tau = fmin(tau, -u.E / d.E);
    if (d.T < R(0)) tau = fmin(tau, -u.T / d.T);
    R c2 = c * c;
    R a = d.Fx * d.Fx + d.Fy * d.Fy - c2 * d.E * d.E;
    R b = u.Fx * d.Fx + u.Fy * d.Fy - c2 * u.E * d.E;
    R c0 = u.Fx * u.Fx + u.Fy * u.Fy - c2 * u.E * u.E;
    c0 = c0 > R(0) ? R(0) : c0;
    R disc = b * b - a * c0;
    R t = inf;
    if (a > R(0)) {
        R sd = sqrt(disc);
        t = b <= R(0) ? (-b + sd) / a : -c0 / (b + sd);
    } else if (a < R(0)) {
        if (b > R(0) && disc >= R(0)) t = -c0 / (b + sqrt(disc));
    } else if (b > R(0)) {
        t = -c0 / (R(2) * b);
    }
    return fmin(tau, t);
}

// The admissible set: E > 0, T > 0, |F| <= c E (with the slack of Slack<R>).
// c2 = c * c, which a caller may form once for many cells.
//
// FP64: |F|^2 <= c^2 E^2 (1 + slack) is first decided in FP32, from the values
// rounded to FP32, wherever those settle it with a relative margin of 1e-5: the
// FP32 sides carry a relative error below 4e-7 (inputs rounded once, three or
// four roundings after), so such a decision is the FP64 test's own.  Cells near
// the boundary (and values outside FP32's normal range) take the FP64 test.
// SLACK: with the factor (1 + Slack<R>) of the prolongation's damping test;
// without it, the plain cone of the explicit pseudo-time step's limiter.
template <typename R, bool SLACK = true>
__device__ __forceinline__ bool admissible_c2(const Cell4<R>& s, R c2)
{
    if constexpr (sizeof(R) == 8) {
        if (!(positive_f64(s.E) && positive_f64(s.T))) return false;
        const float e32 = narrow(s.E), x32 = narrow(s.Fx), y32 = narrow(s.Fy);
        const float a32 = fmaf(y32, y32, x32 * x32);
        const float b32 = narrow(c2) * e32 * e32;
        if (b32 >= FLT_MIN && b32 <= FLT_MAX && a32 <= FLT_MAX) {
            if (a32 <= b32 * 0.99999f) return true;
            if (a32 >= b32 * 1.00001f) return false;
        }
        if (SLACK) return s.Fx * s.Fx + s.Fy * s.Fy <= c2 * s.E * s.E * (R(1) + Slack<R>::v);
        return s.Fx * s.Fx + s.Fy * s.Fy <= c2 * s.E * s.E;
    } else {
        if (SLACK)
            return s.E > R(0) && s.T > R(0) &&
                   s.Fx * s.Fx + s.Fy * s.Fy <= c2 * s.E * s.E * (R(1) + Slack<R>::v);
        return s.E > R(0) && s.T > R(0) && s.Fx * s.Fx + s.Fy * s.Fy <= c2 * s.E * s.E;
    }
}

template <typename R>
__device__ __forceinline__ bool admissible(const Cell4<R>& s, R c)
{
    return admissible_c2(s, c * c);
}

// Newton on g(T) = C T + K T^4 - R (increasing, convex for T > 0) started at
// T0 = min(R/C, (R/K)^(1/4)), which lies at or right of the root.
// FP32 iterations reach about 1e-7; the FP64 variant then takes one Halley
// step in FP64, reaching FP64 rounding.
__device__ __forceinline__ float newton_quartic_f32(float C, float K, float Rr, bool& ok)
{
    float T = fminf(Rr / C, sqrtf(sqrtf(Rr / K)));
    ok = false;
    for (int it = 0; it < 40; ++it) {
        float T3 = T * T * T;
        float g = fmaf(K, T3 * T, C * T) - Rr;
        float dg = fmaf(4.0f * K, T3, C);
        float dT = g * Fm<float>::rcp(dg);
        T -= dT;
        if (fabsf(dT) <= 4e-7f * T) { ok = true; break; }
    }
    return T;
}

template <typename R> struct Quartic;
template <> struct Quartic<float> {
    __device__ static float solve(float C, float K, float Rr, bool& ok)
    {
        return newton_quartic_f32(C, K, Rr, ok);
    }
};
// FP64 Newton from T0 = min(R/C, (R/K)^(1/4)) with IEEE division and square
// root: the path for cells where FP32 cannot seed the root (C, K or R outside
// FP32's range, an FP32 iteration that overflowed, produced a NaN or did not
// converge).  From T0, at or right of the root, Newton decreases monotonically.
// ok: converged to |dT| <= 1e-15 T within 60 steps, with T finite and positive.
static __device__ __noinline__ double newton_quartic_f64(double C, double K, double Rr, bool& ok)
{
    double T = Rr / C;
    if (K > 0.0) T = fmin(T, ::sqrt(::sqrt(Rr / K)));
    ok = false;
    for (int it = 0; it < 60; ++it) {
        const double T3 = T * T * T;
        const double g = fma(K, T3 * T, C * T) - Rr;
        const double dg = fma(4.0 * K, T3, C);
        const double dT = g / dg;
        T -= dT;
        if (fabs(dT) <= 1e-15 * T) { ok = true; break; }
    }
    ok = ok && isfinite(T) && T > 0.0;
    return T;
}

template <> struct Quartic<double> {
    __device__ static double solve(double C, double K, double Rr, bool& ok)
    {
        bool ok32;
        const float T32 = newton_quartic_f32(narrow(C), narrow(K), narrow(Rr), ok32);
        // FP32 seeds only a finite positive root that its iteration reached;
        // every comparison below is false for a NaN, which takes the FP64 path
        if (!(ok32 && T32 > 0.0f && T32 <= FLT_MAX)) return newton_quartic_f64(C, K, Rr, ok);
        double T = widen(T32);
        // One step of Halley's method (cubically convergent):
        // T <- T - 2 g g' / (2 g'^2 - g g'') = T - g g' / (g'^2 - 6 K T^2 g),
        // g' = C + 4 K T^3, g'' = 12 K T^2.  From the FP32 root (relative
        // error near 1e-7) it lands at FP64 rounding.  The quotient needs only
        // ~1e-14 relative accuracy (it multiplies a correction of ~1e-7 T):
        // FP32 reciprocal estimate of the denominator plus one FP64 Newton step,
        // or an FP64 division where the denominator is outside FP32's normal
        // range (g'^2 overflows FP32 for K T^3 above ~1e19).
        const double T2 = T * T;
        const double KT2 = K * T2;
        const double g = fma(KT2, T2, fma(C, T, -Rr));
        const double d1 = fma(4.0 * KT2, T, C);
        const double den = fma(d1, d1, -(6.0 * KT2) * g);
        const float den32 = narrow(den);
        const float denf = fabsf(den32);
        double r;
        if (denf >= FLT_MIN && denf <= FLT_MAX) {
            r = widen(Fm<float>::rcp(den32));
            r = fma(r, fma(-den, r, 1.0), r);
        } else {
            r = 1.0 / den;
        }
        const double dT = g * d1 * r;
        T -= dT;
        // the FP32 start was not close enough for one cubic step (or the step
        // is not a number): FP64 Newton from the FP64 start
        if (!(fabs(dT) <= 1e-6 * T)) return newton_quartic_f64(C, K, Rr, ok);
        ok = true;
        return T;
    }
};

// Local solve D^{-1} of one cell with the backward-Euler sources:
//   (w0 + w1 diag) E + w1 ka (E - a_r T^4)   = bE
//   (w0 + w1 (diag + kt)) F                  = bF
//   (w0 + w1 C_v) T - w1 ka (E - a_r T^4)    = bT
// (w0, w1) = (0, 1): fine-level Jacobi (Algorithm 1); (1, dtau): implicit
// pseudo-time step (Eq. (30)).  E is eliminated; the quartic in T is solved by
// Newton; E follows.  Without absorption the T equation is linear.
template <typename R>
__device__ __forceinline__ Cell4<R> local_solve(R w0, R w1, R diag, R ka, R kt, R c_v, R a_r,
                                                R bE, R bFx, R bFy, R bT, bool& ok)
{
    Cell4<R> o;
    R A = w0 + w1 * diag;
    R k = w1 * ka;
    R C = w0 + w1 * c_v;
    ok = true;
    bool k0;
    if constexpr (sizeof(R) == 8) k0 = is_zero_f64(k);
    else k0 = k == R(0);
    if (k0) {
        const R iF = Fm<R>::rcp(w0 + w1 * (diag + kt));
        o.Fx = bFx * iF;
        o.Fy = bFy * iF;
        o.T = bT / C;
        o.E = bE / A;
        return o;
    }
    // one reciprocal serves both denominators: 1/a = b / (a b), 1/b = a / (a b)
    const R dF = w0 + w1 * (diag + kt), dE = A + k;
    const R ip = Fm<R>::rcp(dF * dE);
    const R iF = dE * ip, iAk = dF * ip;
    o.Fx = bFx * iF;
    o.Fy = bFy * iF;
    // with kk = k / (A + k): K = kk A a_r, R = bT + kk bE,
    // E = (bE + k a_r T^4) / (A + k) = bE / (A + k) + kk a_r T^4
    const R kk = k * iAk;
    const R K = (A * a_r) * kk;
    const R Rr = fma(kk, bE, bT);
    const R T = Quartic<R>::solve(C, K, Rr, ok);
    const R T2 = T * T;
    o.T = T;
    o.E = fma(a_r * kk, T2 * T2, bE * iAk);
    return o;
}


// ---------------------------------------------------------------------------
// Correction form (mixed precision).  The FP32 cycle carries a correction e
// around a base state w and evaluates differences A(w + e) - A(w) directly,
// with every term of size O(e), so that FP32 rounding is relative to |e| and
// not to |w| (a subtraction u32 - w32 would lose the correction to the
// rounding of the full state).

// P(w + e) - P(w) for the closure of Eq. (5) written as
// P = E a I + (q / c^2) E phi phi^T, phi = F / E, a = (s - 1)/3, q = 3/(2 + s),
// s = sqrt(4 - 3 f^2), f^2 = |phi|^2 / c^2, using
//   d phi = (e_F - phi0 e_E) / E1,  d(f^2) = d phi . (phi0 + phi1) / c^2,
//   d s = -3 d(f^2) / (s0 + s1),  d q = -3 d s / ((2 + s0)(2 + s1)).
template <typename R>
__device__ __forceinline__ void closure_delta(R wE, R wFx, R wFy, R eE, R eFx, R eFy, R inv_c2,
                                              R& dPxx, R& dPxy, R& dPyy)
{
    const R E1 = wE + eE;
    const R iE0 = Fm<R>::rcp(wE), iE1 = Fm<R>::rcp(E1);
    const R px0 = wFx * iE0, py0 = wFy * iE0;
    const R dpx = (eFx - px0 * eE) * iE1, dpy = (eFy - py0 * eE) * iE1;
    const R px1 = px0 + dpx, py1 = py0 + dpy;
    const R f20 = (px0 * px0 + py0 * py0) * inv_c2;
    const R df2 = (dpx * (px0 + px1) + dpy * (py0 + py1)) * inv_c2;
    const R f21 = f20 + df2;
    const R c0 = f20 < R(1) ? f20 : R(1), c1 = f21 < R(1) ? f21 : R(1);
    const R dc = (f20 <= R(1) && f21 <= R(1)) ? df2 : c1 - c0;
    const R s0 = Fm<R>::sqrt(R(4) - R(3) * c0), s1 = Fm<R>::sqrt(R(4) - R(3) * c1);
    const R ds = R(-3) * dc * Fm<R>::rcp(s0 + s1);
    const R a1 = (s1 - R(1)) * (R(1) / R(3)), da = ds * (R(1) / R(3));
    const R i20 = Fm<R>::rcp(R(2) + s0), i21 = Fm<R>::rcp(R(2) + s1);
    const R q0 = R(3) * i20;
    const R dq = R(-3) * ds * i20 * i21;
    const R iso = eE * a1 + wE * da;
    dPxx = iso + inv_c2 * (dq * E1 * px1 * px1 + q0 * (eE * px1 * px1 + wE * dpx * (px0 + px1)));
    dPyy = iso + inv_c2 * (dq * E1 * py1 * py1 + q0 * (eE * py1 * py1 + wE * dpy * (py0 + py1)));
    dPxy = inv_c2 * (dq * E1 * px1 * py1 + q0 * (eE * px1 * py1 + wE * (dpx * py1 + px0 * dpy)));
}

// (T + x)^4 - T^4 = x (4 T^3 + 6 T^2 x + 4 T x^2 + x^3), without cancellation.
template <typename R>
__device__ __forceinline__ R quartic_delta(R T, R x)
{
    return x * (R(4) * T * T * T + x * (R(6) * T * T + x * (R(4) * T + x)));
}

// The local solve of `local_solve` for the correction (e_E, e_F, x = e_T) of a
// base cell with temperature T:
//   (w0 + w1 diag) e_E + w1 ka (e_E - a_r dT4)  = bE,  dT4 = (T + x)^4 - T^4
//   (w0 + w1 (diag + kt)) e_F                   = bF
//   (w0 + w1 C_v) x - w1 ka (e_E - a_r dT4)     = bT
// Eliminating e_E leaves h(x) = C x + K dT4(x) - R = 0, increasing and convex
// for T + x > 0; Newton from x = 0 lands right of the root after one step and
// then decreases monotonically.
template <typename R>
__device__ __forceinline__ Cell4<R> local_solve_delta(R w0, R w1, R diag, R ka, R kt, R c_v,
                                                      R a_r, R T, R bE, R bFx, R bFy, R bT,
                                                      bool& ok)
{
    Cell4<R> o;
    const R A = w0 + w1 * diag;
    const R k = w1 * ka;
    const R iF = Fm<R>::rcp(w0 + w1 * (diag + kt));
    o.Fx = bFx * iF;
    o.Fy = bFy * iF;
    const R C = w0 + w1 * c_v;
    ok = true;
    if (k == R(0)) {
        o.T = bT / C;
        o.E = bE / A;
        return o;
    }
    const R iAk = Fm<R>::rcp(A + k);
    const R K = k * A * a_r * iAk;
    const R Rr = bT + k * bE * iAk;
    R x = R(0);
    ok = false;
    for (int it = 0; it < 40; ++it) {
        const R Tx = T + x;
        const R h = C * x + K * quartic_delta(T, x) - Rr;
        const R dh = C + R(4) * K * Tx * Tx * Tx;
        const R dx = h * Fm<R>::rcp(dh);
        x -= dx;
        if (fabs(dx) <= R(1e-6) * fabs(x) || dx == R(0)) { ok = true; break; }
    }
    o.T = x;
    o.E = (bE + k * a_r * quartic_delta(T, x)) * iAk;
    return o;
}

// ---------------------------------------------------------------------------
// Ghost cells: one layer per wall.  periodic: wrap; reflecting: mirror with the
// wall-normal flux negated; Neumann: copy; inflow: the prescribed (E, Fx, Fy)
// with T from the mirror cell.  Differences (kind DIFF) hold zero at inflow
// walls.  A corner resolves the y wall on the cell the x wall points to, then
// applies the x wall on top (the x wall is the outer rule).
// The rules of `fetch` (below) split in two, so that a caller can map several
// ghosts first and issue their loads together: fetch(L, s, i, j, kind) =
// ghost_apply(L, s[g.k], g, kind) with g = ghost_map(L, i, j) (zero for a
// difference at an inflow wall, whatever was loaded).
struct Ghost {
    size_t k;          // index of the source cell
    int i, jo;         // mapped column, original row
    int xrule, yrule;  // BC of the wall crossed (-1: none or periodic)
    int xwall, ywall;
};

template <typename R>
__device__ __forceinline__ Ghost ghost_map(const Level<R>& L, int i, int j)
{
    Ghost g;
    g.jo = j;
    g.xrule = -1; g.xwall = 0; g.yrule = -1; g.ywall = 0;
    if (i < 0 || i >= L.nx) {
        g.xwall = i < 0 ? WALL_W : WALL_E;
        const int bc = L.bc[g.xwall];
        if (bc == BC_PERIODIC) {
            i = i < 0 ? i + L.nx : i - L.nx;
        } else {
            i = i < 0 ? -1 - i : 2 * L.nx - 1 - i;
            g.xrule = bc;
        }
    }
    if (j < 0 || j >= L.ny) {
        g.ywall = j < 0 ? WALL_S : WALL_N;
        const int bc = L.bc[g.ywall];
        if (bc == BC_PERIODIC) {
            j = j < 0 ? j + L.ny : j - L.ny;
        } else {
            j = j < 0 ? -1 - j : 2 * L.ny - 1 - j;
            g.yrule = bc;
        }
    }
    g.i = i;
    g.k = (size_t)j * L.nx + i;
    return g;
}

template <typename R>
__device__ __forceinline__ Cell4<R> ghost_apply(const Level<R>& L, Cell4<R> c, const Ghost& g,
                                                int kind)
{
    if (kind == KIND_DIFF && (g.xrule == BC_INFLOW || g.yrule == BC_INFLOW))
        return Cell4<R>{ R(0), R(0), R(0), R(0) };
    if (g.yrule == BC_REFLECT) c.Fy = -c.Fy;
    if (g.yrule == BC_INFLOW) {
        const R* p = L.inflow + (size_t)(g.ywall * 3) * L.prof_len;
        c.E = p[g.i]; c.Fx = p[L.prof_len + g.i]; c.Fy = p[2 * L.prof_len + g.i];
    }
    if (g.xrule == BC_REFLECT) c.Fx = -c.Fx;
    if (g.xrule == BC_INFLOW) {
        const int jj = g.jo < 0 ? 0 : (g.jo >= L.ny ? L.ny - 1 : g.jo);
        const R* p = L.inflow + (size_t)(g.xwall * 3) * L.prof_len;
        c.E = p[jj]; c.Fx = p[L.prof_len + jj]; c.Fy = p[2 * L.prof_len + jj];
    }
    return c;
}

// (The same rules as ghost_map + ghost_apply, written as one pass: the sweeps'
// code generation is tuned on this form, and splitting it cost the fine FP64
// sweep 3%.)
template <typename R>
__device__ __forceinline__ Cell4<R> fetch(const Level<R>& L, const Cell4<R>* __restrict__ s,
                                          int i, int j, int kind)
{
    const int jo = j;
    int xrule = -1, xwall = 0, yrule = -1, ywall = 0;
    if (i < 0 || i >= L.nx) {
        xwall = i < 0 ? WALL_W : WALL_E;
        int bc = L.bc[xwall];
        if (bc == BC_PERIODIC) {
            i = i < 0 ? i + L.nx : i - L.nx;
        } else {
            i = i < 0 ? -1 - i : 2 * L.nx - 1 - i;
            xrule = bc;
        }
    }
    if (j < 0 || j >= L.ny) {
        ywall = j < 0 ? WALL_S : WALL_N;
        int bc = L.bc[ywall];
        if (bc == BC_PERIODIC) {
            j = j < 0 ? j + L.ny : j - L.ny;
        } else {
            j = j < 0 ? -1 - j : 2 * L.ny - 1 - j;
            yrule = bc;
        }
    }
    if (kind == KIND_DIFF && (xrule == BC_INFLOW || yrule == BC_INFLOW)) {
        Cell4<R> z = { R(0), R(0), R(0), R(0) };
        return z;
    }
    Cell4<R> c = s[(size_t)j * L.nx + i];
    if (yrule == BC_REFLECT) c.Fy = -c.Fy;
    if (yrule == BC_INFLOW) {
        const R* p = L.inflow + (size_t)(ywall * 3) * L.prof_len;
        c.E = p[i]; c.Fx = p[L.prof_len + i]; c.Fy = p[2 * L.prof_len + i];
    }
    if (xrule == BC_REFLECT) c.Fx = -c.Fx;
    if (xrule == BC_INFLOW) {
        int jj = jo < 0 ? 0 : (jo >= L.ny ? L.ny - 1 : jo);
        const R* p = L.inflow + (size_t)(xwall * 3) * L.prof_len;
        c.E = p[jj]; c.Fx = p[L.prof_len + jj]; c.Fy = p[2 * L.prof_len + jj];
    }
    return c;
}

template <typename R>
__device__ __forceinline__ Sig2<R> fetch_sig(const Level<R>& L, const Sig2<R>* __restrict__ s,
                                             int i, int j)
{
    if (i < 0 || i >= L.nx) {
        if (L.bc[i < 0 ? WALL_W : WALL_E] == BC_PERIODIC) i = i < 0 ? i + L.nx : i - L.nx;
        else i = i < 0 ? -1 - i : 2 * L.nx - 1 - i;
    }
    if (j < 0 || j >= L.ny) {
        if (L.bc[j < 0 ? WALL_S : WALL_N] == BC_PERIODIC) j = j < 0 ? j + L.ny : j - L.ny;
        else j = j < 0 ? -1 - j : 2 * L.ny - 1 - j;
    }
    return s[(size_t)j * L.nx + i];
}

}  // namespace m1
