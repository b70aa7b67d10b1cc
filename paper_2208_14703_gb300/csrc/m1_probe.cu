// Arithmetic peak probe: the issue rate of fused multiply-adds on this GPU, the
// denominator of the roofline of the FP64 kernels (their bound is the FP64
// pipe, not HBM).
//
// Each thread runs kChains independent FMA recurrences x <- x a + b (no chain
// waits on another, so the pipe, not the FMA latency, limits the rate) for
// `iters` rounds, unrolled by kUnroll.  With 0 < a < 1 and b > 0 the values
// stay near b / (1 - a): no overflow, no subnormals.  Every thread stores its
// sum, so the compiler cannot drop the work.  A launch is 152 x 8 blocks of 256
// threads; the count of FMA instructions per launch (summed over lanes) is
// blocks x threads x kChains x iters.
//
// Also here: m1_op_elementwise, which runs the kernels' inline per-element
// arithmetic (the FP64 reciprocal and square root, the FP32 approximations,
// the double-word split and the FP32 -> FP64 widening) on caller data, so that
// tests can hold it against correctly rounded results.
#include <m1.h>

#include <algorithm>
#include <cstdio>
#include <vector>

#include <cuda_runtime.h>

#include "m1_device.cuh"
#include "m1_dw.cuh"

namespace m1 {
void set_error_text(const char* msg);   // m1_api.cu: the text m1_last_error returns
}

namespace {

constexpr int kChains = 8, kUnroll = 16;
constexpr int kBlocks = 152 * 8, kThreadsPerBlock = 256, kIters = 4096;

template <typename R>
__global__ void __launch_bounds__(kThreadsPerBlock) k_fma_peak(R* out, int iters, R a, R b)
{
    R x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = R(threadIdx.x + c) * R(1e-3);
    for (int it = 0; it < iters; it += kUnroll) {
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
#pragma unroll
            for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
        }
    }
    R s = R(0);
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <typename R>
m1_status probe(cudaStream_t s, int reps, double* ops_per_s)
{
    R* out = nullptr;
    cudaEvent_t a = nullptr, b = nullptr;
    std::vector<float> ms;
    m1_status st = M1_OK;
    auto fail = [&](const char* what, cudaError_t e) {
        char msg[256];
        std::snprintf(msg, sizeof(msg), "m1_probe_fma_peak: %s: %s", what, cudaGetErrorString(e));
        m1::set_error_text(msg);
        st = M1_ERR_CUDA;
    };
    cudaError_t e = cudaMalloc(&out, sizeof(R) * kBlocks * kThreadsPerBlock);
    if (e != cudaSuccess) { fail("cudaMalloc", e); return st; }
    if ((e = cudaEventCreate(&a)) != cudaSuccess || (e = cudaEventCreate(&b)) != cudaSuccess) {
        fail("cudaEventCreate", e);
    } else {
        const R fa = R(0.999999), fb = R(1e-6);
        for (int r = 0; r <= reps && st == M1_OK; ++r) {   // launch 0 warms up
            if ((e = cudaEventRecord(a, s)) != cudaSuccess) { fail("cudaEventRecord", e); break; }
            k_fma_peak<R><<<kBlocks, kThreadsPerBlock, 0, s>>>(out, kIters, fa, fb);
            if ((e = cudaGetLastError()) != cudaSuccess) { fail("launch", e); break; }
            if ((e = cudaEventRecord(b, s)) != cudaSuccess) { fail("cudaEventRecord", e); break; }
            if ((e = cudaEventSynchronize(b)) != cudaSuccess) { fail("cudaEventSynchronize", e); break; }
            float t = 0.f;
            if ((e = cudaEventElapsedTime(&t, a, b)) != cudaSuccess) { fail("elapsed time", e); break; }
            if (r > 0) ms.push_back(t);
        }
    }
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
    cudaFree(out);
    if (st != M1_OK) return st;
    std::sort(ms.begin(), ms.end());
    const double med = ms[ms.size() / 2];
    const double ops = (double)kBlocks * kThreadsPerBlock * kChains * kIters;
    *ops_per_s = ops / (med * 1e-3);
    return M1_OK;
}

}  // namespace

namespace {

template <int FN>
__global__ void __launch_bounds__(256) k_elementwise(const void* __restrict__ x, long long n,
                                                     void* __restrict__ y)
{
    const long long step = (long long)gridDim.x * blockDim.x;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += step) {
        if constexpr (FN == M1_FN_RCP64) {
            ((double*)y)[i] = m1::Fm<double>::rcp(((const double*)x)[i]);
        } else if constexpr (FN == M1_FN_SQRT64) {
            ((double*)y)[i] = m1::Fm<double>::sqrt(((const double*)x)[i]);
        } else if constexpr (FN == M1_FN_RCP32) {
            ((float*)y)[i] = m1::Fm<float>::rcp(((const float*)x)[i]);
        } else if constexpr (FN == M1_FN_SQRT32) {
            ((float*)y)[i] = m1::Fm<float>::sqrt(((const float*)x)[i]);
        } else if constexpr (FN == M1_FN_DW_SPLIT) {
            const m1::DW d = m1::dw_split(((const double*)x)[i]);
            ((float2*)y)[i] = make_float2(d.hi, d.lo);
        } else {
            ((double*)y)[i] = m1::widen(((const float*)x)[i]);
        }
    }
}

template <int FN>
cudaError_t launch_elementwise(const void* x, long long n, void* y, cudaStream_t s)
{
    const long long blocks = std::min<long long>((n + 255) / 256, 152LL * 16);
    k_elementwise<FN><<<(int)std::max<long long>(blocks, 1), 256, 0, s>>>(x, n, y);
    return cudaGetLastError();
}

}  // namespace

extern "C" m1_status m1_op_elementwise(int fn, const void* x, long long n, void* y,
                                       void* cuda_stream)
{
    if (n < 0 || (n > 0 && (!x || !y)) || fn < M1_FN_RCP64 || fn > M1_FN_WIDEN)
        return M1_ERR_INVALID_ARG;
    if (n == 0) return M1_OK;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    cudaError_t e = cudaSuccess;
    switch (fn) {
    case M1_FN_RCP64: e = launch_elementwise<M1_FN_RCP64>(x, n, y, s); break;
    case M1_FN_SQRT64: e = launch_elementwise<M1_FN_SQRT64>(x, n, y, s); break;
    case M1_FN_RCP32: e = launch_elementwise<M1_FN_RCP32>(x, n, y, s); break;
    case M1_FN_SQRT32: e = launch_elementwise<M1_FN_SQRT32>(x, n, y, s); break;
    case M1_FN_DW_SPLIT: e = launch_elementwise<M1_FN_DW_SPLIT>(x, n, y, s); break;
    default: e = launch_elementwise<M1_FN_WIDEN>(x, n, y, s); break;
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        m1::set_error_text(cudaGetErrorString(e));
        return M1_ERR_CUDA;
    }
    return M1_OK;
}

extern "C" m1_status m1_probe_fma_peak(int precision, void* cuda_stream, int reps,
                                       double* ops_per_s)
{
    if (!ops_per_s || reps < 1) return M1_ERR_INVALID_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    if (precision == M1_FP64) return probe<double>(s, reps, ops_per_s);
    if (precision == M1_MIXED) return probe<float>(s, reps, ops_per_s);
    return M1_ERR_INVALID_ARG;
}
