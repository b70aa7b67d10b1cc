// Single-level operators of a 3D grid: A(u), b - A(u) and Jacobi sweeps of
// A(u) = b (Eq. (12), Eq. (13), Algorithm 1 with the Rusanov faces of Eq. (6)
// and the closure of Eq. (5) on three axes; the [EXT] sources and local E-T
// solve of the 2D path).  The first GPU step of the 3D extension: the multigrid
// cycle in 3D is not built yet.
//
// FP64 is what bounds these kernels on GB300 (two FP64 operations per clock per
// SM), so a cell's closure is evaluated once per sweep: a first pass writes the
// pressure tensor P of every cell, the second pass reads the six neighbours'
// (E, F) and P instead of re-evaluating six closures per cell.  The tensor costs
// 48 bytes per cell of traffic, far inside the bandwidth an FP64-bound kernel
// leaves unused.
#include <m1.h>

#include <cstdio>

#include "m1_device.cuh"

namespace m1 {
void set_err(cudaError_t e, const char* what);
void set_error_text(const char* msg);
}

namespace {

using m1::Fm;
using m1::Quartic;
using m1::Sig2;

struct alignas(32) EF { double E, F[3]; };                       // energy and flux of a cell
struct P6 { double xx, xy, xz, yy, yz, zz; };                    // symmetric pressure tensor

struct G3 {
    int n[3];
    int bc[6];
    double c, a_r, c_v, ic2, diag, cdt;
    double beta[3];                                              // dt / (2 h_d)
};

constexpr int kThreads3 = 256;
constexpr int kMaxBlocks3 = 152 * 8;

__device__ __forceinline__ double P_at(const P6& p, int a, int b)
{
    if (a > b) { const int t = a; a = b; b = t; }
    if (a == 0) return b == 0 ? p.xx : (b == 1 ? p.xy : p.xz);
    if (a == 1) return b == 1 ? p.yy : p.yz;
    return p.zz;
}

// Eq. (5) in the algebraically equal form of the 2D path:
// P = E (s - 1)/3 I + 3/(2 + s) F F^T / (c^2 E), s = sqrt(4 - 3 f^2), f^2 clamped to 1.
__device__ __forceinline__ P6 closure3(const EF& u, double ic2)
{
    const double iE = Fm<double>::rcp(u.E);
    const double px = u.F[0] * iE, py = u.F[1] * iE, pz = u.F[2] * iE;
    double a = fma(fma(pz, pz, fma(py, py, px * px)), -3.0 * ic2, 4.0);
    a = a > 1.0 ? a : 1.0;
    const double s = Fm<double>::sqrt(a);
    const double Eiso = u.E * fma(s, 1.0 / 3.0, -1.0 / 3.0);
    const double q = Fm<double>::rcp(2.0 + s) * (3.0 * ic2);
    const double qx = q * px, qy = q * py, qz = q * pz;
    return P6{ fma(qx, u.F[0], Eiso), qx * u.F[1], qx * u.F[2],
               fma(qy, u.F[1], Eiso), qy * u.F[2], fma(qz, u.F[2], Eiso) };
}

__global__ void k_closure3(G3 g, const EF* __restrict__ u, P6* __restrict__ P, size_t n)
{
    for (size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x; q < n;
         q += (size_t)gridDim.x * blockDim.x)
        P[q] = closure3(u[q], g.ic2);
}

// The face neighbour of cell (i, j, k) across axis d on side `side` (-1 / +1),
// with the wall rules: periodic wrap, reflecting mirror with the wall-normal
// flux negated (and the tensor's entries that pair the normal with another axis
// negated, as the closure of the mirrored state gives), Neumann copy.
__device__ __forceinline__ void neighbour3(const G3& g, const EF* __restrict__ u,
                                           const P6* __restrict__ P, int i, int j, int k, int d,
                                           int side, EF& nb, P6& pn)
{
    int p[3] = { i, j, k };
    p[d] += side;
    bool flip = false;
    if (p[d] < 0 || p[d] >= g.n[d]) {
        const int bc = g.bc[2 * d + (side < 0 ? 0 : 1)];
        if (bc == m1::BC_PERIODIC) {
            p[d] = p[d] < 0 ? p[d] + g.n[d] : p[d] - g.n[d];
        } else {
            p[d] = p[d] < 0 ? -1 - p[d] : 2 * g.n[d] - 1 - p[d];
            flip = bc == m1::BC_REFLECT;
        }
    }
    const size_t q = ((size_t)p[2] * g.n[1] + p[1]) * g.n[0] + p[0];
    nb = u[q];
    pn = P[q];
    if (flip) {
        nb.F[d] = -nb.F[d];
        if (d == 0) { pn.xy = -pn.xy; pn.xz = -pn.xz; }
        else if (d == 1) { pn.xy = -pn.xy; pn.yz = -pn.yz; }
        else { pn.xz = -pn.xz; pn.yz = -pn.yz; }
    }
}

enum { OP3_APPLY = 0, OP3_RESIDUAL = 1, OP3_JACOBI = 2 };

// One cell-parallel pass: the neighbour terms of Eq. (9) on the three axes, then
// A(u) = D(u) - N (APPLY), b - A(u) (RESIDUAL), or the Jacobi update
// D^{-1}(b + N) (JACOBI, the local E-T solve of the 2D path with three flux
// components).
template <int MODE>
__global__ void __launch_bounds__(kThreads3) k_op3(G3 g, const EF* __restrict__ u,
                                                   const double* __restrict__ T,
                                                   const P6* __restrict__ P,
                                                   const Sig2<double>* __restrict__ sig,
                                                   const EF* __restrict__ b,
                                                   const double* __restrict__ bT,
                                                   EF* __restrict__ out,
                                                   double* __restrict__ outT, size_t n)
{
    const double c = g.c;
    for (size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x; q < n;
         q += (size_t)gridDim.x * blockDim.x) {
        const int i = (int)(q % g.n[0]);
        const int j = (int)((q / g.n[0]) % g.n[1]);
        const int k = (int)(q / ((size_t)g.n[0] * g.n[1]));
        double N[4] = { 0.0, 0.0, 0.0, 0.0 };
        for (int d = 0; d < 3; ++d)
            for (int side = -1; side <= 1; side += 2) {
                EF nb;
                P6 pn;
                neighbour3(g, u, P, i, j, k, d, side, nb, pn);
                const double sg = side < 0 ? 1.0 : -1.0, bd = g.beta[d];
                N[0] += bd * (c * nb.E + sg * nb.F[d]);
                for (int a = 0; a < 3; ++a) N[1 + a] += c * bd * (nb.F[a] + sg * c * P_at(pn, d, a));
            }
        const Sig2<double> s = sig[q];
        const double ka = g.cdt * s.sa, kt = g.cdt * (s.sa + s.ss);
        const EF uc = u[q];
        const double Tc = T[q];
        if (MODE != OP3_JACOBI) {
            const double T2 = Tc * Tc;
            const double src = ka * (uc.E - g.a_r * T2 * T2);
            EF a;
            a.E = g.diag * uc.E + src - N[0];
            for (int m = 0; m < 3; ++m) a.F[m] = (g.diag + kt) * uc.F[m] - N[1 + m];
            double aT = g.c_v * Tc - src;
            if (MODE == OP3_RESIDUAL) {
                const EF bb = b[q];
                a.E = bb.E - a.E;
                for (int m = 0; m < 3; ++m) a.F[m] = bb.F[m] - a.F[m];
                aT = bT[q] - aT;
            }
            out[q] = a;
            outT[q] = aT;
        } else {
            const EF bb = b[q];
            const double bE = bb.E + N[0], bTq = bT[q];
            EF o;
            double oT;
            if (ka == 0.0) {
                const double iF = Fm<double>::rcp(g.diag + kt);
                for (int m = 0; m < 3; ++m) o.F[m] = (bb.F[m] + N[1 + m]) * iF;
                oT = bTq / g.c_v;
                o.E = bE / g.diag;
            } else {
                // one reciprocal for both denominators, as in the 2D local solve
                const double dF = g.diag + kt, dE = g.diag + ka;
                const double ip = Fm<double>::rcp(dF * dE);
                const double iF = dE * ip, iAk = dF * ip;
                for (int m = 0; m < 3; ++m) o.F[m] = (bb.F[m] + N[1 + m]) * iF;
                const double kk = ka * iAk;
                const double K = (g.diag * g.a_r) * kk;
                const double R = fma(kk, bE, bTq);
                bool ok;
                oT = Quartic<double>::solve(g.c_v, K, R, ok);
                const double T2 = oT * oT;
                o.E = fma(g.a_r * kk, T2 * T2, bE * iAk);
            }
            out[q] = o;
            outT[q] = oT;
        }
    }
}

__global__ void k_pack3(const double* __restrict__ planes, EF* __restrict__ ef,
                        double* __restrict__ T, size_t n)
{
    for (size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x; q < n;
         q += (size_t)gridDim.x * blockDim.x) {
        EF e;
        e.E = planes[q];
        e.F[0] = planes[n + q];
        e.F[1] = planes[2 * n + q];
        e.F[2] = planes[3 * n + q];
        ef[q] = e;
        T[q] = planes[4 * n + q];
    }
}

__global__ void k_unpack3(const EF* __restrict__ ef, const double* __restrict__ T,
                          double* __restrict__ planes, size_t n)
{
    for (size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x; q < n;
         q += (size_t)gridDim.x * blockDim.x) {
        const EF e = ef[q];
        planes[q] = e.E;
        planes[n + q] = e.F[0];
        planes[2 * n + q] = e.F[1];
        planes[3 * n + q] = e.F[2];
        planes[4 * n + q] = T[q];
    }
}

__global__ void k_pack_sig3(const double* __restrict__ planes, Sig2<double>* __restrict__ s,
                            size_t n)
{
    for (size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x; q < n;
         q += (size_t)gridDim.x * blockDim.x)
        s[q] = Sig2<double>{ planes[q], planes[n + q] };
}

// Device buffers of one call, freed on every return path.
struct Buffers {
    void* p[12] = {};
    int count = 0;
    ~Buffers()
    {
        for (int k = 0; k < count; ++k)
            if (p[k]) cudaFree(p[k]);
    }
    template <typename T>
    cudaError_t get(T** out, size_t bytes)
    {
        void* q = nullptr;
        const cudaError_t e = cudaMalloc(&q, bytes);
        if (e == cudaSuccess) p[count++] = q;
        *out = static_cast<T*>(q);
        return e;
    }
};

struct Events {
    cudaEvent_t e[2] = { nullptr, nullptr };
    ~Events()
    {
        for (auto x : e)
            if (x) cudaEventDestroy(x);
    }
};

int blocks3(size_t n)
{
    const size_t b = (n + kThreads3 - 1) / kThreads3;
    return (int)(b < (size_t)kMaxBlocks3 ? (b > 0 ? b : 1) : kMaxBlocks3);
}

}  // namespace

#define M1_CK3(call)                                                                               \
    do {                                                                                           \
        cudaError_t e_ = (call);                                                                   \
        if (e_ != cudaSuccess) {                                                                   \
            ::m1::set_err(e_, #call);                                                              \
            return e_ == cudaErrorMemoryAllocation ? M1_ERR_OOM : M1_ERR_CUDA;                     \
        }                                                                                          \
    } while (0)

extern "C" m1_status m1_op_level3(const m1_grid3_desc* d, double dt, const double* sig,
                                  const double* state, const double* rhs, int mode, int sweeps,
                                  double* out, int on_device, void* cuda_stream, double* ms)
{
    if (!d || !sig || !state || !out || !(dt > 0)) return M1_ERR_INVALID_ARG;
    if (mode != M1_OP3_APPLY && mode != M1_OP3_RESIDUAL && mode != M1_OP3_JACOBI)
        return M1_ERR_INVALID_ARG;
    if (mode != M1_OP3_APPLY && !rhs) return M1_ERR_INVALID_ARG;
    if (mode == M1_OP3_JACOBI && sweeps < 1) return M1_ERR_INVALID_ARG;
    if (d->nx < 1 || d->ny < 1 || d->nz < 1 || !(d->lx > 0) || !(d->ly > 0) || !(d->lz > 0) ||
        !(d->c > 0) || !(d->a_r > 0) || !(d->c_v > 0))
        return M1_ERR_INVALID_ARG;
    for (int w = 0; w < 6; ++w)
        if (d->bc[w] != M1_BC_PERIODIC && d->bc[w] != M1_BC_REFLECT && d->bc[w] != M1_BC_NEUMANN)
            return M1_ERR_INVALID_ARG;
    const size_t n = (size_t)d->nx * d->ny * d->nz;
    if (n > ((size_t)1 << 31)) return M1_ERR_INVALID_ARG;

    G3 g{};
    g.n[0] = d->nx; g.n[1] = d->ny; g.n[2] = d->nz;
    for (int w = 0; w < 6; ++w) g.bc[w] = (int)d->bc[w];
    const double h[3] = { d->lx / d->nx, d->ly / d->ny, d->lz / d->nz };
    g.c = d->c; g.a_r = d->a_r; g.c_v = d->c_v;
    g.ic2 = 1.0 / (d->c * d->c);
    g.cdt = d->c * dt;
    g.diag = 1.0 + d->c * dt / h[0] + d->c * dt / h[1] + d->c * dt / h[2];
    for (int a = 0; a < 3; ++a) g.beta[a] = dt / (2.0 * h[a]);

    const cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    Buffers buf;
    EF *u0 = nullptr, *u1 = nullptr, *b = nullptr;
    double *T0 = nullptr, *T1 = nullptr, *bT = nullptr, *stage = nullptr;
    P6* P = nullptr;
    Sig2<double>* sg = nullptr;
    M1_CK3(buf.get(&u0, n * sizeof(EF)));
    M1_CK3(buf.get(&u1, n * sizeof(EF)));
    M1_CK3(buf.get(&T0, n * sizeof(double)));
    M1_CK3(buf.get(&T1, n * sizeof(double)));
    M1_CK3(buf.get(&P, n * sizeof(P6)));
    M1_CK3(buf.get(&sg, n * sizeof(Sig2<double>)));
    if (rhs) {
        M1_CK3(buf.get(&b, n * sizeof(EF)));
        M1_CK3(buf.get(&bT, n * sizeof(double)));
    }
    if (!on_device) M1_CK3(buf.get(&stage, 5 * n * sizeof(double)));

    const int nb = blocks3(n);
    // caller planes -> device layout
    auto pack = [&](const double* src, EF* ef, double* T) -> cudaError_t {
        const double* planes = src;
        if (!on_device) {
            const cudaError_t e = cudaMemcpyAsync(stage, src, 5 * n * sizeof(double),
                                                  cudaMemcpyHostToDevice, s);
            if (e != cudaSuccess) return e;
            planes = stage;
        }
        k_pack3<<<nb, kThreads3, 0, s>>>(planes, ef, T, n);
        return cudaGetLastError();
    };
    M1_CK3(pack(state, u0, T0));
    if (rhs) M1_CK3(pack(rhs, b, bT));
    {
        const double* planes = sig;
        if (!on_device) {
            M1_CK3(cudaMemcpyAsync(stage, sig, 2 * n * sizeof(double), cudaMemcpyHostToDevice, s));
            planes = stage;
        }
        k_pack_sig3<<<nb, kThreads3, 0, s>>>(planes, sg, n);
        M1_CK3(cudaGetLastError());
    }

    Events ev;
    if (ms) {
        M1_CK3(cudaEventCreate(&ev.e[0]));
        M1_CK3(cudaEventCreate(&ev.e[1]));
        M1_CK3(cudaEventRecord(ev.e[0], s));
    }
    EF* cur = u0;
    double* curT = T0;
    EF* nxt = u1;
    double* nxtT = T1;
    const int passes = mode == M1_OP3_JACOBI ? sweeps : 1;
    for (int it = 0; it < passes; ++it) {
        k_closure3<<<nb, kThreads3, 0, s>>>(g, cur, P, n);
        if (mode == M1_OP3_APPLY)
            k_op3<OP3_APPLY><<<nb, kThreads3, 0, s>>>(g, cur, curT, P, sg, b, bT, nxt, nxtT, n);
        else if (mode == M1_OP3_RESIDUAL)
            k_op3<OP3_RESIDUAL><<<nb, kThreads3, 0, s>>>(g, cur, curT, P, sg, b, bT, nxt, nxtT, n);
        else
            k_op3<OP3_JACOBI><<<nb, kThreads3, 0, s>>>(g, cur, curT, P, sg, b, bT, nxt, nxtT, n);
        M1_CK3(cudaGetLastError());
        EF* t = cur; cur = nxt; nxt = t;
        double* tt = curT; curT = nxtT; nxtT = tt;
    }
    if (ms) M1_CK3(cudaEventRecord(ev.e[1], s));

    // device layout -> caller planes
    double* dst = on_device ? out : stage;
    k_unpack3<<<nb, kThreads3, 0, s>>>(cur, curT, dst, n);
    M1_CK3(cudaGetLastError());
    if (!on_device)
        M1_CK3(cudaMemcpyAsync(out, stage, 5 * n * sizeof(double), cudaMemcpyDeviceToHost, s));
    M1_CK3(cudaStreamSynchronize(s));
    if (ms) {
        float t = 0.f;
        M1_CK3(cudaEventElapsedTime(&t, ev.e[0], ev.e[1]));
        *ms = t;
    }
    return M1_OK;
}
