// m1_residual_norm_noalloc: the residual norm ||b - A(v)|| of caller-owned
// device arrays, computed without allocating any device memory.
//
// Who needs it: callers that cannot call cudaMalloc at the point where they
// want the norm -- a framework that hands every byte of device memory to its
// own pool, or a latency-critical loop in which a cudaMalloc (which may
// synchronise the whole device) is not allowed.  Such a caller supplies the
// inputs and the output slot; the per-tile partial sums that the norm needs
// live in a fixed array in this library's own device memory instead.
//
// The scratch: kNoallocPartials doubles (512 KiB) in file-scope __device__
// memory.  Every GPU that loads the library holds it until the process exits.
// All calls share it: a call overwrites the entries it uses before reading them
// (nothing has to start at zero), and two calls whose kernels overlap on the
// GPU (different streams, no ordering) race on it.
#include <m1.h>

#include <cstdio>
#include <mutex>

#include "m1_device.cuh"

namespace m1 {
void set_error_text(const char* msg);   // m1_api.cu: the text m1_last_error returns
}

namespace {

constexpr int kNoallocPartials = 65536;   // tiles: 2D up to 4096 x 4096 cells

static __device__ __align__(256) double g_noalloc_partials[kNoallocPartials];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
double* g_scratch[kMaxDevices] = {};      // device address of the array, per device


using m1::Cell4;
using m1::Level;
using m1::set_error_text;

// Ghost rules of the library (periodic wrap, reflect with the wall-normal flux
// negated, Neumann copy, inflow prescribed E/Fx/Fy with T from the mirror cell),
// read from planar arrays state[4][n] and inflow[4 walls][3][prof_len].
__device__ __forceinline__ Cell4<double> fetch_planar(const Level<double>& L,
                                                      const double* __restrict__ s,
                                                      const double* __restrict__ inflow, int i,
                                                      int j)
{
    const int jo = j;
    int xrule = -1, xwall = 0, yrule = -1, ywall = 0;
    if (i < 0 || i >= L.nx) {
        xwall = i < 0 ? m1::WALL_W : m1::WALL_E;
        const int bc = L.bc[xwall];
        if (bc == m1::BC_PERIODIC) i = i < 0 ? i + L.nx : i - L.nx;
        else { i = i < 0 ? -1 - i : 2 * L.nx - 1 - i; xrule = bc; }
    }
    if (j < 0 || j >= L.ny) {
        ywall = j < 0 ? m1::WALL_S : m1::WALL_N;
        const int bc = L.bc[ywall];
        if (bc == m1::BC_PERIODIC) j = j < 0 ? j + L.ny : j - L.ny;
        else { j = j < 0 ? -1 - j : 2 * L.ny - 1 - j; yrule = bc; }
    }
    const size_t n = (size_t)L.n, k = (size_t)j * L.nx + i;
    Cell4<double> c = { s[k], s[n + k], s[2 * n + k], s[3 * n + k] };
    if (yrule == m1::BC_REFLECT) c.Fy = -c.Fy;
    if (yrule == m1::BC_INFLOW) {
        const double* p = inflow + (size_t)(ywall * 3) * L.prof_len;
        c.E = p[i]; c.Fx = p[L.prof_len + i]; c.Fy = p[2 * L.prof_len + i];
    }
    if (xrule == m1::BC_REFLECT) c.Fx = -c.Fx;
    if (xrule == m1::BC_INFLOW) {
        const int jj = jo < 0 ? 0 : (jo >= L.ny ? L.ny - 1 : jo);
        const double* p = inflow + (size_t)(xwall * 3) * L.prof_len;
        c.E = p[jj]; c.Fx = p[L.prof_len + jj]; c.Fy = p[2 * L.prof_len + jj];
    }
    return c;
}

// Per tile (32 x 8 cells in 2D, 256 in 1D, as the library's residual kernel):
// r = b - A(v) per cell and the tile's sum of h^d (rE^2 + |rF|^2/c^2 + rT^2),
// written to partials[tile].  The closure is evaluated per neighbour here (no
// shared-memory staging): this variant trades speed for having no state.
__global__ void __launch_bounds__(m1::kThreads)
k_residual_partials_planar(Level<double> L, const double* __restrict__ state,
                           const double* __restrict__ rhs, const double* __restrict__ sig,
                           const double* __restrict__ inflow, double* __restrict__ partials)
{
    __shared__ double red[m1::kThreads / 32];
    const int x0 = (blockIdx.x % L.tiles_x) * L.tx, y0 = (blockIdx.x / L.tiles_x) * L.ty;
    const int i = x0 + threadIdx.x % L.tx, j = y0 + threadIdx.x / L.tx;
    double nrm = 0.0;
    if (i < L.nx && j < L.ny) {
        const size_t n = (size_t)L.n, k = (size_t)j * L.nx + i;
        const double c = L.c, ic2 = 1.0 / (c * c);
        double NE = 0.0, NFx = 0.0, NFy = 0.0;
        const int naxes = L.dim == 2 ? 2 : 1;
        for (int ax = 0; ax < naxes; ++ax) {
            const double beta = ax == 0 ? L.bx : L.by;
            for (int side = -1; side <= 1; side += 2) {
                const Cell4<double> nb = fetch_planar(L, state, inflow, ax == 0 ? i + side : i,
                                                      ax == 0 ? j : j + side);
                double pxx, pxy, pyy;
                m1::closure(nb.E, nb.Fx, nb.Fy, ic2, pxx, pxy, pyy);
                const double sg = side < 0 ? 1.0 : -1.0;   // L (low side) or R (high side)
                const double Fn = ax == 0 ? nb.Fx : nb.Fy;
                const double Pnx = ax == 0 ? pxx : pxy, Pny = ax == 0 ? pxy : pyy;
                NE += beta * (c * nb.E + sg * Fn);
                NFx += c * beta * (nb.Fx + sg * c * Pnx);
                NFy += c * beta * (nb.Fy + sg * c * Pny);
            }
        }
        const double E = state[k], Fx = state[n + k], Fy = state[2 * n + k], T = state[3 * n + k];
        const double ka = L.cdt * sig[k], kt = L.cdt * (sig[k] + sig[n + k]);
        const double T2 = T * T, src = ka * (E - L.a_r * T2 * T2);
        const double rE = rhs[k] - (L.diag * E + src - NE);
        const double rFx = rhs[n + k] - ((L.diag + kt) * Fx - NFx);
        const double rFy = rhs[2 * n + k] - ((L.diag + kt) * Fy - NFy);
        const double rT = rhs[3 * n + k] - (L.c_v * T - src);
        nrm = rE * rE + (rFx * rFx + rFy * rFy) * ic2 + rT * rT;
    }
    for (int o = 16; o > 0; o >>= 1) nrm += __shfl_down_sync(0xffffffffu, nrm, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = nrm;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
        partials[blockIdx.x] = s * L.vol;
    }
}

// One CTA: fixed-order sum of the first `np` partials, sqrt, to *out.
__global__ void __launch_bounds__(m1::kThreads)
k_reduce_partials(const double* __restrict__ partials, int np, double* __restrict__ out)
{
    __shared__ double red[m1::kThreads];
    double s = 0.0;
    for (int k = threadIdx.x; k < np; k += blockDim.x) s += partials[k];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = sqrt(red[0]);
}

// Device address of the scratch array for the current device, looked up once per
// device with that device current (host code cannot take the address of a
// __device__ variable directly: its name there is a host-side stand-in).
m1_status scratch_for_current_device(double** out)
{
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        char msg[256];
        std::snprintf(msg, sizeof(msg), "cudaGetDevice: %s", cudaGetErrorString(e));
        set_error_text(msg);
        return M1_ERR_CUDA;
    }
    if (dev < 0 || dev >= kMaxDevices) {
        char msg[256];
        std::snprintf(msg, sizeof(msg),
                      "m1_residual_norm_noalloc: device %d is beyond the %d devices this "
                      "library tracks", dev, kMaxDevices);
        set_error_text(msg);
        return M1_ERR_INVALID_ARG;
    }
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_partials);
        if (e != cudaSuccess || !p) {
            char msg[256];
            std::snprintf(msg, sizeof(msg), "cudaGetSymbolAddress: %s", cudaGetErrorString(e));
            set_error_text(msg);
            return M1_ERR_CUDA;
        }
        g_scratch[dev] = static_cast<double*>(p);
    }
    *out = g_scratch[dev];
    return M1_OK;
}

}  // namespace

extern "C" m1_status m1_residual_norm_noalloc(const m1_grid_desc* desc, double dt,
                                              const double* state, const double* rhs,
                                              const double* sig, const double* inflow,
                                              double* norm_out, void* cuda_stream)
{
    if (!desc || !state || !rhs || !sig || !norm_out || !(dt > 0)) return M1_ERR_INVALID_ARG;
    if (desc->dim != 1 && desc->dim != 2) return M1_ERR_INVALID_ARG;
    if (desc->dim == 1 && desc->ny != 1) return M1_ERR_INVALID_ARG;
    if (desc->nx < 1 || desc->ny < 1 || !(desc->lx > 0) || !(desc->c > 0)) return M1_ERR_INVALID_ARG;
    if (desc->dim == 2 && !(desc->ly > 0)) return M1_ERR_INVALID_ARG;
    for (int w = 0; w < 4; ++w) {
        if (desc->bc[w] < M1_BC_PERIODIC || desc->bc[w] > M1_BC_INFLOW) return M1_ERR_INVALID_ARG;
        if (desc->bc[w] == M1_BC_INFLOW && !inflow) return M1_ERR_INVALID_ARG;
    }
    // sizes in 64-bit first: the tile count is checked against the scratch
    // before anything is narrowed to the kernels' int fields
    const long long nx = desc->nx, ny = desc->dim == 2 ? desc->ny : 1;
    const long long tx = desc->dim == 2 ? m1::kTx2 : m1::kTx1, ty = desc->dim == 2 ? m1::kTy2 : 1;
    const long long tiles_x = (nx + tx - 1) / tx, tiles = tiles_x * ((ny + ty - 1) / ty);
    if (tiles > kNoallocPartials) {
        char msg[256];
        std::snprintf(msg, sizeof(msg),
                      "m1_residual_norm_noalloc: the grid needs %lld partial sums, the fixed "
                      "scratch holds %d (2D: 2^24 cells at most)", tiles, kNoallocPartials);
        set_error_text(msg);
        return M1_ERR_INVALID_ARG;
    }
    Level<double> L{};
    L.dim = desc->dim; L.nx = (int)nx; L.ny = (int)ny;
    L.n = (int)(nx * ny);
    for (int w = 0; w < 4; ++w) L.bc[w] = desc->bc[w];
    L.tx = (int)tx; L.ty = (int)ty;
    L.tiles_x = (int)tiles_x;
    L.tiles = (int)tiles;
    L.prof_len = L.nx > L.ny ? L.nx : L.ny;
    const double hx = desc->lx / desc->nx, hy = desc->dim == 2 ? desc->ly / desc->ny : 1.0;
    L.c = desc->c; L.a_r = desc->a_r; L.c_v = desc->c_v;
    L.ax = desc->c * dt / hx; L.ay = desc->dim == 2 ? desc->c * dt / hy : 0.0;
    L.bx = dt / (2.0 * hx); L.by = desc->dim == 2 ? dt / (2.0 * hy) : 0.0;
    L.diag = 1.0 + L.ax + L.ay;
    L.cdt = desc->c * dt;
    L.vol = desc->dim == 2 ? hx * hy : hx;

    double* scratch = nullptr;
    m1_status st = scratch_for_current_device(&scratch);
    if (st != M1_OK) return st;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    // each launch reports its own error (cudaLaunchKernel returns it), so an
    // earlier unrelated error pending on this thread is neither taken for this
    // call's nor cleared
    const double* p_state = state;
    const double* p_rhs = rhs;
    const double* p_sig = sig;
    const double* p_inflow = inflow;
    double* p_scratch = scratch;
    void* args1[] = { &L, &p_state, &p_rhs, &p_sig, &p_inflow, &p_scratch };
    cudaError_t e = cudaLaunchKernel((const void*)k_residual_partials_planar, dim3(L.tiles),
                                     dim3(m1::kThreads), args1, 0, s);
    const char* what = "k_residual_partials_planar";
    if (e == cudaSuccess) {
        const double* p_part = scratch;
        int np = L.tiles;
        double* p_out = norm_out;
        void* args2[] = { &p_part, &np, &p_out };
        e = cudaLaunchKernel((const void*)k_reduce_partials, dim3(1), dim3(m1::kThreads), args2, 0,
                             s);
        what = "k_reduce_partials";
    }
    if (e != cudaSuccess) {
        char msg[256];
        std::snprintf(msg, sizeof(msg), "m1_residual_norm_noalloc launch of %s: %s", what,
                      cudaGetErrorString(e));
        set_error_text(msg);
        return M1_ERR_CUDA;
    }
    return M1_OK;
}
