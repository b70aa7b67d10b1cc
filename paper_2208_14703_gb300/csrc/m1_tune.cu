// Autotuner of the sweep kernels' strip shape.
//
// The Jacobi / pseudo-time sweep gives each warp a strip of 30 columns and
// `sh` rows (2D).  Tall strips evaluate fewer halo closures per updated cell
// ((sh + 2) / sh) but leave fewer strips, hence fewer warps, per level; the
// best height depends on the level size, the precision and the GPU.  The tuner
// times one sweep of a synthetic admissible 2D level for every candidate height
// and size class (n = 16 .. 2048; the FP32 form up to 4096) and keeps the
// fastest; for the FP32 correction form it also
// chooses how strip rows are staged (loads into registers one row ahead, or
// asynchronous copies into a shared-memory ring three rows ahead).  Levels
// created afterwards take both from the table (before any tuning: ny / 64
// rows, between 1 and 16, staged through registers).
// The height changes no arithmetic: every cell's update is the same whatever
// strip it falls in, so grids of any height give identical results.  The two
// stagings are separate kernels; their FP32 roundings may differ in the last
// bit (the mixed path's FP64 defect correction makes results agree to rounding).
#include <m1.h>

#include <cmath>
#include <mutex>
#include <vector>

#include "m1_engine.h"
#include "m1_kernels.cuh"

namespace m1 {

namespace {

constexpr int kClasses = 16;                 // size classes 2^0 .. 2^15 (sqrt of the cell count)
constexpr int kCandidates[] = { 1, 2, 4, 8, 12, 16, 24, 32, 48, 64, 96, 128 };

std::mutex g_tune_mu;
int g_rows[2][kClasses] = {};                // [kind][class], 0 = untuned
int g_ring[kClasses] = {};                   // FP32 correction form: 1 = cp.async staging

int size_class(int nx, int ny)
{
    const double s = std::sqrt((double)nx * (double)ny);
    int c = (int)std::lround(std::log2(s > 1.0 ? s : 1.0));
    return c < 0 ? 0 : (c >= kClasses ? kClasses - 1 : c);
}

// Deterministic admissible test data: E in [0.5, 1.5], |F| <= 0.6 c E, T near 1,
// opacities spanning 1e-2 .. 1e2.
template <typename R>
void synth(int n, std::vector<Cell4<R>>& u, std::vector<Cell4<R>>& f, std::vector<Sig2<R>>& sig)
{
    u.resize((size_t)n * n);
    f.resize((size_t)n * n);
    sig.resize((size_t)n * n);
    for (int j = 0; j < n; ++j)
        for (int i = 0; i < n; ++i) {
            const double x = (i + 0.5) / n, y = (j + 0.5) / n;
            const double E = 1.0 + 0.5 * std::sin(6.28318 * (x + 2 * y));
            const double fx = 0.4 * std::cos(6.28318 * 3 * x), fy = 0.4 * std::sin(6.28318 * 2 * y);
            const double T = 1.0 + 0.2 * std::cos(6.28318 * (2 * x - y));
            const size_t k = (size_t)j * n + i;
            u[k] = Cell4<R>{ (R)E, (R)(fx * E), (R)(fy * E), (R)T };
            f[k] = u[k];
            sig[k] = Sig2<R>{ (R)std::pow(10.0, 2.0 * std::sin(6.28318 * 5 * x * y)),
                              (R)std::pow(10.0, 2.0 * std::cos(6.28318 * 3 * (x - y))) };
        }
}

// Milliseconds per sweep of an n x n level for every candidate strip height
// and staging (`out[s * ncand + c]`, s = 0 registers, 1 cp.async ring (FP32
// correction form only); NAN where not applicable).
template <typename R>
m1_status time_level(int n, bool delta, cudaStream_t stream, std::vector<double>& out)
{
    Engine<R> e;
    M1_TRY(e.init(1, 1, delta, stream, 0));
    m1_grid_desc g{};
    g.dim = 2; g.nx = n; g.ny = n; g.lx = 1.0; g.ly = 1.0;
    for (int w = 0; w < 4; ++w) g.bc[w] = M1_BC_REFLECT;
    g.lmax = 1; g.c = 1.0; g.a_r = 1.0; g.c_v = 1.0;
    int slot = 0;
    M1_TRY(e.add_slot(g, &slot));
    std::vector<Cell4<R>> u, f;
    std::vector<Sig2<R>> sig;
    synth<R>(n, u, f, sig);
    Level<R>& q = e.h[0];
    const size_t bytes = sizeof(Cell4<R>) * u.size();
    if (delta) {
        // correction form: base w = the state, correction e = a small fraction
        M1_CK(cudaMemcpyAsync(q.w, u.data(), bytes, cudaMemcpyHostToDevice, e.stream));
        for (auto& c : u) { c.E *= R(1e-3); c.Fx *= R(1e-3); c.Fy *= R(1e-3); c.T *= R(1e-3); }
        for (auto& c : f) { c.E *= R(1e-3); c.Fx *= R(1e-3); c.Fy *= R(1e-3); c.T *= R(1e-3); }
    }
    M1_CK(cudaMemcpyAsync(q.u[0], u.data(), bytes, cudaMemcpyHostToDevice, e.stream));
    M1_CK(cudaMemcpyAsync(q.f, f.data(), bytes, cudaMemcpyHostToDevice, e.stream));
    M1_CK(cudaMemcpyAsync(q.sig, sig.data(), sizeof(Sig2<R>) * sig.size(), cudaMemcpyHostToDevice,
                          e.stream));
    M1_TRY(e.set_dt(0, 100.0 / n));
    M1_TRY(e.set_ctl_simple(0, 0.0, 0.5, 0.5));
    const int ncand = (int)(sizeof(kCandidates) / sizeof(int));
    out.assign(2 * ncand, NAN);
    const int reps = n >= 1024 ? 4 : 10;
    for (int idx = 0; idx < 2 * ncand; ++idx) {
        const int c = idx % ncand, ring = idx / ncand;
        const int sh = kCandidates[c];
        if (sh > n || (ring && !delta)) continue;
        e.h[0].sh = sh;
        e.h[0].strips = e.h[0].sx * ((n + sh - 1) / sh);
        e.h[0].ring = ring;
        M1_TRY(e.rebuild());
        int cur = 0;
        e.sweeps_fine(cur, 2, e.stream);              // warm-up
        M1_CK(cudaEventRecord(e.ev0, e.stream));
        e.sweeps_fine(cur, reps, e.stream);
        M1_CK(cudaEventRecord(e.ev1, e.stream));
        M1_CK(cudaGetLastError());
        M1_CK(cudaEventSynchronize(e.ev1));
        float ms = 0.f;
        M1_CK(cudaEventElapsedTime(&ms, e.ev0, e.ev1));
        out[idx] = ms / reps;
    }
    return M1_OK;
}

}  // namespace

int strip_rows(int kind, int nx, int ny)
{
    int r = 0;
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        r = g_rows[kind ? 1 : 0][size_class(nx, ny)];
    }
    if (r <= 0) r = std::max(1, std::min(kStripH, ny / 64));
    return std::max(1, std::min(r, ny));
}

int strip_ring(int nx, int ny)
{
    std::lock_guard<std::mutex> lk(g_tune_mu);
    return g_ring[size_class(nx, ny)];
}

}  // namespace m1

using m1::kClasses;

extern "C" {

m1_status m1_autotune(void* cuda_stream, m1_tune_entry* out, int max_entries, int* n_entries)
{
    if (max_entries < 0 || (max_entries > 0 && !out)) return M1_ERR_INVALID_ARG;
    const cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    std::vector<m1_tune_entry> found;
    // FP64 up to 2048^2 (the FP64 workloads); the FP32 correction form also at
    // 4096^2, the mixed-precision configuration
    for (int kind = 0; kind < 2; ++kind)
        for (int lg = 4; lg <= (kind == 0 ? 11 : 12); ++lg) {
            const int n = 1 << lg;
            std::vector<double> ms;
            m1_status st = kind == 0 ? m1::time_level<double>(n, false, s, ms)
                                     : m1::time_level<float>(n, true, s, ms);
            if (st != M1_OK) return st;
            const int ncand = (int)(sizeof(m1::kCandidates) / sizeof(int));
            int best = -1;
            for (int c = 0; c < (int)ms.size(); ++c)
                if (!std::isnan(ms[c]) && (best < 0 || ms[c] < ms[best])) best = c;
            if (best < 0) continue;
            m1_tune_entry t{};
            t.kind = kind;
            t.n = n;
            t.strip_rows = m1::kCandidates[best % ncand];
            t.staging = best / ncand;
            t.ms = ms[best];
            t.ms_default = NAN;
            const int def = std::max(1, std::min(m1::kStripH, n / 64));
            for (int c = 0; c < ncand; ++c)
                if (m1::kCandidates[c] == def) t.ms_default = ms[c];
            found.push_back(t);
        }
    {
        std::lock_guard<std::mutex> lk(m1::g_tune_mu);
        for (const auto& t : found) {
            m1::g_rows[t.kind][m1::size_class(t.n, t.n)] = t.strip_rows;
            if (t.kind == 1) m1::g_ring[m1::size_class(t.n, t.n)] = t.staging;
        }
    }
    if (n_entries) *n_entries = (int)found.size();
    for (int k = 0; k < (int)found.size() && k < max_entries; ++k) out[k] = found[k];
    return M1_OK;
}

m1_status m1_set_tuning(const m1_tune_entry* in, int n)
{
    if (n < 0 || (n > 0 && !in)) return M1_ERR_INVALID_ARG;
    for (int k = 0; k < n; ++k)
        if ((in[k].kind != 0 && in[k].kind != 1) || in[k].n < 1 || in[k].strip_rows < 0 ||
            in[k].strip_rows > 256 || in[k].staging < 0 || in[k].staging > 1 ||
            (in[k].kind == 0 && in[k].staging != 0))
            return M1_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(m1::g_tune_mu);
    for (int k = 0; k < n; ++k) {
        m1::g_rows[in[k].kind][m1::size_class(in[k].n, in[k].n)] = in[k].strip_rows;
        if (in[k].kind == 1) m1::g_ring[m1::size_class(in[k].n, in[k].n)] = in[k].staging;
    }
    return M1_OK;
}

m1_status m1_strip_rows(int kind, int nx, int ny, int* rows)
{
    if (!rows || (kind != 0 && kind != 1) || nx < 1 || ny < 1) return M1_ERR_INVALID_ARG;
    *rows = m1::strip_rows(kind, nx, ny);
    return M1_OK;
}

}  // extern "C"
