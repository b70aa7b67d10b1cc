// Host side of libm1: the level hierarchy, the V-cycle of Algorithm 4 (Appendix
// A) recorded once into a CUDA graph and relaunched until the device-side stop
// flag is set, and the C ABI declared in include/m1.h.
#include <m1.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <memory>
#include <string>
#include <vector>

#include "m1_kernels.cuh"

namespace {

thread_local char g_err[512] = "";

void set_err(cudaError_t e, const char* what)
{
    std::snprintf(g_err, sizeof(g_err), "%s: %s", what, cudaGetErrorString(e));
}

#define M1_CK(call)                                                                                \
    do {                                                                                           \
        cudaError_t e_ = (call);                                                                   \
        if (e_ != cudaSuccess) {                                                                   \
            set_err(e_, #call);                                                                    \
            return e_ == cudaErrorMemoryAllocation ? M1_ERR_OOM : M1_ERR_CUDA;                     \
        }                                                                                          \
    } while (0)

#define M1_TRY(expr)                                                                               \
    do {                                                                                           \
        m1_status s_ = (expr);                                                                     \
        if (s_ != M1_OK) return s_;                                                                \
    } while (0)

using m1::Cell4;
using m1::Ctl;
using m1::Level;
using m1::Sig2;

// Full-weighting restriction of an inflow profile along its wall (1/4, 1/2,
// 1/4; ends copied), giving the coarse level's prescribed ghost states.
void restrict_profile(const double* fine, int nf, double* coarse, int nc)
{
    for (int i = 0; i < nc; ++i) {
        if (nc == nf) { coarse[i] = fine[i]; continue; }
        int a = std::max(2 * i - 1, 0), b = 2 * i, c = std::min(2 * i + 1, nf - 1);
        coarse[i] = 0.25 * fine[a] + 0.5 * fine[b] + 0.25 * fine[c];
    }
}

// Relaunch a captured cycle graph until the device control block reports done.
// Batch k is queued before the host waits on the flag copied after batch k-1,
// so the GPU never idles on the poll; cycles queued past convergence return at
// once (every kernel checks the flag).  At most max_cycles + 2 graphs' worth.
m1_status run_until_done(cudaGraphExec_t graph, int graph_cycles, int max_cycles,
                         cudaStream_t stream, Ctl* ctl, int* done_h, cudaEvent_t* poll,
                         long long* launched_out)
{
    long long launched = 0;
    const long long cap_cycles = (long long)max_cycles + 2 * graph_cycles;
    int batch = 1;
    for (long long k = 0;; ++k) {
        const int slot = (int)(k & 1);
        for (int b = 0; b < batch && launched < cap_cycles; ++b) {
            M1_CK(cudaGraphLaunch(graph, stream));
            launched += graph_cycles;
        }
        M1_CK(cudaMemcpyAsync(done_h + slot, &ctl->done, sizeof(int), cudaMemcpyDeviceToHost, stream));
        M1_CK(cudaEventRecord(poll[slot], stream));
        if (k > 0) {
            M1_CK(cudaEventSynchronize(poll[slot ^ 1]));
            if (done_h[slot ^ 1]) break;
        }
        if (launched >= cap_cycles) break;
        batch = std::min(batch * 2, 8);
    }
    *launched_out = launched;
    return M1_OK;
}

struct Params {
    int nu0, nu_l, m, mc;
    bool operator==(const Params& o) const
    {
        return nu0 == o.nu0 && nu_l == o.nu_l && m == o.m && mc == o.mc;
    }
};

struct ImplBase {
    virtual ~ImplBase() = default;
    virtual m1_status set_state(const double* E, const double* Fx, const double* Fy,
                                const double* T, const double* sa, const double* ss, int dev) = 0;
    virtual m1_status set_inflow(int side, const double* E, const double* Fx, const double* Fy) = 0;
    virtual m1_status get_state(double* E, double* Fx, double* Fy, double* T, int dev) = 0;
    virtual m1_status step(double dt, const m1_solve_params& p, m1_step_stats* st) = 0;
    virtual m1_status residual_norm(double dt, double* out) = 0;
    virtual m1_status history(double* hist, double* dtau, int len) = 0;
    virtual m1_status jacobi(double dt, int sweeps) = 0;
};

template <typename R>
struct Impl : ImplBase {
    m1_grid_desc desc{};
    int L = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    cudaStream_t cap = nullptr;
    std::vector<Level<R>> h;       // host copies of the level descriptors
    Level<R>* d = nullptr;         // device array of descriptors
    std::vector<void*> allocs;
    std::vector<std::vector<double>> prof;   // inflow profiles per level [4*3*prof_len]
    Ctl* ctl = nullptr;            // device control block
    Ctl* ctl_h = nullptr;          // pinned host mirror
    int* done_h = nullptr;         // pinned flags for polling
    double* hist = nullptr;
    double* dtau_hist = nullptr;
    int hist_len = 0;
    double* part = nullptr;        // per-tile norm partials (fine level)
    double* partb = nullptr;
    double* stage = nullptr;       // planar FP64 staging, 6 * n0
    Sig2<R>* sig_stage = nullptr;
    unsigned int* bad = nullptr;
    unsigned int* bad_h = nullptr;
    double dt_levels = NAN;        // dt the level constants were computed for
    double dt_rhs = NAN;           // dt of the last step (level-0 f holds its b)
    bool rhs_valid = false;
    cudaGraphExec_t graph = nullptr;
    Params gparams{};
    int graph_cycles = 1;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    cudaEvent_t poll[2] = { nullptr, nullptr };
    int last_cycles = 0;
    bool delta = false;            // correction-form FP32 hierarchy of the mixed path

    ~Impl() override
    {
        if (graph) cudaGraphExecDestroy(graph);
        if (stream) cudaStreamSynchronize(stream);
        for (void* p : allocs) cudaFree(p);
        if (ctl_h) cudaFreeHost(ctl_h);
        if (done_h) cudaFreeHost(done_h);
        if (bad_h) cudaFreeHost(bad_h);
        if (ev0) cudaEventDestroy(ev0);
        if (ev1) cudaEventDestroy(ev1);
        for (auto& e : poll) if (e) cudaEventDestroy(e);
        if (cap) cudaStreamDestroy(cap);
        if (own_stream && stream) cudaStreamDestroy(stream);
    }

    template <typename T>
    m1_status dalloc(T** p, size_t count)
    {
        void* q = nullptr;
        M1_CK(cudaMalloc(&q, std::max<size_t>(count, 1) * sizeof(T)));
        allocs.push_back(q);
        *p = static_cast<T*>(q);
        return M1_OK;
    }

    m1_status init(const m1_grid_desc& dsc, cudaStream_t s, bool correction_form = false)
    {
        desc = dsc;
        L = dsc.lmax;
        delta = correction_form;
        if (s) stream = s;
        else { M1_CK(cudaStreamCreateWithFlags(&stream, cudaStreamNonBlocking)); own_stream = true; }
        M1_CK(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
        M1_CK(cudaEventCreate(&ev0));
        M1_CK(cudaEventCreate(&ev1));
        M1_CK(cudaEventCreateWithFlags(&poll[0], cudaEventDisableTiming));
        M1_CK(cudaEventCreateWithFlags(&poll[1], cudaEventDisableTiming));
        h.resize(L);
        prof.resize(L);
        int nx = dsc.nx, ny = dsc.dim == 2 ? dsc.ny : 1;
        double hx = dsc.lx / dsc.nx, hy = dsc.dim == 2 ? dsc.ly / dsc.ny : 1.0;
        for (int l = 0; l < L; ++l) {
            Level<R>& q = h[l];
            std::memset(&q, 0, sizeof(q));
            q.dim = dsc.dim; q.nx = nx; q.ny = ny; q.n = nx * ny;
            for (int w = 0; w < 4; ++w) q.bc[w] = dsc.bc[w];
            q.tx = dsc.dim == 2 ? m1::kTx2 : m1::kTx1;
            q.ty = dsc.dim == 2 ? m1::kTy2 : 1;
            q.tiles_x = (nx + q.tx - 1) / q.tx;
            q.tiles = q.tiles_x * ((ny + q.ty - 1) / q.ty);
            q.prof_len = std::max(nx, ny);
            q.c = (R)dsc.c; q.a_r = (R)dsc.a_r; q.c_v = (R)dsc.c_v;
            q.vol = dsc.dim == 2 ? hx * hy : hx;
            M1_TRY(dalloc(&q.v, q.n));
            M1_TRY(dalloc(&q.u[0], q.n));
            M1_TRY(dalloc(&q.u[1], q.n));
            M1_TRY(dalloc(&q.f, q.n));
            M1_TRY(dalloc(&q.r, q.n));
            if (delta) M1_TRY(dalloc(&q.w, q.n));
            M1_TRY(dalloc(&q.sig, q.n));
            M1_TRY(dalloc(&q.inflow, (size_t)12 * q.prof_len));
            M1_CK(cudaMemsetAsync(q.inflow, 0, sizeof(R) * 12 * q.prof_len, stream));
            prof[l].assign((size_t)12 * q.prof_len, 0.0);
            nx /= 2; if (dsc.dim == 2) ny /= 2;
            hx *= 2; if (dsc.dim == 2) hy *= 2;
        }
        M1_TRY(dalloc(&d, L));
        M1_TRY(dalloc(&ctl, 1));
        M1_CK(cudaMallocHost(&ctl_h, sizeof(Ctl)));
        M1_CK(cudaMallocHost(&done_h, 2 * sizeof(int)));
        M1_CK(cudaMallocHost(&bad_h, sizeof(unsigned int)));
        std::memset(ctl_h, 0, sizeof(Ctl));
        hist_len = 20001;
        M1_TRY(dalloc(&hist, hist_len));
        M1_TRY(dalloc(&dtau_hist, hist_len));
        M1_TRY(dalloc(&part, h[0].tiles));
        M1_TRY(dalloc(&partb, h[0].tiles));
        M1_TRY(dalloc(&stage, (size_t)6 * h[0].n));
        M1_TRY(dalloc(&sig_stage, h[0].n));
        M1_TRY(dalloc(&bad, 1));
        M1_TRY(upload_levels());
        M1_CK(cudaMemsetAsync(ctl, 0, sizeof(Ctl), stream));
        M1_CK(cudaStreamSynchronize(stream));
        return M1_OK;
    }

    m1_status upload_levels()
    {
        M1_CK(cudaMemcpyAsync(d, h.data(), sizeof(Level<R>) * L, cudaMemcpyHostToDevice, stream));
        M1_CK(cudaStreamSynchronize(stream));   // h may change right after
        return M1_OK;
    }

    m1_status set_dt(double dt)
    {
        if (dt == dt_levels) return M1_OK;
        for (int l = 0; l < L; ++l) {
            Level<R>& q = h[l];
            double hx = desc.lx / desc.nx * (double)(1 << l);
            double hy = desc.dim == 2 ? desc.ly / desc.ny * (double)(1 << l) : 1.0;
            double ax = desc.c * dt / hx, ay = desc.dim == 2 ? desc.c * dt / hy : 0.0;
            q.ax = (R)ax; q.ay = (R)ay;
            q.bx = (R)(dt / (2.0 * hx)); q.by = desc.dim == 2 ? (R)(dt / (2.0 * hy)) : R(0);
            q.diag = (R)(1.0 + ax + ay);
            q.cdt = (R)(desc.c * dt);
        }
        M1_TRY(upload_levels());
        dt_levels = dt;
        return M1_OK;
    }

    // ---- state in / out ------------------------------------------------------
    m1_status pack_into(Cell4<R>* dst, const double* E, const double* Fx, const double* Fy,
                        const double* T, double tscale, int dev)
    {
        const int n = h[0].n;
        if (!dev) {
            M1_CK(cudaMemcpyAsync(stage, E, n * 8, cudaMemcpyHostToDevice, stream));
            M1_CK(cudaMemcpyAsync(stage + n, Fx, n * 8, cudaMemcpyHostToDevice, stream));
            if (Fy) M1_CK(cudaMemcpyAsync(stage + 2 * (size_t)n, Fy, n * 8, cudaMemcpyHostToDevice, stream));
            M1_CK(cudaMemcpyAsync(stage + 3 * (size_t)n, T, n * 8, cudaMemcpyHostToDevice, stream));
            E = stage; Fx = stage + n; Fy = Fy ? stage + 2 * (size_t)n : nullptr; T = stage + 3 * (size_t)n;
        }
        m1::launch_pack_state<R>(E, Fx, Fy, T, tscale, dst, n, stream);
        M1_CK(cudaGetLastError());
        return M1_OK;
    }

    m1_status unpack_from(const Cell4<R>* src, int n, double* E, double* Fx, double* Fy, double* T,
                          int dev)
    {
        if (dev) {
            m1::launch_unpack_state<R>(src, E, Fx, Fy, T, n, stream);
            M1_CK(cudaGetLastError());
            M1_CK(cudaStreamSynchronize(stream));
            return M1_OK;
        }
        double* s = stage;
        m1::launch_unpack_state<R>(src, s, s + n, Fy ? s + 2 * (size_t)n : nullptr, s + 3 * (size_t)n,
                                   n, stream);
        M1_CK(cudaGetLastError());
        M1_CK(cudaMemcpyAsync(E, s, n * 8, cudaMemcpyDeviceToHost, stream));
        M1_CK(cudaMemcpyAsync(Fx, s + n, n * 8, cudaMemcpyDeviceToHost, stream));
        if (Fy) M1_CK(cudaMemcpyAsync(Fy, s + 2 * (size_t)n, n * 8, cudaMemcpyDeviceToHost, stream));
        M1_CK(cudaMemcpyAsync(T, s + 3 * (size_t)n, n * 8, cudaMemcpyDeviceToHost, stream));
        M1_CK(cudaStreamSynchronize(stream));
        return M1_OK;
    }

    m1_status set_state(const double* E, const double* Fx, const double* Fy, const double* T,
                        const double* sa, const double* ss, int dev) override
    {
        const int n = h[0].n;
        if (!E || !Fx || !T || (desc.dim == 2 && !Fy) || (!sa != !ss)) return M1_ERR_INVALID_ARG;
        // stage into u[1] / sig_stage, check, then commit
        M1_TRY(pack_into(h[0].u[1], E, Fx, Fy, T, 1.0, dev));
        const Sig2<R>* sig_chk = nullptr;
        if (sa) {
            const double *a = sa, *b = ss;
            if (!dev) {
                M1_CK(cudaMemcpyAsync(stage + 4 * (size_t)n, sa, n * 8, cudaMemcpyHostToDevice, stream));
                M1_CK(cudaMemcpyAsync(stage + 5 * (size_t)n, ss, n * 8, cudaMemcpyHostToDevice, stream));
                a = stage + 4 * (size_t)n; b = stage + 5 * (size_t)n;
            }
            m1::launch_pack_sig<R>(a, b, sig_stage, n, stream);
            sig_chk = sig_stage;
        }
        M1_CK(cudaMemsetAsync(bad, 0, sizeof(unsigned int), stream));
        m1::launch_check_state<R>(h[0].u[1], sig_chk, n, desc.c, bad, stream);
        M1_CK(cudaGetLastError());
        M1_CK(cudaMemcpyAsync(bad_h, bad, sizeof(unsigned int), cudaMemcpyDeviceToHost, stream));
        M1_CK(cudaStreamSynchronize(stream));
        if (*bad_h) return M1_ERR_NONADMISSIBLE_INPUT;
        M1_CK(cudaMemcpyAsync(h[0].u[0], h[0].u[1], sizeof(Cell4<R>) * n, cudaMemcpyDeviceToDevice, stream));
        if (sa) {
            M1_CK(cudaMemcpyAsync(h[0].sig, sig_stage, sizeof(Sig2<R>) * n, cudaMemcpyDeviceToDevice, stream));
            for (int l = 1; l < L; ++l) m1::launch_restrict_sig<R>(d + l - 1, d + l, h[l], stream);
            M1_CK(cudaGetLastError());
        }
        rhs_valid = false;
        M1_CK(cudaStreamSynchronize(stream));
        return M1_OK;
    }

    m1_status set_inflow(int side, const double* E, const double* Fx, const double* Fy) override
    {
        if (side < 0 || side > 3 || !E || !Fx || !Fy) return M1_ERR_INVALID_ARG;
        for (int l = 0; l < L; ++l) {
            const int len = side < 2 ? h[l].ny : h[l].nx;
            const int pl = h[l].prof_len;
            for (int fld = 0; fld < 3; ++fld) {
                double* dst = prof[l].data() + (size_t)(side * 3 + fld) * pl;
                if (l == 0) {
                    const double* src = fld == 0 ? E : (fld == 1 ? Fx : Fy);
                    std::copy(src, src + len, dst);
                } else {
                    const int plf = h[l - 1].prof_len;
                    const int nf = side < 2 ? h[l - 1].ny : h[l - 1].nx;
                    restrict_profile(prof[l - 1].data() + (size_t)(side * 3 + fld) * plf, nf, dst, len);
                }
            }
            std::vector<R> tmp(prof[l].begin(), prof[l].end());
            M1_CK(cudaMemcpyAsync(h[l].inflow, tmp.data(), sizeof(R) * tmp.size(), cudaMemcpyHostToDevice, stream));
            M1_CK(cudaStreamSynchronize(stream));
        }
        return M1_OK;
    }

    m1_status get_state(double* E, double* Fx, double* Fy, double* T, int dev) override
    {
        if (!E || !Fx || !T) return M1_ERR_INVALID_ARG;
        return unpack_from(h[0].u[0], h[0].n, E, Fx, Fy, T, dev);
    }

    // ---- the V-cycle ------------------------------------------------------------
    void sweeps_fine(int& cur, int count, cudaStream_t s)
    {
        for (int k = 0; k < count; ++k) {
            m1::launch_sweep<R>(d, h[0], false, cur, 1 - cur, ctl, s, delta);
            cur = 1 - cur;
        }
    }

    // m pseudo-time steps (nu_l = 1 Jacobi sweep each) at level l; from_v: the
    // first step starts from v_l (initial guess u_l = v_l, Algorithm 4).
    void pseudo(int l, int& cur, int m, bool from_v, cudaStream_t s)
    {
        for (int k = 0; k < m; ++k) {
            if (k == 0 && from_v) { m1::launch_sweep<R>(d + l, h[l], true, -1, 0, ctl, s, delta); cur = 0; }
            else { m1::launch_sweep<R>(d + l, h[l], true, cur, 1 - cur, ctl, s, delta); cur = 1 - cur; }
        }
    }

    // One V-cycle of Algorithm 4 on this hierarchy.  tail: end with the fine
    // residual norm and the stop test (the mixed-precision driver does its own).
    void record_cycle(const Params& p, int& cur0, cudaStream_t s, bool tail = true)
    {
        std::vector<int> cur(L, 0);
        cur[0] = cur0;
        for (int l = 0; l < L - 1; ++l) {
            if (l == 0) {
                sweeps_fine(cur[0], p.nu0, s);
                m1::launch_apply<R>(d, h[0], m1::APPLY_RESID, cur[0], nullptr, 1, ctl, s, delta);
            } else {
                m1::launch_apply<R>(d + l, h[l], m1::APPLY_FAS, -1, nullptr, 0, ctl, s, delta);
                pseudo(l, cur[l], p.m, true, s);
                m1::launch_apply<R>(d + l, h[l], m1::APPLY_RESID, cur[l], nullptr, 1, ctl, s, delta);
            }
            m1::launch_restrict<R>(d + l, d + l + 1, h[l + 1], cur[l], ctl, s, delta);
        }
        if (L == 1) {
            sweeps_fine(cur[0], p.nu0, s);
        } else {
            const int l = L - 1;
            m1::launch_apply<R>(d + l, h[l], m1::APPLY_FAS, -1, nullptr, 0, ctl, s, delta);
            pseudo(l, cur[l], p.mc, true, s);
        }
        for (int l = L - 2; l >= 0; --l) {
            m1::launch_prolong<R>(d + l + 1, d + l, h[l], cur[l + 1], cur[l], ctl, s, delta);
            if (l == 0) sweeps_fine(cur[0], p.nu0, s);
            else pseudo(l, cur[l], p.m, false, s);
        }
        if (tail) {
            m1::launch_apply<R>(d, h[0], m1::APPLY_RESID, cur[0], part, 0, ctl, s);
            m1::launch_finalize(ctl, part, h[0].tiles, nullptr, 0, m1::FIN_CYCLE, cur[0], s);
        }
        cur0 = cur[0];
    }

    long long kernels_per_cycle(const Params& p) const
    {
        if (L == 1) return p.nu0 + 2;
        long long k = p.nu0 + 2;                           // fine pre-smooth, residual, restrict
        k += (long long)(L - 2) * (p.m + 3);               // FAS rhs, pseudo, residual, restrict
        k += 1 + p.mc;                                     // coarsest
        k += (long long)(L - 2) * (1 + p.m) + 1 + p.nu0;   // prolong + post-smooth
        return k + 2;                                      // final residual, finalize
    }

    m1_status build_graph(const Params& p)
    {
        if (graph && gparams == p) return M1_OK;
        if (graph) { cudaGraphExecDestroy(graph); graph = nullptr; }
        // a captured graph must return the fine iterate to buffer 0
        const int per_cycle = L == 1 ? p.nu0 : 2 * p.nu0;
        graph_cycles = (per_cycle % 2) ? 2 : 1;
        cudaGraph_t g = nullptr;
        M1_CK(cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal));
        int cur0 = 0;
        for (int c = 0; c < graph_cycles; ++c) record_cycle(p, cur0, cap);
        cudaError_t e = cudaStreamEndCapture(cap, &g);
        if (e != cudaSuccess) { set_err(e, "cudaStreamEndCapture"); return M1_ERR_CUDA; }
        if (cur0 != 0) { cudaGraphDestroy(g); return M1_ERR_INVALID_ARG; }
        e = cudaGraphInstantiate(&graph, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) { set_err(e, "cudaGraphInstantiate"); graph = nullptr; return M1_ERR_CUDA; }
        gparams = p;
        return M1_OK;
    }

    m1_status step(double dt, const m1_solve_params& sp, m1_step_stats* st) override
    {
        if (!(dt > 0) || sp.nu0 < 1 || sp.nu_l != 1 || sp.m_pseudo < 1 || sp.m_coarse < 1 ||
            sp.max_cycles < 1 || !(sp.tol >= 0))
            return M1_ERR_INVALID_ARG;
        M1_TRY(set_dt(dt));
        Params p{ sp.nu0, sp.nu_l, sp.m_pseudo, sp.m_coarse };
        M1_TRY(build_graph(p));
        // control block: parameters, reset counters
        Ctl c{};
        c.tol = sp.tol; c.grow = sp.grow; c.shrink = sp.shrink; c.eps_i = sp.eps_i;
        c.eps_d = sp.eps_d; c.dtau0 = sp.dtau0; c.dtau_min = sp.dtau_min; c.dtau_max = sp.dtau_max;
        c.theta_ex = sp.theta_ex; c.theta_c = sp.theta_c; c.max_cycles = sp.max_cycles;
        c.hist_len = hist_len; c.hist = hist; c.dtau_hist = dtau_hist;
        c.res0_floor = 1e-14 * (double)h[0].diag;   // rounding floor of evaluating A
        *ctl_h = c;
        M1_CK(cudaEventRecord(ev0, stream));
        M1_CK(cudaMemcpyAsync(ctl, ctl_h, sizeof(Ctl), cudaMemcpyHostToDevice, stream));
        // b = (E^n, F^n, C_v T^n); r_0 = b - A(v^n); ||b||
        m1::launch_make_rhs<R>(d, h[0], 0, stream);
        m1::launch_apply<R>(d, h[0], m1::APPLY_RESID, 0, part, 0, ctl, stream);
        m1::launch_norm_state<R>(d, h[0], h[0].f, partb, stream);
        m1::launch_finalize(ctl, part, h[0].tiles, partb, h[0].tiles, m1::FIN_INIT, 0, stream);
        M1_CK(cudaGetLastError());
        dt_rhs = dt; rhs_valid = true;
        long long launched = 0;
        M1_TRY(run_until_done(graph, graph_cycles, sp.max_cycles, stream, ctl, done_h, poll, &launched));
        M1_CK(cudaMemcpyAsync(ctl_h, ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, stream));
        M1_CK(cudaStreamSynchronize(stream));
        if (ctl_h->result_buf == 1) {
            M1_CK(cudaMemcpyAsync(h[0].u[0], h[0].u[1], sizeof(Cell4<R>) * h[0].n,
                                  cudaMemcpyDeviceToDevice, stream));
        }
        M1_CK(cudaEventRecord(ev1, stream));
        M1_CK(cudaEventSynchronize(ev1));
        last_cycles = ctl_h->kappa;
        if (st) {
            float ms = 0.f;
            cudaEventElapsedTime(&ms, ev0, ev1);
            st->cycles = ctl_h->kappa;
            st->res0 = ctl_h->res0;
            st->res = ctl_h->kappa > 0 ? ctl_h->res : ctl_h->res0;
            st->dtau_final = ctl_h->dtau;
            st->sweeps = (long long)ctl_h->kappa * (L == 1 ? p.nu0 : 2 * p.nu0);
            st->ms = ms;
            st->status = ctl_h->status;
            st->newton_fail = ctl_h->newton_fail;
            st->damped = ctl_h->damped;
            st->launches = 4 + launched * (long long)kernels_per_cycle(p);
        }
        return ctl_h->status == m1::CTL_OK ? M1_OK : M1_ERR_NOT_CONVERGED;
    }

    m1_status residual_norm(double dt, double* out) override
    {
        if (!out || !(dt > 0)) return M1_ERR_INVALID_ARG;
        M1_TRY(set_dt(dt));
        if (!(rhs_valid && dt == dt_rhs)) m1::launch_make_rhs<R>(d, h[0], 0, stream);
        m1::launch_apply<R>(d, h[0], m1::APPLY_RESID, 0, part, 0, nullptr, stream);
        M1_CK(cudaGetLastError());
        std::vector<double> p(h[0].tiles);
        M1_CK(cudaMemcpyAsync(p.data(), part, sizeof(double) * p.size(), cudaMemcpyDeviceToHost, stream));
        M1_CK(cudaStreamSynchronize(stream));
        double s = 0.0;
        for (double x : p) s += x;
        *out = std::sqrt(s);
        return M1_OK;
    }

    m1_status jacobi(double dt, int sweeps) override
    {
        if (!(dt > 0) || sweeps < 0) return M1_ERR_INVALID_ARG;
        M1_TRY(set_dt(dt));
        M1_TRY(set_ctl_simple(0.0, 0.5, 0.5));
        m1::launch_make_rhs<R>(d, h[0], 0, stream);
        int cur = 0;
        sweeps_fine(cur, sweeps, stream);
        M1_CK(cudaGetLastError());
        if (cur == 1)
            M1_CK(cudaMemcpyAsync(h[0].u[0], h[0].u[1], sizeof(Cell4<R>) * h[0].n,
                                  cudaMemcpyDeviceToDevice, stream));
        dt_rhs = dt; rhs_valid = true;
        return M1_OK;
    }

    m1_status history(double* hs, double* dt, int len) override
    {
        const int n = std::min(len, std::min(last_cycles + 1, hist_len));
        if (n <= 0) return M1_OK;
        if (hs) M1_CK(cudaMemcpy(hs, hist, sizeof(double) * n, cudaMemcpyDeviceToHost));
        if (dt && n > 1) M1_CK(cudaMemcpy(dt, dtau_hist, sizeof(double) * (n - 1), cudaMemcpyDeviceToHost));
        return M1_OK;
    }

    // ---- single-kernel checks ----------------------------------------------------
    m1_status pack_planar(Cell4<R>* dst, int n, const double* planar)
    {
        M1_CK(cudaMemcpyAsync(stage, planar, sizeof(double) * 4 * n, cudaMemcpyHostToDevice, stream));
        m1::launch_pack_state<R>(stage, stage + n, stage + 2 * (size_t)n, stage + 3 * (size_t)n, 1.0, dst, n, stream);
        M1_CK(cudaGetLastError());
        return M1_OK;
    }
    m1_status unpack_planar(const Cell4<R>* src, int n, double* planar)
    {
        return unpack_from(src, n, planar, planar + n, planar + 2 * (size_t)n, planar + 3 * (size_t)n, 0);
    }
    m1_status set_sig_planar(const double* sig)
    {
        const int n = h[0].n;
        M1_CK(cudaMemcpyAsync(stage + 4 * (size_t)n, sig, sizeof(double) * 2 * n, cudaMemcpyHostToDevice, stream));
        m1::launch_pack_sig<R>(stage + 4 * (size_t)n, stage + 5 * (size_t)n, h[0].sig, n, stream);
        M1_CK(cudaGetLastError());
        return M1_OK;
    }
    m1_status set_ctl_simple(double dtau, double theta_ex, double theta_c)
    {
        Ctl c{};
        c.dtau = dtau; c.theta_ex = theta_ex; c.theta_c = theta_c;
        *ctl_h = c;
        M1_CK(cudaMemcpyAsync(ctl, ctl_h, sizeof(Ctl), cudaMemcpyHostToDevice, stream));
        return M1_OK;
    }

    m1_status op_level(double dt, const double* sig, const double* state, const double* rhs,
                       int mode, double dtau, double theta, double* out, double* norm)
    {
        const int n = h[0].n;
        M1_TRY(set_dt(dt));
        M1_TRY(set_sig_planar(sig));
        M1_TRY(set_ctl_simple(dtau, theta, 0.5));
        const Level<R>& q = h[0];
        switch (mode) {
        case M1_OP_APPLY:
            M1_TRY(pack_planar(q.u[0], n, state));
            m1::launch_apply<R>(d, q, m1::APPLY_A, 0, nullptr, 0, ctl, stream);
            M1_CK(cudaGetLastError());
            return unpack_planar(q.r, n, out);
        case M1_OP_RESIDUAL: {
            M1_TRY(pack_planar(q.u[0], n, state));
            M1_TRY(pack_planar(q.f, n, rhs));
            m1::launch_apply<R>(d, q, m1::APPLY_RESID, 0, part, 1, ctl, stream);
            M1_CK(cudaGetLastError());
            M1_TRY(unpack_planar(q.r, n, out));
            if (norm) {
                std::vector<double> p(q.tiles);
                M1_CK(cudaMemcpy(p.data(), part, sizeof(double) * p.size(), cudaMemcpyDeviceToHost));
                double s = 0.0;
                for (double x : p) s += x;
                *norm = std::sqrt(s);
            }
            return M1_OK;
        }
        case M1_OP_FAS_RHS:
            M1_TRY(pack_planar(q.v, n, state));
            M1_TRY(pack_planar(q.r, n, rhs));
            m1::launch_apply<R>(d, q, m1::APPLY_FAS, -1, nullptr, 0, ctl, stream);
            M1_CK(cudaGetLastError());
            return unpack_planar(q.f, n, out);
        case M1_OP_JACOBI:
        case M1_OP_PSEUDO:
            M1_TRY(pack_planar(q.u[0], n, state));
            M1_TRY(pack_planar(q.f, n, rhs));
            m1::launch_sweep<R>(d, q, mode == M1_OP_PSEUDO, 0, 1, ctl, stream);
            M1_CK(cudaGetLastError());
            return unpack_planar(q.u[1], n, out);
        default:
            return M1_ERR_INVALID_ARG;
        }
    }

    m1_status op_restrict(const double* state, const double* resid, double* cs, double* cr)
    {
        const int n = h[0].n;
        M1_TRY(set_ctl_simple(0, 0.5, 0.5));
        M1_TRY(pack_planar(h[0].u[0], n, state));
        M1_TRY(pack_planar(h[0].r, n, resid));
        m1::launch_restrict<R>(d, d + 1, h[1], 0, ctl, stream);
        M1_CK(cudaGetLastError());
        M1_TRY(unpack_planar(h[1].v, h[1].n, cs));
        return unpack_planar(h[1].r, h[1].n, cr);
    }

    m1_status op_prolong(const double* uc, const double* vc, const double* uf, double theta,
                         double* out, int* damped)
    {
        M1_TRY(set_ctl_simple(0, 0.5, theta));
        M1_TRY(pack_planar(h[1].u[0], h[1].n, uc));
        M1_TRY(pack_planar(h[1].v, h[1].n, vc));
        M1_TRY(pack_planar(h[0].u[0], h[0].n, uf));
        m1::launch_prolong<R>(d + 1, d, h[0], 0, 0, ctl, stream);
        M1_CK(cudaGetLastError());
        M1_TRY(unpack_planar(h[0].u[0], h[0].n, out));
        if (damped) {
            M1_CK(cudaMemcpy(ctl_h, ctl, sizeof(Ctl), cudaMemcpyDeviceToHost));
            *damped = (int)ctl_h->damped;
        }
        return M1_OK;
    }
};

// Mixed precision (row a11): the FP32 hierarchy `lo` runs the V-cycles of
// Algorithm 4 on the correction problem A32(u) = A32(v32) + r64; the FP64 fine
// level `hi` holds v^n, b and the opacities, computes the residual r64 and its
// norm (stop test, dtau control), and accumulates the corrections in FP64.
// Both share `hi`'s control block and stream.
struct MixedImpl : ImplBase {
    Impl<double> hi;
    Impl<float> lo;
    cudaGraphExec_t graph = nullptr;
    Params gparams{};

    ~MixedImpl() override
    {
        if (graph) cudaGraphExecDestroy(graph);
    }

    m1_status init(const m1_grid_desc& dsc, cudaStream_t s)
    {
        m1_grid_desc d = dsc;
        d.lmax = 1;
        d.precision = M1_FP64;
        M1_TRY(hi.init(d, s));
        M1_TRY(lo.init(dsc, hi.stream, true));
        lo.ctl = hi.ctl;
        return M1_OK;
    }

    m1_status set_state(const double* E, const double* Fx, const double* Fy, const double* T,
                        const double* sa, const double* ss, int dev) override
    {
        M1_TRY(hi.set_state(E, Fx, Fy, T, sa, ss, dev));
        return lo.set_state(E, Fx, Fy, T, sa, ss, dev);
    }

    m1_status set_inflow(int side, const double* E, const double* Fx, const double* Fy) override
    {
        M1_TRY(hi.set_inflow(side, E, Fx, Fy));
        return lo.set_inflow(side, E, Fx, Fy);
    }

    m1_status get_state(double* E, double* Fx, double* Fy, double* T, int dev) override
    {
        return hi.get_state(E, Fx, Fy, T, dev);
    }

    m1_status residual_norm(double dt, double* out) override { return hi.residual_norm(dt, out); }
    m1_status history(double* hs, double* dt, int len) override { return hi.history(hs, dt, len); }
    m1_status jacobi(double, int) override { return M1_ERR_INVALID_ARG; }

    // FP32 V-cycle, FP64 accumulation of its correction, FP64 defect of the new
    // iterate with the FP32 right-hand side of the next cycle, stop test.
    void record_mixed_cycle(const Params& p, cudaStream_t s)
    {
        int cur0 = 0;
        lo.record_cycle(p, cur0, s, false);
        m1::launch_accumulate(hi.d, hi.h[0], lo.d, cur0, hi.ctl, s);
        m1::launch_defect(hi.d, hi.h[0], lo.d, hi.part, hi.ctl, s);
        m1::launch_finalize(hi.ctl, hi.part, hi.h[0].tiles, nullptr, 0, m1::FIN_CYCLE, 0, s);
    }

    m1_status build_graph(const Params& p)
    {
        if (graph && gparams == p) return M1_OK;
        if (graph) { cudaGraphExecDestroy(graph); graph = nullptr; }
        cudaGraph_t g = nullptr;
        M1_CK(cudaStreamBeginCapture(lo.cap, cudaStreamCaptureModeThreadLocal));
        record_mixed_cycle(p, lo.cap);
        cudaError_t e = cudaStreamEndCapture(lo.cap, &g);
        if (e != cudaSuccess) { set_err(e, "cudaStreamEndCapture"); return M1_ERR_CUDA; }
        e = cudaGraphInstantiate(&graph, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) { set_err(e, "cudaGraphInstantiate"); graph = nullptr; return M1_ERR_CUDA; }
        gparams = p;
        return M1_OK;
    }

    m1_status step(double dt, const m1_solve_params& sp, m1_step_stats* st) override
    {
        if (!(dt > 0) || sp.nu0 < 1 || sp.nu_l != 1 || sp.m_pseudo < 1 || sp.m_coarse < 1 ||
            sp.max_cycles < 1 || !(sp.tol >= 0))
            return M1_ERR_INVALID_ARG;
        M1_TRY(hi.set_dt(dt));
        M1_TRY(lo.set_dt(dt));
        Params p{ sp.nu0, sp.nu_l, sp.m_pseudo, sp.m_coarse };
        M1_TRY(build_graph(p));
        Ctl c{};
        c.tol = sp.tol; c.grow = sp.grow; c.shrink = sp.shrink; c.eps_i = sp.eps_i;
        c.eps_d = sp.eps_d; c.dtau0 = sp.dtau0; c.dtau_min = sp.dtau_min; c.dtau_max = sp.dtau_max;
        c.theta_ex = sp.theta_ex; c.theta_c = sp.theta_c; c.max_cycles = sp.max_cycles;
        c.hist_len = hi.hist_len; c.hist = hi.hist; c.dtau_hist = hi.dtau_hist;
        c.res0_floor = 1e-14 * (double)hi.h[0].diag;
        *hi.ctl_h = c;
        cudaStream_t s = hi.stream;
        M1_CK(cudaEventRecord(hi.ev0, s));
        M1_CK(cudaMemcpyAsync(hi.ctl, hi.ctl_h, sizeof(Ctl), cudaMemcpyHostToDevice, s));
        m1::launch_make_rhs<double>(hi.d, hi.h[0], 0, s);
        m1::launch_norm_state<double>(hi.d, hi.h[0], hi.h[0].f, hi.partb, s);
        m1::launch_defect(hi.d, hi.h[0], lo.d, hi.part, hi.ctl, s);
        m1::launch_finalize(hi.ctl, hi.part, hi.h[0].tiles, hi.partb, hi.h[0].tiles, m1::FIN_INIT, 0, s);
        M1_CK(cudaGetLastError());
        hi.dt_rhs = dt; hi.rhs_valid = true;
        long long launched = 0;
        M1_TRY(run_until_done(graph, 1, sp.max_cycles, s, hi.ctl, hi.done_h, hi.poll, &launched));
        M1_CK(cudaMemcpyAsync(hi.ctl_h, hi.ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, s));
        M1_CK(cudaEventRecord(hi.ev1, s));
        M1_CK(cudaEventSynchronize(hi.ev1));
        hi.last_cycles = hi.ctl_h->kappa;
        if (st) {
            float ms = 0.f;
            cudaEventElapsedTime(&ms, hi.ev0, hi.ev1);
            st->cycles = hi.ctl_h->kappa;
            st->res0 = hi.ctl_h->res0;
            st->res = hi.ctl_h->kappa > 0 ? hi.ctl_h->res : hi.ctl_h->res0;
            st->dtau_final = hi.ctl_h->dtau;
            st->sweeps = (long long)hi.ctl_h->kappa * (lo.L == 1 ? p.nu0 : 2 * p.nu0);
            st->ms = ms;
            st->status = hi.ctl_h->status;
            st->newton_fail = hi.ctl_h->newton_fail;
            st->damped = hi.ctl_h->damped;
            st->launches = 4 + launched * (lo.kernels_per_cycle(p) + 1);
        }
        return hi.ctl_h->status == m1::CTL_OK ? M1_OK : M1_ERR_NOT_CONVERGED;
    }
};

m1_status validate(const m1_grid_desc* d)
{
    if (!d) return M1_ERR_INVALID_ARG;
    if (d->dim != 1 && d->dim != 2) return M1_ERR_INVALID_ARG;
    if (d->dim == 1 && d->ny != 1) return M1_ERR_INVALID_ARG;
    if (d->nx < 1 || d->ny < 1 || d->lmax < 1 || d->lmax > 20) return M1_ERR_INVALID_ARG;
    if (!(d->lx > 0) || (d->dim == 2 && !(d->ly > 0))) return M1_ERR_INVALID_ARG;
    if (!(d->c > 0) || !(d->a_r > 0) || !(d->c_v > 0)) return M1_ERR_INVALID_ARG;
    if (d->precision != M1_FP64 && d->precision != M1_MIXED) return M1_ERR_INVALID_ARG;
    const long long div = 1LL << (d->lmax - 1);
    if (d->nx % div) return M1_ERR_INVALID_ARG;
    if (d->dim == 2 && d->ny % div) return M1_ERR_INVALID_ARG;
    if ((long long)d->nx * d->ny > (1LL << 30)) return M1_ERR_INVALID_ARG;
    for (int w = 0; w < 4; ++w)
        if (d->bc[w] < M1_BC_PERIODIC || d->bc[w] > M1_BC_INFLOW) return M1_ERR_INVALID_ARG;
    // periodic walls come in pairs
    if ((d->bc[0] == M1_BC_PERIODIC) != (d->bc[1] == M1_BC_PERIODIC)) return M1_ERR_INVALID_ARG;
    if (d->dim == 2 && (d->bc[2] == M1_BC_PERIODIC) != (d->bc[3] == M1_BC_PERIODIC))
        return M1_ERR_INVALID_ARG;
    return M1_OK;
}

template <typename R>
m1_status make_op_impl(const m1_grid_desc* desc, int lmax, const double* inflow,
                       std::unique_ptr<Impl<R>>& out)
{
    m1_grid_desc d = *desc;
    d.lmax = lmax;
    M1_TRY(validate(&d));
    out.reset(new Impl<R>());
    M1_TRY(out->init(d, nullptr));
    if (inflow) {
        const int Lp = std::max(d.nx, d.dim == 2 ? d.ny : 1);
        for (int w = 0; w < 4; ++w)
            if (d.bc[w] == M1_BC_INFLOW)
                M1_TRY(out->set_inflow(w, inflow + (size_t)(w * 3) * Lp, inflow + (size_t)(w * 3 + 1) * Lp,
                                       inflow + (size_t)(w * 3 + 2) * Lp));
    }
    return M1_OK;
}

}  // namespace

namespace m1 {
void set_error_text(const char* msg) { std::snprintf(g_err, sizeof(g_err), "%s", msg); }
}  // namespace m1

struct m1_grid {
    std::unique_ptr<ImplBase> impl;
};

extern "C" {

const char* m1_last_error(void) { return g_err; }

m1_status m1_default_params(m1_solve_params* p)
{
    if (!p) return M1_ERR_INVALID_ARG;
    p->nu0 = 3; p->nu_l = 1; p->m_pseudo = 3; p->m_coarse = 3;
    p->dtau0 = 1e-3; p->grow = 1.1; p->shrink = 0.5; p->eps_i = 1e-2; p->eps_d = 1e-4;
    p->tol = 1e-8; p->dtau_min = 1e-12; p->dtau_max = 1e6; p->theta_ex = 0.5; p->theta_c = 0.5;
    p->max_cycles = 20000;
    return M1_OK;
}

m1_status m1_create_grid(const m1_grid_desc* desc, void* cuda_stream, m1_grid_t* out)
{
    if (!out) return M1_ERR_INVALID_ARG;
    *out = nullptr;
    M1_TRY(validate(desc));
    m1_grid* g = new m1_grid;
    m1_status s;
    if (desc->precision == M1_MIXED) {
        std::unique_ptr<MixedImpl> impl(new MixedImpl());
        s = impl->init(*desc, static_cast<cudaStream_t>(cuda_stream));
        g->impl = std::move(impl);
    } else {
        std::unique_ptr<Impl<double>> impl(new Impl<double>());
        s = impl->init(*desc, static_cast<cudaStream_t>(cuda_stream));
        g->impl = std::move(impl);
    }
    if (s != M1_OK) { delete g; return s; }
    *out = g;
    return M1_OK;
}

m1_status m1_destroy_grid(m1_grid_t g)
{
    if (!g) return M1_ERR_INVALID_ARG;
    delete g;
    return M1_OK;
}

m1_status m1_set_state(m1_grid_t g, const double* E, const double* Fx, const double* Fy,
                       const double* T, const double* sig_a, const double* sig_s, int on_device)
{
    if (!g) return M1_ERR_INVALID_ARG;
    return g->impl->set_state(E, Fx, Fy, T, sig_a, sig_s, on_device);
}

m1_status m1_set_inflow(m1_grid_t g, int side, const double* E, const double* Fx, const double* Fy)
{
    if (!g) return M1_ERR_INVALID_ARG;
    return g->impl->set_inflow(side, E, Fx, Fy);
}

m1_status m1_get_state(m1_grid_t g, double* E, double* Fx, double* Fy, double* T, int on_device)
{
    if (!g) return M1_ERR_INVALID_ARG;
    return g->impl->get_state(E, Fx, Fy, T, on_device);
}

m1_status m1_implicit_step(m1_grid_t g, double dt, const m1_solve_params* params,
                           m1_step_stats* stats)
{
    if (!g) return M1_ERR_INVALID_ARG;
    m1_solve_params p;
    if (params) p = *params; else m1_default_params(&p);
    return g->impl->step(dt, p, stats);
}

m1_status m1_residual_norm(m1_grid_t g, double dt, double* out)
{
    if (!g) return M1_ERR_INVALID_ARG;
    return g->impl->residual_norm(dt, out);
}

m1_status m1_jacobi(m1_grid_t g, double dt, int sweeps)
{
    if (!g) return M1_ERR_INVALID_ARG;
    return g->impl->jacobi(dt, sweeps);
}

m1_status m1_step_history(m1_grid_t g, double* hist, double* dtau, int len)
{
    if (!g) return M1_ERR_INVALID_ARG;
    return g->impl->history(hist, dtau, len);
}

m1_status m1_op_level(const m1_grid_desc* desc, const double* inflow, double dt, const double* sig,
                      const double* state, const double* rhs, int mode, double dtau, double theta,
                      double* out, double* norm)
{
    if (!desc || !sig || !state || !out || !(dt > 0)) return M1_ERR_INVALID_ARG;
    if (mode != M1_OP_APPLY && !rhs) return M1_ERR_INVALID_ARG;
    if (desc->precision == M1_FP64) {
        std::unique_ptr<Impl<double>> im;
        M1_TRY(make_op_impl(desc, 1, inflow, im));
        return im->op_level(dt, sig, state, rhs, mode, dtau, theta, out, norm);
    }
    std::unique_ptr<Impl<float>> im;
    M1_TRY(make_op_impl(desc, 1, inflow, im));
    return im->op_level(dt, sig, state, rhs, mode, dtau, theta, out, norm);
}

m1_status m1_op_restrict(const m1_grid_desc* fine, const double* inflow, const double* state,
                         const double* resid, double* coarse_state, double* coarse_resid)
{
    if (!fine || !state || !resid || !coarse_state || !coarse_resid) return M1_ERR_INVALID_ARG;
    if (fine->precision == M1_FP64) {
        std::unique_ptr<Impl<double>> im;
        M1_TRY(make_op_impl(fine, 2, inflow, im));
        return im->op_restrict(state, resid, coarse_state, coarse_resid);
    }
    std::unique_ptr<Impl<float>> im;
    M1_TRY(make_op_impl(fine, 2, inflow, im));
    return im->op_restrict(state, resid, coarse_state, coarse_resid);
}

m1_status m1_op_prolong_correct(const m1_grid_desc* fine, const double* uc, const double* vc,
                                const double* uf, double theta, double* out, int* damped)
{
    if (!fine || !uc || !vc || !uf || !out) return M1_ERR_INVALID_ARG;
    if (fine->precision == M1_FP64) {
        std::unique_ptr<Impl<double>> im;
        M1_TRY(make_op_impl(fine, 2, nullptr, im));
        return im->op_prolong(uc, vc, uf, theta, out, damped);
    }
    std::unique_ptr<Impl<float>> im;
    M1_TRY(make_op_impl(fine, 2, nullptr, im));
    return im->op_prolong(uc, vc, uf, theta, out, damped);
}

}  // extern "C"
