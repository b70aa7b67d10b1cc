// Host side of libm1: slot-based engines (one engine = instances sharing a level
// count and a precision; a single grid is an engine with one slot), the V-cycle
// of Algorithm 4 (Appendix A) recorded once into a CUDA graph whose persistent
// kernels walk device-resident work lists and relaunched until every instance's
// device-side stop flag is set, and the C ABI declared in include/m1.h.
#include <m1.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <memory>
#include <vector>

#include <type_traits>

#include "m1_engine.h"

namespace m1 {

thread_local char g_err[512] = "";

void set_error_text(const char* msg) { std::snprintf(g_err, sizeof(g_err), "%s", msg); }

void set_err(cudaError_t e, const char* what)
{
    std::snprintf(g_err, sizeof(g_err), "%s: %s", what, cudaGetErrorString(e));
}

// Relaunch a captured cycle graph until the batch control block reports that
// every active instance is done.  Batch k is queued before the host waits on the
// flag copied after batch k-1, so the GPU never idles on the poll; cycles queued
// past convergence return at once (every kernel checks its instance's flag).
// At most max_cycles + 2 graphs' worth are launched.
m1_status run_until_done(cudaGraphExec_t graph, int graph_cycles, int max_cycles,
                         cudaStream_t stream, BatchCtl* bctl, int* done_h, cudaEvent_t* poll,
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
        M1_CK(cudaMemcpyAsync(done_h + slot, &bctl->all_done, sizeof(int), cudaMemcpyDeviceToHost,
                              stream));
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

m1_status validate_desc(const m1_grid_desc* d)
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

m1_status validate_params(const m1_solve_params& sp)
{
    if (sp.nu0 < 1 || sp.nu_l != 1 || sp.m_pseudo < 1 || sp.m_coarse < 1 || sp.max_cycles < 1 ||
        !(sp.tol >= 0) || !(sp.dtau0 > 0) || !(sp.theta_ex > 0) || !(sp.theta_c > 0) ||
        (sp.dtau_rule != M1_DTAU_ABS && sp.dtau_rule != M1_DTAU_SIGNED) ||
        sp.cycle < M1_CYCLE_V || sp.cycle > M1_CYCLE_F)
        return M1_ERR_INVALID_ARG;
    return M1_OK;
}

Ctl make_ctl(const m1_solve_params& sp, double diag0)
{
    Ctl c{};
    c.tol = sp.tol; c.grow = sp.grow; c.shrink = sp.shrink; c.eps_i = sp.eps_i;
    c.eps_d = sp.eps_d; c.dtau0 = sp.dtau0; c.dtau_min = sp.dtau_min; c.dtau_max = sp.dtau_max;
    c.theta_ex = sp.theta_ex; c.theta_c = sp.theta_c; c.max_cycles = sp.max_cycles;
    c.dtau_rule = sp.dtau_rule;
    c.res0_floor = 1e-14 * diag0;   // rounding floor of evaluating A
    // double words carry ~48 bits: the defect they form differs from the FP64
    // one by at most ~4e-15 diag ||b|| (measured at converged states of the hot
    // square and the beam, where the terms of A are general numbers); the cycles
    // take it only when tol ||r_0|| is over 1000 times that, so its noise stays
    // below 0.1% of the stop test's threshold
    c.dw_floor = 5e-12 * diag0;
    c.active = 1;
    return c;
}

// ---------------------------------------------------------------------------
template <typename R>
Engine<R>::~Engine()
{
    if (graph) cudaGraphExecDestroy(graph);
    if (stream) cudaStreamSynchronize(stream);
    for (auto& v : mem)
        for (void* p : v) cudaFree(p);
    for (void* p : common) cudaFree(p);
    for (DevList* l : all_lists()) {
        if (l->items) cudaFree(l->items);
        if (l->count) cudaFree(l->count);
    }
    if (ctl_h) cudaFreeHost(ctl_h);
    if (bctl_h) cudaFreeHost(bctl_h);
    if (done_h) cudaFreeHost(done_h);
    if (bad_h) cudaFreeHost(bad_h);
    if (ev0) cudaEventDestroy(ev0);
    if (ev1) cudaEventDestroy(ev1);
    for (auto& e : poll)
        if (e) cudaEventDestroy(e);
    if (cap_stream) cudaStreamDestroy(cap_stream);
    if (own_stream && stream) cudaStreamDestroy(stream);
}

template <typename R>
std::vector<DevList*> Engine<R>::all_lists()
{
    std::vector<DevList*> v;
    for (auto& l : chunks) v.push_back(&l);
    for (auto& l : strips) v.push_back(&l);
    v.push_back(&init_strips);
    v.push_back(&init_chunks);
    return v;
}

template <typename R>
m1_status Engine<R>::calloc_common(void** p, size_t bytes)
{
    M1_CK(cudaMalloc(p, std::max<size_t>(bytes, 8)));
    common.push_back(*p);
    return M1_OK;
}

template <typename R>
m1_status Engine<R>::init(int capacity, int levels, bool correction_form, cudaStream_t s,
                          int history_len)
{
    cap = capacity;
    L = levels;
    delta = correction_form;
    if (s) stream = s;
    else { M1_CK(cudaStreamCreateWithFlags(&stream, cudaStreamNonBlocking)); own_stream = true; }
    M1_CK(cudaStreamCreateWithFlags(&cap_stream, cudaStreamNonBlocking));
    M1_CK(cudaEventCreate(&ev0));
    M1_CK(cudaEventCreate(&ev1));
    M1_CK(cudaEventCreateWithFlags(&poll[0], cudaEventDisableTiming));
    M1_CK(cudaEventCreateWithFlags(&poll[1], cudaEventDisableTiming));
    desc.assign(cap, m1_grid_desc{});
    used.assign(cap, 0);
    mem.assign(cap, {});
    h.assign((size_t)L * cap, Level<R>{});
    prof.assign((size_t)L * cap, {});
    dt_set.assign(cap, NAN);
    dt_rhs.assign(cap, NAN);
    rhs_valid.assign(cap, 0);
    last_cycles.assign(cap, 0);
    chunks.assign(L, DevList{});
    strips.assign(L, DevList{});
    M1_TRY(calloc_common((void**)&d, sizeof(Level<R>) * L * cap));
    M1_TRY(calloc_common((void**)&ctl, sizeof(Ctl) * cap));
    M1_TRY(calloc_common((void**)&bctl, sizeof(BatchCtl)));
    M1_TRY(calloc_common((void**)&init_slots, sizeof(int) * cap));
    M1_TRY(calloc_common((void**)&bad, sizeof(unsigned int)));
    M1_CK(cudaMallocHost(&ctl_h, sizeof(Ctl) * cap));
    M1_CK(cudaMallocHost(&bctl_h, sizeof(BatchCtl)));
    M1_CK(cudaMallocHost(&done_h, 2 * sizeof(int)));
    M1_CK(cudaMallocHost(&bad_h, sizeof(unsigned int)));
    std::memset(ctl_h, 0, sizeof(Ctl) * cap);
    std::memset(bctl_h, 0, sizeof(BatchCtl));
    M1_CK(cudaMemsetAsync(ctl, 0, sizeof(Ctl) * cap, stream));
    M1_CK(cudaMemsetAsync(bctl, 0, sizeof(BatchCtl), stream));
    hist_len = history_len;
    if (hist_len > 0) {
        M1_TRY(calloc_common((void**)&hist, sizeof(double) * hist_len * cap));
        M1_TRY(calloc_common((void**)&dtau_hist, sizeof(double) * hist_len * cap));
    }
    M1_CK(cudaStreamSynchronize(stream));
    return M1_OK;
}

// Keep double-word copies of every slot's level-0 iterate, right-hand side and
// opacities (slots added afterwards get them).
template <typename R>
m1_status Engine<R>::enable_dw()
{
    dw = true;
    dwh.assign(cap, DwLevel{ nullptr, nullptr, nullptr });
    M1_TRY(calloc_common((void**)&dwd, sizeof(DwLevel) * cap));
    M1_CK(cudaMemsetAsync(dwd, 0, sizeof(DwLevel) * cap, stream));
    return M1_OK;
}

template <typename R>
m1_status Engine<R>::slot_alloc(int i, void** p, size_t bytes)
{
    M1_CK(cudaMalloc(p, std::max<size_t>(bytes, 16)));
    mem[i].push_back(*p);
    return M1_OK;
}

template <typename R>
m1_status Engine<R>::add_slot(const m1_grid_desc& dsc, int* out)
{
    int i = -1;
    for (int k = 0; k < cap; ++k)
        if (!used[k]) { i = k; break; }
    if (i < 0) return M1_ERR_REJECTED;
    m1_grid_desc g = dsc;
    g.lmax = L;
    desc[i] = g;
    int nx = g.nx, ny = g.dim == 2 ? g.ny : 1;
    double hx = g.lx / g.nx, hy = g.dim == 2 ? g.ly / g.ny : 1.0;
    for (int l = 0; l < L; ++l) {
        Level<R>& q = h[(size_t)l * cap + i];
        std::memset(&q, 0, sizeof(q));
        q.dim = g.dim; q.nx = nx; q.ny = ny; q.n = nx * ny;
        for (int w = 0; w < 4; ++w) q.bc[w] = g.bc[w];
        q.chunks = (q.n + kThreads - 1) / kThreads;
        q.prof_len = std::max(nx, ny);
        // strip height: the autotuned value for this level size and precision
        q.sh = g.dim == 2 ? strip_rows(sizeof(R) == 4 ? 1 : 0, nx, ny) : 1;
        q.ring = (sizeof(R) == 4 && delta && g.dim == 2) ? strip_ring(nx, ny) : 0;
        q.sx = (nx + kStripW - 1) / kStripW;
        q.strips = q.sx * ((ny + q.sh - 1) / q.sh);
        q.c = (R)g.c; q.a_r = (R)g.a_r; q.c_v = (R)g.c_v;
        q.ic2 = (R)(1.0 / (g.c * g.c));
        q.vol = g.dim == 2 ? hx * hy : hx;
        const size_t c4 = sizeof(Cell4<R>) * q.n;
        M1_TRY(slot_alloc(i, (void**)&q.v, c4));
        M1_TRY(slot_alloc(i, (void**)&q.u[0], c4));
        M1_TRY(slot_alloc(i, (void**)&q.u[1], c4));
        M1_TRY(slot_alloc(i, (void**)&q.f, c4));
        M1_TRY(slot_alloc(i, (void**)&q.r, c4));
        if (delta) {
            M1_TRY(slot_alloc(i, (void**)&q.w, c4));
            M1_TRY(slot_alloc(i, (void**)&q.aw, c4));
        }
        M1_TRY(slot_alloc(i, (void**)&q.sig, sizeof(Sig2<R>) * q.n));
        M1_TRY(slot_alloc(i, (void**)&q.inflow, sizeof(R) * 12 * q.prof_len));
        M1_CK(cudaMemsetAsync(q.inflow, 0, sizeof(R) * 12 * q.prof_len, stream));
        M1_CK(cudaMemsetAsync(q.sig, 0, sizeof(Sig2<R>) * q.n, stream));
        prof[(size_t)l * cap + i].assign((size_t)12 * q.prof_len, 0.0);
        if (dw && l == 0) {
            DwLevel& D = dwh[i];
            M1_TRY(slot_alloc(i, (void**)&D.v, sizeof(DW4) * q.n));
            M1_TRY(slot_alloc(i, (void**)&D.b, sizeof(DW4) * q.n));
            M1_TRY(slot_alloc(i, (void**)&D.sig, sizeof(DW2) * q.n));
            M1_CK(cudaMemcpyAsync(dwd + i, &D, sizeof(DwLevel), cudaMemcpyHostToDevice, stream));
        }
        nx /= 2; if (g.dim == 2) ny /= 2;
        hx *= 2; if (g.dim == 2) hy *= 2;
    }
    used[i] = 1;
    dt_set[i] = NAN;
    rhs_valid[i] = 0;
    last_cycles[i] = 0;
    ctl_h[i] = Ctl{};
    M1_CK(cudaMemcpyAsync(ctl + i, ctl_h + i, sizeof(Ctl), cudaMemcpyHostToDevice, stream));
    M1_TRY(ensure_stage((size_t)h[i].n));
    M1_CK(cudaStreamSynchronize(stream));
    *out = i;
    return M1_OK;
}

template <typename R>
m1_status Engine<R>::remove_slot(int i)
{
    if (i < 0 || i >= cap || !used[i]) return M1_ERR_INVALID_ARG;
    M1_CK(cudaStreamSynchronize(stream));
    for (void* p : mem[i]) cudaFree(p);
    mem[i].clear();
    used[i] = 0;
    if (dw) {
        dwh[i] = DwLevel{ nullptr, nullptr, nullptr };
        M1_CK(cudaMemcpyAsync(dwd + i, &dwh[i], sizeof(DwLevel), cudaMemcpyHostToDevice, stream));
    }
    for (int l = 0; l < L; ++l) std::memset(&h[(size_t)l * cap + i], 0, sizeof(Level<R>));
    ctl_h[i] = Ctl{};
    M1_CK(cudaMemcpyAsync(ctl + i, ctl_h + i, sizeof(Ctl), cudaMemcpyHostToDevice, stream));
    M1_CK(cudaStreamSynchronize(stream));
    return M1_OK;
}

template <typename R>
m1_status Engine<R>::ensure_stage(size_t n)
{
    if (n <= stage_n) return M1_OK;
    M1_CK(cudaStreamSynchronize(stream));
    auto drop = [this](void* p) {
        if (!p) return;
        cudaFree(p);
        common.erase(std::find(common.begin(), common.end(), p));
    };
    drop(stage);
    drop(sig_stage);
    void* p = nullptr;
    M1_TRY(calloc_common(&p, sizeof(double) * 6 * n));
    stage = static_cast<double*>(p);
    M1_TRY(calloc_common(&p, sizeof(Sig2<R>) * n));
    sig_stage = static_cast<Sig2<R>*>(p);
    stage_n = n;
    return M1_OK;
}

// Upload a host list into its device buffer, growing the buffer (which changes
// the pointers a captured graph holds, so the graph is rebuilt) when needed.
template <typename R>
m1_status Engine<R>::upload_list(DevList& l)
{
    const int n = (int)l.host.size();
    if (n > l.capacity || !l.items) {
        int capn = 1;
        while (capn < n) capn <<= 1;
        M1_CK(cudaStreamSynchronize(stream));
        if (l.items) cudaFree(l.items);
        if (l.count) cudaFree(l.count);
        l.items = nullptr;
        l.count = nullptr;
        M1_CK(cudaMalloc(&l.items, sizeof(int2) * capn));
        M1_CK(cudaMalloc(&l.count, sizeof(int)));
        l.capacity = capn;
        graph_dirty = true;
    }
    l.n = n;
    if (n)
        M1_CK(cudaMemcpyAsync(l.items, l.host.data(), sizeof(int2) * n, cudaMemcpyHostToDevice, stream));
    M1_CK(cudaMemcpyAsync(l.count, &l.n, sizeof(int), cudaMemcpyHostToDevice, stream));
    M1_CK(cudaStreamSynchronize(stream));
    return M1_OK;
}

// Work lists of every level over the used slots, the slots' offsets into the
// norm partials, and the descriptors, uploaded to the device.
template <typename R>
m1_status Engine<R>::rebuild()
{
    int off = 0;
    for (int i = 0; i < cap; ++i)
        if (used[i]) { h[i].part_off = off; off += h[i].strips; }
    if (off > part_cap || !part) {
        int capn = 1;
        while (capn < off) capn <<= 1;
        M1_CK(cudaStreamSynchronize(stream));
        auto drop = [this](void* p) {
            if (!p) return;
            cudaFree(p);
            common.erase(std::find(common.begin(), common.end(), p));
        };
        drop(part);
        drop(partb);
        M1_TRY(calloc_common((void**)&part, sizeof(double) * capn));
        M1_TRY(calloc_common((void**)&partb, sizeof(double) * capn));
        part_cap = capn;
        graph_dirty = true;
    }
    for (int l = 0; l < L; ++l) {
        chunks[l].host.clear();
        strips[l].host.clear();
        for (int i = 0; i < cap; ++i) {
            if (!used[i]) continue;
            const Level<R>& q = h[(size_t)l * cap + i];
            for (int t = 0; t < q.strips; ++t) strips[l].host.push_back(make_int2(i, t));
            for (int c = 0; c < q.chunks; ++c) chunks[l].host.push_back(make_int2(i, c));
        }
        M1_TRY(upload_list(strips[l]));
        M1_TRY(upload_list(chunks[l]));
    }
    // a captured cycle launches nothing for an empty list: re-capture when a
    // list becomes empty or stops being empty
    std::vector<char> sig;
    for (int l = 0; l < L; ++l) {
        sig.push_back(strips[l].n > 0);
        sig.push_back(chunks[l].n > 0);
    }
    if (sig != list_sig) { list_sig = sig; graph_dirty = true; }
    // the sweeps of a level share one launch for all slots: the cp.async kernel
    // when the slots holding most of the level's cells chose it
    std::vector<char> rl(L, 0);
    for (int l = 0; l < L; ++l) {
        long long with = 0, without = 0;
        for (int i = 0; i < cap; ++i)
            if (used[i]) {
                const Level<R>& q = h[(size_t)l * cap + i];
                (q.ring ? with : without) += q.n;
            }
        rl[l] = with > without;
    }
    if (rl != ring) { ring = rl; graph_dirty = true; }
    M1_CK(cudaMemcpyAsync(d, h.data(), sizeof(Level<R>) * h.size(), cudaMemcpyHostToDevice, stream));
    M1_CK(cudaStreamSynchronize(stream));
    return M1_OK;
}

template <typename R>
m1_status Engine<R>::set_dt(int i, double dt)
{
    if (dt == dt_set[i]) return M1_OK;
    const m1_grid_desc& g = desc[i];
    for (int l = 0; l < L; ++l) {
        Level<R>& q = h[(size_t)l * cap + i];
        const double hx = g.lx / g.nx * (double)(1 << l);
        const double hy = g.dim == 2 ? g.ly / g.ny * (double)(1 << l) : 1.0;
        const double ax = g.c * dt / hx, ay = g.dim == 2 ? g.c * dt / hy : 0.0;
        q.ax = (R)ax; q.ay = (R)ay;
        q.bx = (R)(dt / (2.0 * hx)); q.by = g.dim == 2 ? (R)(dt / (2.0 * hy)) : R(0);
        q.diag = (R)(1.0 + ax + ay);
        q.cdt = (R)(g.c * dt);
        M1_CK(cudaMemcpyAsync(d + (size_t)l * cap + i, &q, sizeof(Level<R>), cudaMemcpyHostToDevice,
                              stream));
    }
    M1_CK(cudaStreamSynchronize(stream));   // h may change right after
    dt_set[i] = dt;
    return M1_OK;
}

// ---- state in / out ---------------------------------------------------------
template <typename R>
m1_status Engine<R>::pack_into(int i, Cell4<R>* dst, const double* E, const double* Fx,
                               const double* Fy, const double* T, int dev)
{
    const int n = h[i].n;
    if (!dev) {
        M1_CK(cudaMemcpyAsync(stage, E, n * 8, cudaMemcpyHostToDevice, stream));
        M1_CK(cudaMemcpyAsync(stage + n, Fx, n * 8, cudaMemcpyHostToDevice, stream));
        if (Fy) M1_CK(cudaMemcpyAsync(stage + 2 * (size_t)n, Fy, n * 8, cudaMemcpyHostToDevice, stream));
        M1_CK(cudaMemcpyAsync(stage + 3 * (size_t)n, T, n * 8, cudaMemcpyHostToDevice, stream));
        E = stage; Fx = stage + n; Fy = Fy ? stage + 2 * (size_t)n : nullptr; T = stage + 3 * (size_t)n;
    }
    launch_pack_state<R>(E, Fx, Fy, T, 1.0, dst, n, stream);
    M1_CK(cudaGetLastError());
    return M1_OK;
}

template <typename R>
m1_status Engine<R>::unpack_from(const Cell4<R>* src, int n, double* E, double* Fx, double* Fy,
                                 double* T, int dev)
{
    if (dev) {
        launch_unpack_state<R>(src, E, Fx, Fy, T, n, stream);
        M1_CK(cudaGetLastError());
        M1_CK(cudaStreamSynchronize(stream));
        return M1_OK;
    }
    double* s = stage;
    launch_unpack_state<R>(src, s, s + n, Fy ? s + 2 * (size_t)n : nullptr, s + 3 * (size_t)n, n, stream);
    M1_CK(cudaGetLastError());
    M1_CK(cudaMemcpyAsync(E, s, n * 8, cudaMemcpyDeviceToHost, stream));
    M1_CK(cudaMemcpyAsync(Fx, s + n, n * 8, cudaMemcpyDeviceToHost, stream));
    if (Fy) M1_CK(cudaMemcpyAsync(Fy, s + 2 * (size_t)n, n * 8, cudaMemcpyDeviceToHost, stream));
    M1_CK(cudaMemcpyAsync(T, s + 3 * (size_t)n, n * 8, cudaMemcpyDeviceToHost, stream));
    M1_CK(cudaStreamSynchronize(stream));
    return M1_OK;
}

template <typename R>
m1_status Engine<R>::set_state(int i, const double* E, const double* Fx, const double* Fy,
                               const double* T, const double* sa, const double* ss, int dev)
{
    if (i < 0 || i >= cap || !used[i]) return M1_ERR_INVALID_ARG;
    const Level<R>& q0 = h[i];
    const int n = q0.n;
    if (!E || !Fx || !T || (q0.dim == 2 && !Fy) || (!sa != !ss)) return M1_ERR_INVALID_ARG;
    // stage into u[1] / sig_stage, check, then commit
    M1_TRY(pack_into(i, q0.u[1], E, Fx, Fy, T, dev));
    const Sig2<R>* sig_chk = nullptr;
    if (sa) {
        const double *a = sa, *b = ss;
        if (!dev) {
            M1_CK(cudaMemcpyAsync(stage + 4 * (size_t)n, sa, n * 8, cudaMemcpyHostToDevice, stream));
            M1_CK(cudaMemcpyAsync(stage + 5 * (size_t)n, ss, n * 8, cudaMemcpyHostToDevice, stream));
            a = stage + 4 * (size_t)n;
            b = stage + 5 * (size_t)n;
        }
        launch_pack_sig<R>(a, b, sig_stage, n, stream);
        sig_chk = sig_stage;
    }
    M1_CK(cudaMemsetAsync(bad, 0, sizeof(unsigned int), stream));
    launch_check_state<R>(q0.u[1], sig_chk, n, desc[i].c, bad, stream);
    M1_CK(cudaGetLastError());
    M1_CK(cudaMemcpyAsync(bad_h, bad, sizeof(unsigned int), cudaMemcpyDeviceToHost, stream));
    M1_CK(cudaStreamSynchronize(stream));
    if (*bad_h) return M1_ERR_NONADMISSIBLE_INPUT;
    M1_CK(cudaMemcpyAsync(q0.u[0], q0.u[1], sizeof(Cell4<R>) * n, cudaMemcpyDeviceToDevice, stream));
    if (sa) {
        M1_CK(cudaMemcpyAsync(q0.sig, sig_stage, sizeof(Sig2<R>) * n, cudaMemcpyDeviceToDevice, stream));
        // opacities of the coarse levels: full weighting, one level after another
        for (int l = 1; l < L; ++l) {
            init_chunks.host.clear();
            for (int c = 0; c < h[(size_t)l * cap + i].chunks; ++c)
                init_chunks.host.push_back(make_int2(i, c));
            M1_TRY(upload_list(init_chunks));
            launch_restrict_sig<R>(d + (size_t)(l - 1) * cap, d + (size_t)l * cap, init_chunks.view(),
                                   stream);
            M1_CK(cudaGetLastError());
        }
    }
    rhs_valid[i] = 0;
    M1_CK(cudaStreamSynchronize(stream));
    return M1_OK;
}

template <typename R>
m1_status Engine<R>::set_inflow(int i, int side, const double* E, const double* Fx, const double* Fy)
{
    if (i < 0 || i >= cap || !used[i] || side < 0 || side > 3 || !E || !Fx || !Fy)
        return M1_ERR_INVALID_ARG;
    for (int l = 0; l < L; ++l) {
        const Level<R>& q = h[(size_t)l * cap + i];
        const int len = side < 2 ? q.ny : q.nx;
        const int pl = q.prof_len;
        std::vector<double>& P = prof[(size_t)l * cap + i];
        for (int fld = 0; fld < 3; ++fld) {
            double* dst = P.data() + (size_t)(side * 3 + fld) * pl;
            if (l == 0) {
                const double* src = fld == 0 ? E : (fld == 1 ? Fx : Fy);
                std::copy(src, src + len, dst);
            } else {
                const Level<R>& p = h[(size_t)(l - 1) * cap + i];
                const int nf = side < 2 ? p.ny : p.nx;
                restrict_profile(prof[(size_t)(l - 1) * cap + i].data() + (size_t)(side * 3 + fld) * p.prof_len,
                                 nf, dst, len);
            }
        }
        std::vector<R> tmp(P.begin(), P.end());
        M1_CK(cudaMemcpyAsync(q.inflow, tmp.data(), sizeof(R) * tmp.size(), cudaMemcpyHostToDevice, stream));
        M1_CK(cudaStreamSynchronize(stream));
    }
    return M1_OK;
}

template <typename R>
m1_status Engine<R>::get_state(int i, double* E, double* Fx, double* Fy, double* T, int dev)
{
    if (i < 0 || i >= cap || !used[i] || !E || !Fx || !T) return M1_ERR_INVALID_ARG;
    return unpack_from(h[i].u[0], h[i].n, E, Fx, Fy, T, dev);
}

// ---- the V-cycle ----------------------------------------------------------------
template <typename R>
void Engine<R>::sweeps_fine(int& cur, int count, cudaStream_t s)
{
    for (int k = 0; k < count; ++k) {
        launch_sweep<R>(d, strips[0].view(), ctl, false, cur, 1 - cur, s, delta, ring[0] != 0);
        cur = 1 - cur;
    }
}

// m pseudo-time steps (nu_l = 1 Jacobi sweep each) at level l; from_v: the
// first step starts from v_l (initial guess u_l = v_l, Algorithm 4).
// fas: the first step also forms the FAS right-hand side (plain form; the
// caller then launches no separate FAS kernel).
template <typename R>
void Engine<R>::pseudo(int l, int& cur, int m, bool from_v, cudaStream_t s, bool fas)
{
    Level<R>* dl = d + (size_t)l * cap;
    const bool go = strips[l].n > 0;          // an empty level only advances the buffer
    const bool rg = ring[l] != 0;
    for (int k = 0; k < m; ++k) {
        if (k == 0 && from_v) {
            if (go)
                launch_sweep<R>(dl, strips[l].view(), ctl, true, -1, 0, s, delta, rg, nullptr,
                                fas && !delta);
            cur = 0;
        } else {
            if (go) launch_sweep<R>(dl, strips[l].view(), ctl, true, cur, 1 - cur, s, delta, rg);
            cur = 1 - cur;
        }
    }
}

// The FAS right-hand side of coarse level l (Eq. (24)); in the correction form
// with the base operator A(w_l) in the same pass.
template <typename R>
void Engine<R>::fas_rhs(int l, cudaStream_t s)
{
    if (strips[l].n == 0) return;
    Level<R>* dl = d + (size_t)l * cap;
    if constexpr (std::is_same<R, float>::value) {
        if (delta) {
            launch_fas_aw32(dl, strips[l].view(), ctl, s);
            return;
        }
    }
    launch_apply<R>(dl, strips[l].view(), ctl, APPLY_FAS, -1, nullptr, 0, s, delta);
}

// Cycle shapes (Section 4.2 builds the V-cycle by recursion; Section 6.3 names
// W- and F-cycles): the coarse-grid corrections of level l are one visit of
// level l + 1 (V), two visits, the second continuing from the corrected
// iterate (W), or an F-visit then a repeated V-visit (F); the coarsest level is
// visited once per correction.  A fresh visit builds its FAS problem from the
// restriction of level l; a repeated one keeps its right-hand side and iterate.
template <typename R>
void Engine<R>::corrections(const Params& p, int l, int shape, std::vector<int>& cur, cudaStream_t s)
{
    if (l + 1 == L - 1 || shape == M1_CYCLE_V) {
        visit(p, l + 1, true, shape, cur, s);
    } else if (shape == M1_CYCLE_W) {
        visit(p, l + 1, true, M1_CYCLE_W, cur, s);
        visit(p, l + 1, false, M1_CYCLE_W, cur, s);
    } else {
        visit(p, l + 1, true, M1_CYCLE_F, cur, s);
        visit(p, l + 1, false, M1_CYCLE_V, cur, s);
    }
}

// One visit of coarse level l >= 1: FAS right-hand side (Eq. (24)) when fresh,
// m pseudo-time steps (Algorithm 3; the coarsest level: m_coarse and nothing
// else), residual, restriction, the coarse-grid corrections, prolongation with
// damping (Eq. (34)), m pseudo-time steps.
template <typename R>
void Engine<R>::visit(const Params& p, int l, bool fresh, int shape, std::vector<int>& cur,
                      cudaStream_t s)
{
    Level<R>* dl = d + (size_t)l * cap;
    // a fresh visit needs the FAS right-hand side first: the plain form forms
    // it inside the first pseudo-time step, the correction form in its own pass
    // (with A(w))
    if (fresh && delta) fas_rhs(l, s);
    if (l == L - 1) {
        pseudo(l, cur[l], p.mc, fresh, s, fresh);
        return;
    }
    pseudo(l, cur[l], p.m, fresh, s, fresh);
    if (strips[l].n)
        launch_apply<R>(dl, strips[l].view(), ctl, APPLY_RESID, cur[l], nullptr, 1, s, delta);
    if (chunks[l + 1].n)
        launch_restrict<R>(dl, dl + cap, chunks[l + 1].view(), ctl, cur[l], s, delta);
    corrections(p, l, shape, cur, s);
    if (chunks[l + 1].n)
        launch_prolong<R>(dl + cap, dl, chunks[l + 1].view(), ctl, cur[l + 1], cur[l], s, delta);
    pseudo(l, cur[l], p.m, false, s);
}

// One cycle of Algorithm 4 (of the shape p.cycle) over every instance.  tail:
// the stop test of the previous cycle at the start (the mixed-precision driver
// does its own after the cycle).  The residual norm of the state a cycle
// leaves is a by-product of the next cycle's first fine sweep, so the test of
// cycle k runs in the graph launch of cycle k + 1: the step takes one launch
// more than it has cycles, and no separate residual pass.
template <typename R>
void Engine<R>::record_cycle(const Params& p, int& cur0, cudaStream_t s, bool tail,
                             bool first_done)
{
    std::vector<int> cur(L, 0);
    cur[0] = cur0;
    if (tail) {
        // the first fine sweep also gives ||b - A(v)|| of the state the previous
        // cycle left (its stop test and dtau update, taken here: if that cycle
        // converged, the state stays in buffer `in` and the rest of this launch
        // returns at once)
        const int in = cur[0];
        launch_sweep<R>(d, strips[0].view(), ctl, false, in, 1 - in, s, delta, ring[0] != 0, part);
        cur[0] = 1 - in;
        launch_finalize<R>(ctl, d, cap, part, nullptr, FIN_DEFER, in, bctl, s);
        sweeps_fine(cur[0], p.nu0 - 1, s);
    } else if (first_done) {
        cur[0] = 1;
        sweeps_fine(cur[0], p.nu0 - 1, s);
    } else {
        sweeps_fine(cur[0], p.nu0, s);
    }
    if (L > 1) {
        launch_apply<R>(d, strips[0].view(), ctl, APPLY_RESID, cur[0], nullptr, 1, s, delta);
        if (chunks[1].n)
            launch_restrict<R>(d, d + cap, chunks[1].view(), ctl, cur[0], s, delta);
        corrections(p, 0, p.cycle, cur, s);
        if (chunks[1].n)
            launch_prolong<R>(d + cap, d, chunks[1].view(), ctl, cur[1], cur[0], s, delta);
        sweeps_fine(cur[0], p.nu0, s);
    }
    cur0 = cur[0];
}

namespace {

// Fresh and repeated visits of each level in one cycle of the given shape.
void count_visits(int L, int l, bool fresh, int shape, std::vector<long long>& fr,
                  std::vector<long long>& rep)
{
    (fresh ? fr : rep)[l] += 1;
    if (l == L - 1) return;
    if (l + 1 == L - 1 || shape == M1_CYCLE_V) {
        count_visits(L, l + 1, true, shape, fr, rep);
    } else if (shape == M1_CYCLE_W) {
        count_visits(L, l + 1, true, M1_CYCLE_W, fr, rep);
        count_visits(L, l + 1, false, M1_CYCLE_W, fr, rep);
    } else {
        count_visits(L, l + 1, true, M1_CYCLE_F, fr, rep);
        count_visits(L, l + 1, false, M1_CYCLE_V, fr, rep);
    }
}

}  // namespace

template <typename R>
long long Engine<R>::kernels_per_cycle(const Params& p) const
{
    if (L == 1) return p.nu0;
    // a fresh visit's FAS right-hand side: fused into the first pseudo-time step
    // in the plain form, its own kernel in the correction form
    const int aw = delta ? 1 : 0;
    std::vector<long long> fr(L, 0), rep(L, 0);
    count_visits(L, 0, true, p.cycle, fr, rep);
    long long k = 2 * p.nu0 + 3;                       // fine smoothing, residual, restrict, prolong
    for (int l = 1; l < L - 1; ++l)                    // pseudo x 2, residual, restrict, prolong
        k += fr[l] * (aw + 2 * p.m + 3) + rep[l] * (2 * p.m + 3);
    k += fr[L - 1] * (aw + p.mc);                      // coarsest
    return k;
}

template <typename R>
m1_status Engine<R>::build_graph(const Params& p)
{
    if (graph && gparams == p && !graph_dirty) return M1_OK;
    if (graph) { cudaGraphExecDestroy(graph); graph = nullptr; }
    // a captured graph must return the fine iterate to buffer 0
    const int per_cycle = L == 1 ? p.nu0 : 2 * p.nu0;
    graph_cycles = (per_cycle % 2) ? 2 : 1;
    cudaGraph_t g = nullptr;
    M1_CK(cudaStreamBeginCapture(cap_stream, cudaStreamCaptureModeThreadLocal));
    int cur0 = 0;
    for (int c = 0; c < graph_cycles; ++c) record_cycle(p, cur0, cap_stream);
    cudaError_t e = cudaStreamEndCapture(cap_stream, &g);
    if (e != cudaSuccess) { set_err(e, "cudaStreamEndCapture"); return M1_ERR_CUDA; }
    if (cur0 != 0) { cudaGraphDestroy(g); return M1_ERR_INVALID_ARG; }
    e = cudaGraphInstantiate(&graph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) { set_err(e, "cudaGraphInstantiate"); graph = nullptr; return M1_ERR_CUDA; }
    gparams = p;
    graph_dirty = false;
    return M1_OK;
}

// Control blocks of the used slots for a step (all used slots take part) and the
// batch completion counter.
template <typename R>
m1_status Engine<R>::begin_step(const double* dts, const m1_solve_params& sp)
{
    int nact = 0;
    for (int i = 0; i < cap; ++i) {
        if (!used[i]) { ctl_h[i] = Ctl{}; continue; }
        M1_TRY(set_dt(i, dts[i]));
        ctl_h[i] = make_ctl(sp, (double)h[i].diag);
        if (hist_len > 0) {
            ctl_h[i].hist_len = hist_len;
            ctl_h[i].hist = hist + (size_t)i * hist_len;
            ctl_h[i].dtau_hist = dtau_hist + (size_t)i * hist_len;
        }
        ++nact;
    }
    *bctl_h = BatchCtl{ 0, nact, 0, 0 };
    M1_CK(cudaMemcpyAsync(ctl, ctl_h, sizeof(Ctl) * cap, cudaMemcpyHostToDevice, stream));
    M1_CK(cudaMemcpyAsync(bctl, bctl_h, sizeof(BatchCtl), cudaMemcpyHostToDevice, stream));
    return M1_OK;
}

template <typename R>
m1_status Engine<R>::step(const double* dts, const m1_solve_params& sp, m1_step_stats* st)
{
    M1_TRY(validate_params(sp));
    for (int i = 0; i < cap; ++i)
        if (used[i] && !(dts[i] > 0)) return M1_ERR_INVALID_ARG;
    Params p{ sp.nu0, sp.nu_l, sp.m_pseudo, sp.m_coarse, sp.cycle };
    M1_TRY(build_graph(p));
    M1_TRY(begin_step(dts, sp));
    M1_CK(cudaEventRecord(ev0, stream));
    const WorkList t0 = strips[0].view(), c0 = chunks[0].view();
    launch_make_rhs<R>(d, c0, ctl, 0, stream);
    launch_apply<R>(d, t0, ctl, APPLY_RESID, 0, part, 0, stream);
    launch_norm_state<R>(d, t0, ctl, partb, stream);
    launch_finalize<R>(ctl, d, cap, part, partb, FIN_INIT, 0, bctl, stream);
    M1_CK(cudaGetLastError());
    for (int i = 0; i < cap; ++i)
        if (used[i]) { dt_rhs[i] = dts[i]; rhs_valid[i] = 1; }
    long long launched = 0;
    M1_TRY(run_until_done(graph, graph_cycles, sp.max_cycles, stream, bctl, done_h, poll, &launched));
    M1_CK(cudaMemcpyAsync(ctl_h, ctl, sizeof(Ctl) * cap, cudaMemcpyDeviceToHost, stream));
    M1_CK(cudaStreamSynchronize(stream));
    for (int i = 0; i < cap; ++i)
        if (used[i] && ctl_h[i].result_buf == 1)
            M1_CK(cudaMemcpyAsync(h[i].u[0], h[i].u[1], sizeof(Cell4<R>) * h[i].n,
                                  cudaMemcpyDeviceToDevice, stream));
    M1_CK(cudaEventRecord(ev1, stream));
    M1_CK(cudaEventSynchronize(ev1));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, ev0, ev1);
    bool all_ok = true;
    int k = 0;
    for (int i = 0; i < cap; ++i) {
        if (!used[i]) continue;
        const Ctl& c = ctl_h[i];
        last_cycles[i] = c.kappa;
        all_ok = all_ok && c.status == CTL_OK;
        if (st) {
            m1_step_stats& s = st[k];
            s.cycles = c.kappa;
            s.res0 = c.res0;
            s.res = c.kappa > 0 ? c.res : c.res0;
            s.dtau_final = c.dtau;
            s.sweeps = (long long)c.kappa * (L == 1 ? p.nu0 : 2 * p.nu0);
            s.ms = ms;
            s.status = c.status;
            s.newton_fail = c.newton_fail;
            s.damped = c.damped;
            s.launches = 4 + launched * (kernels_per_cycle(p) + 1);   // + deferred finalize
        }
        ++k;
    }
    return all_ok ? M1_OK : M1_ERR_NOT_CONVERGED;
}

template <typename R>
m1_status Engine<R>::residual_norm(int i, double dt, double* out)
{
    if (i < 0 || i >= cap || !used[i] || !out || !(dt > 0)) return M1_ERR_INVALID_ARG;
    M1_TRY(set_dt(i, dt));
    init_strips.host.clear();
    init_chunks.host.clear();
    for (int t = 0; t < h[i].strips; ++t) init_strips.host.push_back(make_int2(i, t));
    for (int c = 0; c < h[i].chunks; ++c) init_chunks.host.push_back(make_int2(i, c));
    M1_TRY(upload_list(init_strips));
    M1_TRY(upload_list(init_chunks));
    if (!(rhs_valid[i] && dt == dt_rhs[i]))
        launch_make_rhs<R>(d, init_chunks.view(), nullptr, 0, stream);
    launch_apply<R>(d, init_strips.view(), nullptr, APPLY_RESID, 0, part, 0, stream);
    M1_CK(cudaGetLastError());
    std::vector<double> p(h[i].strips);
    M1_CK(cudaMemcpyAsync(p.data(), part + h[i].part_off, sizeof(double) * p.size(),
                          cudaMemcpyDeviceToHost, stream));
    M1_CK(cudaStreamSynchronize(stream));
    double s = 0.0;
    for (double x : p) s += x;
    *out = std::sqrt(s);
    return M1_OK;
}

template <typename R>
m1_status Engine<R>::history(int i, double* hs, double* dt, int len)
{
    if (i < 0 || i >= cap || !used[i]) return M1_ERR_INVALID_ARG;
    const int n = std::min(len, std::min(last_cycles[i] + 1, hist_len));
    if (n <= 0) return M1_OK;
    if (hs) M1_CK(cudaMemcpy(hs, hist + (size_t)i * hist_len, sizeof(double) * n, cudaMemcpyDeviceToHost));
    if (dt && n > 1)
        M1_CK(cudaMemcpy(dt, dtau_hist + (size_t)i * hist_len, sizeof(double) * (n - 1),
                         cudaMemcpyDeviceToHost));
    return M1_OK;
}

template <typename R>
m1_status Engine<R>::set_ctl_simple(int i, double dtau, double theta_ex, double theta_c)
{
    Ctl c{};
    c.dtau = dtau; c.theta_ex = theta_ex; c.theta_c = theta_c; c.active = 1;
    ctl_h[i] = c;
    M1_CK(cudaMemcpyAsync(ctl + i, ctl_h + i, sizeof(Ctl), cudaMemcpyHostToDevice, stream));
    return M1_OK;
}

template <typename R>
m1_status Engine<R>::jacobi(int i, double dt, int sweeps)
{
    if (cap != 1 || i != 0 || !used[0] || !(dt > 0) || sweeps < 0) return M1_ERR_INVALID_ARG;
    M1_TRY(set_dt(0, dt));
    M1_TRY(set_ctl_simple(0, 0.0, 0.5, 0.5));
    launch_make_rhs<R>(d, chunks[0].view(), ctl, 0, stream);
    int cur = 0;
    sweeps_fine(cur, sweeps, stream);
    M1_CK(cudaGetLastError());
    if (cur == 1)
        M1_CK(cudaMemcpyAsync(h[0].u[0], h[0].u[1], sizeof(Cell4<R>) * h[0].n,
                              cudaMemcpyDeviceToDevice, stream));
    dt_rhs[0] = dt;
    rhs_valid[0] = 1;
    return M1_OK;
}

// ---- single-kernel checks (slot 0) -----------------------------------------------
template <typename R>
m1_status Engine<R>::pack_planar(Cell4<R>* dst, int n, const double* planar)
{
    M1_CK(cudaMemcpyAsync(stage, planar, sizeof(double) * 4 * n, cudaMemcpyHostToDevice, stream));
    launch_pack_state<R>(stage, stage + n, stage + 2 * (size_t)n, stage + 3 * (size_t)n, 1.0, dst, n,
                         stream);
    M1_CK(cudaGetLastError());
    return M1_OK;
}

template <typename R>
m1_status Engine<R>::unpack_planar(const Cell4<R>* src, int n, double* planar)
{
    return unpack_from(src, n, planar, planar + n, planar + 2 * (size_t)n, planar + 3 * (size_t)n, 0);
}

template <typename R>
m1_status Engine<R>::op_level(double dt, const double* sig, const double* state, const double* rhs,
                              int mode, double dtau, double theta, double* out, double* norm)
{
    const Level<R>& q = h[0];
    const int n = q.n;
    M1_TRY(set_dt(0, dt));
    M1_CK(cudaMemcpyAsync(stage + 4 * (size_t)n, sig, sizeof(double) * 2 * n, cudaMemcpyHostToDevice,
                          stream));
    launch_pack_sig<R>(stage + 4 * (size_t)n, stage + 5 * (size_t)n, q.sig, n, stream);
    M1_TRY(set_ctl_simple(0, dtau, theta, 0.5));
    const WorkList t0 = strips[0].view();
    switch (mode) {
    case M1_OP_APPLY:
        M1_TRY(pack_planar(q.u[0], n, state));
        launch_apply<R>(d, t0, ctl, APPLY_A, 0, nullptr, 0, stream);
        M1_CK(cudaGetLastError());
        return unpack_planar(q.r, n, out);
    case M1_OP_RESIDUAL: {
        M1_TRY(pack_planar(q.u[0], n, state));
        M1_TRY(pack_planar(q.f, n, rhs));
        launch_apply<R>(d, t0, ctl, APPLY_RESID, 0, part, 1, stream);
        M1_CK(cudaGetLastError());
        M1_TRY(unpack_planar(q.r, n, out));
        if (norm) {
            std::vector<double> p(q.strips);
            M1_CK(cudaMemcpy(p.data(), part, sizeof(double) * p.size(), cudaMemcpyDeviceToHost));
            double s = 0.0;
            for (double x : p) s += x;
            *norm = std::sqrt(s);
        }
        return M1_OK;
    }
    case M1_OP_RESIDUAL_DW:
        if constexpr (std::is_same<R, double>::value) {
            M1_TRY(pack_planar(q.u[0], n, state));
            M1_TRY(pack_planar(q.f, n, rhs));
            DW4* scratch = nullptr;
            M1_TRY(calloc_common((void**)&scratch, sizeof(DW4) * n));
            launch_residual_dw(d, q.u[0], scratch, n, t0, part, stream);
            M1_CK(cudaGetLastError());
            M1_TRY(unpack_planar(q.r, n, out));
            if (norm) {
                std::vector<double> p(q.strips);
                M1_CK(cudaMemcpy(p.data(), part, sizeof(double) * p.size(), cudaMemcpyDeviceToHost));
                double sum = 0.0;
                for (double x : p) sum += x;
                *norm = std::sqrt(sum);
            }
            return M1_OK;
        } else {
            return M1_ERR_INVALID_ARG;
        }
    case M1_OP_FAS_RHS:
        M1_TRY(pack_planar(q.v, n, state));
        M1_TRY(pack_planar(q.r, n, rhs));
        launch_apply<R>(d, t0, ctl, APPLY_FAS, -1, nullptr, 0, stream);
        M1_CK(cudaGetLastError());
        return unpack_planar(q.f, n, out);
    case M1_OP_JACOBI:
    case M1_OP_PSEUDO:
        M1_TRY(pack_planar(q.u[0], n, state));
        M1_TRY(pack_planar(q.f, n, rhs));
        launch_sweep<R>(d, strips[0].view(), ctl, mode == M1_OP_PSEUDO, 0, 1, stream);
        M1_CK(cudaGetLastError());
        M1_TRY(unpack_planar(q.u[1], n, out));
        if (norm) {
            // cells whose local E-T solve did not converge to a finite positive T
            Ctl c;
            M1_CK(cudaMemcpy(&c, ctl, sizeof(Ctl), cudaMemcpyDeviceToHost));
            *norm = (double)c.newton_fail;
        }
        return M1_OK;
    default:
        return M1_ERR_INVALID_ARG;
    }
}

template <typename R>
m1_status Engine<R>::op_restrict(const double* state, const double* resid, double* cs, double* cr)
{
    M1_TRY(set_ctl_simple(0, 0, 0.5, 0.5));
    M1_TRY(pack_planar(h[0].u[0], h[0].n, state));
    M1_TRY(pack_planar(h[0].r, h[0].n, resid));
    launch_restrict<R>(d, d + cap, chunks[1].view(), ctl, 0, stream);
    M1_CK(cudaGetLastError());
    M1_TRY(unpack_planar(h[cap].v, h[cap].n, cs));
    return unpack_planar(h[cap].r, h[cap].n, cr);
}

template <typename R>
m1_status Engine<R>::op_prolong(const double* uc, const double* vc, const double* uf, double theta,
                                double* out, int* damped)
{
    M1_TRY(set_ctl_simple(0, 0, 0.5, theta));
    M1_TRY(pack_planar(h[cap].u[0], h[cap].n, uc));
    M1_TRY(pack_planar(h[cap].v, h[cap].n, vc));
    M1_TRY(pack_planar(h[0].u[0], h[0].n, uf));
    launch_prolong<R>(d + cap, d, chunks[1].view(), ctl, 0, 0, stream);
    M1_CK(cudaGetLastError());
    M1_TRY(unpack_planar(h[0].u[0], h[0].n, out));
    if (damped) {
        M1_CK(cudaMemcpy(ctl_h, ctl, sizeof(Ctl), cudaMemcpyDeviceToHost));
        *damped = (int)ctl_h[0].damped;
    }
    return M1_OK;
}


// ---------------------------------------------------------------------------
// Serving support: slots joining and leaving a running engine.

// Device bytes a slot of this engine takes for grid `g` (its levels' buffers).
template <typename R>
size_t Engine<R>::slot_bytes(const m1_grid_desc& g) const
{
    size_t b = 0;
    long long nx = g.nx, ny = g.dim == 2 ? g.ny : 1;
    const int states = delta ? 7 : 5;
    for (int l = 0; l < L; ++l) {
        const long long n = nx * ny;
        b += (size_t)n * (states * sizeof(Cell4<R>) + sizeof(Sig2<R>));
        b += sizeof(R) * 12 * (size_t)std::max(nx, ny) + 8 * 256;
        if (dw && l == 0) b += (size_t)n * (2 * sizeof(DW4) + sizeof(DW2));
        nx /= 2; if (g.dim == 2) ny /= 2;
    }
    return b;
}

// Level-0 work lists of the given slots (for the start of their steps).
template <typename R>
m1_status Engine<R>::set_init_lists(const std::vector<int>& slots)
{
    init_strips.host.clear();
    init_chunks.host.clear();
    for (int i : slots) {
        for (int t = 0; t < h[i].strips; ++t) init_strips.host.push_back(make_int2(i, t));
        for (int c = 0; c < h[i].chunks; ++c) init_chunks.host.push_back(make_int2(i, c));
    }
    M1_TRY(upload_list(init_strips));
    M1_TRY(upload_list(init_chunks));
    if (!slots.empty())
        M1_CK(cudaMemcpyAsync(init_slots, slots.data(), sizeof(int) * slots.size(),
                              cudaMemcpyHostToDevice, stream));
    M1_CK(cudaStreamSynchronize(stream));
    return M1_OK;
}

// State, opacities (and their coarse restrictions) and inflow profiles of slot 0
// of `src` (a caller's grid, same precision and level count) into `slot`.
template <typename R>
m1_status Engine<R>::copy_slot_in(int slot, Engine<R>& src)
{
    M1_CK(cudaStreamSynchronize(src.stream));
    const Level<R>& q = h[slot];
    const Level<R>& p = src.h[0];
    if (q.n != p.n) return M1_ERR_INVALID_ARG;
    M1_CK(cudaMemcpyAsync(q.u[0], p.u[0], sizeof(Cell4<R>) * q.n, cudaMemcpyDeviceToDevice, stream));
    M1_CK(cudaMemcpyAsync(q.sig, p.sig, sizeof(Sig2<R>) * q.n, cudaMemcpyDeviceToDevice, stream));
    for (int l = 1; l < L; ++l) {
        init_chunks.host.clear();
        for (int c = 0; c < h[(size_t)l * cap + slot].chunks; ++c)
            init_chunks.host.push_back(make_int2(slot, c));
        M1_TRY(upload_list(init_chunks));
        launch_restrict_sig<R>(d + (size_t)(l - 1) * cap, d + (size_t)l * cap, init_chunks.view(), stream);
        M1_CK(cudaGetLastError());
    }
    for (int l = 0; l < L; ++l) {
        prof[(size_t)l * cap + slot] = src.prof[(size_t)l * src.cap];
        std::vector<R> tmp(prof[(size_t)l * cap + slot].begin(), prof[(size_t)l * cap + slot].end());
        M1_CK(cudaMemcpyAsync(h[(size_t)l * cap + slot].inflow, tmp.data(), sizeof(R) * tmp.size(),
                              cudaMemcpyHostToDevice, stream));
        M1_CK(cudaStreamSynchronize(stream));
    }
    rhs_valid[slot] = 0;
    return M1_OK;
}

template <typename R>
m1_status Engine<R>::copy_slot_out(int slot, Engine<R>& dst)
{
    const Level<R>& q = h[slot];
    M1_CK(cudaMemcpyAsync(dst.h[0].u[0], q.u[0], sizeof(Cell4<R>) * q.n, cudaMemcpyDeviceToDevice, stream));
    M1_CK(cudaStreamSynchronize(stream));
    dst.rhs_valid[0] = 0;
    return M1_OK;
}

// Bring a finished slot's result into buffer 0 (where its next step starts).
template <typename R>
m1_status Engine<R>::settle(int slot, int result_buf)
{
    if (result_buf == 1)
        M1_CK(cudaMemcpyAsync(h[slot].u[0], h[slot].u[1], sizeof(Cell4<R>) * h[slot].n,
                              cudaMemcpyDeviceToDevice, stream));
    return M1_OK;
}

template struct Engine<double>;
template struct Engine<float>;

m1_status PlainModel::sv_copy_in(int slot, Model& src)
{
    auto* p = dynamic_cast<PlainModel*>(&src);
    if (!p) return M1_ERR_INVALID_ARG;
    return e.copy_slot_in(slot, p->e);
}

m1_status PlainModel::sv_copy_out(int slot, Model& dst)
{
    auto* p = dynamic_cast<PlainModel*>(&dst);
    if (!p) return M1_ERR_INVALID_ARG;
    return e.copy_slot_out(slot, p->e);
}

// Start a step on the given slots while the other slots keep cycling.
m1_status PlainModel::sv_begin(const std::vector<int>& slots, const std::vector<double>& dts,
                               const std::vector<m1_solve_params>& ps)
{
    for (size_t k = 0; k < slots.size(); ++k) {
        const int i = slots[k];
        M1_TRY(validate_params(ps[k]));
        M1_TRY(e.set_dt(i, dts[k]));
        e.ctl_h[i] = make_ctl(ps[k], (double)e.h[i].diag);
        M1_CK(cudaMemcpyAsync(e.ctl + i, e.ctl_h + i, sizeof(Ctl), cudaMemcpyHostToDevice, e.stream));
    }
    M1_TRY(e.set_init_lists(slots));
    launch_make_rhs<double>(e.d, e.init_chunks.view(), e.ctl, 0, e.stream);
    launch_apply<double>(e.d, e.init_strips.view(), e.ctl, APPLY_RESID, 0, e.part, 0, e.stream);
    launch_norm_state<double>(e.d, e.init_strips.view(), e.ctl, e.partb, e.stream);
    launch_finalize<double>(e.ctl, e.d, (int)slots.size(), e.part, e.partb, FIN_INIT, 0, e.bctl,
                            e.stream, e.init_slots);
    M1_CK(cudaGetLastError());
    return M1_OK;
}

m1_status PlainModel::sv_cycles(const Params& p, int n)
{
    M1_TRY(e.build_graph(p));
    for (int k = 0; k < n; ++k) M1_CK(cudaGraphLaunch(e.graph, e.stream));
    return M1_OK;
}


m1_status MixedModel::sv_init(int cap, int L, cudaStream_t s)
{
    M1_TRY(hi.init(cap, 1, false, s, 0));
    M1_TRY(hi.enable_dw());
    M1_TRY(lo.init(cap, L, true, hi.stream, 0));
    lo.ctl = hi.ctl;
    return M1_OK;
}

size_t MixedModel::sv_bytes(const m1_grid_desc& d) const
{
    m1_grid_desc g = d;
    g.lmax = 1;
    return hi.slot_bytes(g) + lo.slot_bytes(d);
}

m1_status MixedModel::sv_add(const m1_grid_desc& d, int* slot)
{
    m1_grid_desc g = d;
    g.lmax = 1;
    g.precision = M1_FP64;
    int a, b;
    M1_TRY(hi.add_slot(g, &a));
    m1_status st = lo.add_slot(d, &b);
    if (st != M1_OK) { hi.remove_slot(a); return st; }
    if (a != b) return M1_ERR_CUDA;
    *slot = a;
    return M1_OK;
}

m1_status MixedModel::sv_remove(int slot)
{
    M1_TRY(hi.remove_slot(slot));
    return lo.remove_slot(slot);   // clears the shared control block of the slot again
}

m1_status MixedModel::sv_rebuild()
{
    M1_TRY(hi.rebuild());
    return lo.rebuild();
}

m1_status MixedModel::sv_copy_in(int slot, Model& src)
{
    auto* p = dynamic_cast<MixedModel*>(&src);
    if (!p) return M1_ERR_INVALID_ARG;
    M1_TRY(hi.copy_slot_in(slot, p->hi));
    return lo.copy_slot_in(slot, p->lo);
}

m1_status MixedModel::sv_copy_out(int slot, Model& dst)
{
    auto* p = dynamic_cast<MixedModel*>(&dst);
    if (!p) return M1_ERR_INVALID_ARG;
    return hi.copy_slot_out(slot, p->hi);
}

m1_status MixedModel::sv_begin(const std::vector<int>& slots, const std::vector<double>& dts,
                               const std::vector<m1_solve_params>& ps)
{
    for (size_t k = 0; k < slots.size(); ++k) {
        const int i = slots[k];
        M1_TRY(validate_params(ps[k]));
        M1_TRY(hi.set_dt(i, dts[k]));
        M1_TRY(lo.set_dt(i, dts[k]));
        hi.ctl_h[i] = make_ctl(ps[k], (double)hi.h[i].diag);
        M1_CK(cudaMemcpyAsync(hi.ctl + i, hi.ctl_h + i, sizeof(Ctl), cudaMemcpyHostToDevice, hi.stream));
    }
    M1_TRY(hi.set_init_lists(slots));
    launch_make_rhs<double>(hi.d, hi.init_chunks.view(), hi.ctl, 0, hi.stream);
    launch_dw_split(hi.d, hi.dwd, hi.init_chunks.view(), hi.stream);
    launch_norm_state<double>(hi.d, hi.init_strips.view(), hi.ctl, hi.partb, hi.stream);
    // the served cycles share the structural parameters (fixed at server creation)
    launch_defect(hi.d, lo.d, hi.init_strips.view(), hi.ctl, hi.part, hi.stream,
                  !ps.empty() && ps[0].nu0 > 0);
    launch_finalize<double>(hi.ctl, hi.d, (int)slots.size(), hi.part, hi.partb, FIN_INIT, 0, hi.bctl,
                            hi.stream, hi.init_slots);
    M1_CK(cudaGetLastError());
    return M1_OK;
}

m1_status MixedModel::sv_cycles(const Params& p, int n)
{
    M1_TRY(build_graph(p));
    for (int k = 0; k < n; ++k) M1_CK(cudaGraphLaunch(graph, hi.stream));
    return M1_OK;
}


// ---------------------------------------------------------------------------
m1_status PlainModel::create(const std::vector<m1_grid_desc>& descs, cudaStream_t s)
{
    const int L = descs[0].lmax;
    M1_TRY(e.init((int)descs.size(), L, false, s, descs.size() == 1 ? 20001 : 0));
    for (const auto& d : descs) {
        int slot;
        M1_TRY(e.add_slot(d, &slot));
    }
    return e.rebuild();
}

m1_status MixedModel::create(const std::vector<m1_grid_desc>& descs, cudaStream_t s)
{
    const int L = descs[0].lmax;
    const int n = (int)descs.size();
    M1_TRY(hi.init(n, 1, false, s, n == 1 ? 20001 : 0));
    M1_TRY(hi.enable_dw());
    M1_TRY(lo.init(n, L, true, hi.stream, 0));
    for (const auto& d : descs) {
        m1_grid_desc g = d;
        g.lmax = 1;
        g.precision = M1_FP64;
        int a, b;
        M1_TRY(hi.add_slot(g, &a));
        M1_TRY(lo.add_slot(d, &b));
    }
    M1_TRY(hi.rebuild());
    M1_TRY(lo.rebuild());
    lo.ctl = hi.ctl;   // the FP32 cycle reads the FP64 level's control blocks
    return M1_OK;
}

m1_status MixedModel::set_state(int i, const double* E, const double* Fx, const double* Fy,
                                const double* T, const double* sa, const double* ss, int dev)
{
    M1_TRY(hi.set_state(i, E, Fx, Fy, T, sa, ss, dev));
    return lo.set_state(i, E, Fx, Fy, T, sa, ss, dev);
}

m1_status MixedModel::set_inflow(int i, int side, const double* E, const double* Fx,
                                 const double* Fy)
{
    M1_TRY(hi.set_inflow(i, side, E, Fx, Fy));
    return lo.set_inflow(i, side, E, Fx, Fy);
}

// FP32 V-cycle in correction form, FP64 accumulation of its correction, FP64
// defect of the new iterate with the FP32 source of the next cycle, stop test.
void MixedModel::record_cycle(const Params& p, cudaStream_t s)
{
    // the defect that ends a cycle (or starts the step) also forms the next
    // cycle's first fine sweep (from e = 0 the sweep needs no neighbour)
    const bool fused = p.nu0 > 0;
    int cur0 = 0;
    lo.record_cycle(p, cur0, s, false, fused);
    launch_accumulate(hi.d, lo.d, hi.chunks[0].view(), hi.ctl, cur0, s, hi.dwd);
    // each instance's defect comes from one of the two: FP64, or double-word FP32
    // where its tolerance lies far above the double-word noise floor (FIN_INIT)
    launch_defect(hi.d, lo.d, hi.strips[0].view(), hi.ctl, hi.part, s, fused);
    launch_defect_dw(hi.d, lo.d, hi.dwd, hi.strips[0].view(), hi.ctl, hi.part, s, fused);
    launch_finalize<double>(hi.ctl, hi.d, hi.cap, hi.part, nullptr, FIN_CYCLE, 0, hi.bctl, s);
}

m1_status MixedModel::build_graph(const Params& p)
{
    if (graph && gparams == p && !hi.graph_dirty && !lo.graph_dirty) return M1_OK;
    if (graph) { cudaGraphExecDestroy(graph); graph = nullptr; }
    cudaGraph_t g = nullptr;
    M1_CK(cudaStreamBeginCapture(lo.cap_stream, cudaStreamCaptureModeThreadLocal));
    record_cycle(p, lo.cap_stream);
    cudaError_t e = cudaStreamEndCapture(lo.cap_stream, &g);
    if (e != cudaSuccess) { set_err(e, "cudaStreamEndCapture"); return M1_ERR_CUDA; }
    e = cudaGraphInstantiate(&graph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) { set_err(e, "cudaGraphInstantiate"); graph = nullptr; return M1_ERR_CUDA; }
    gparams = p;
    hi.graph_dirty = lo.graph_dirty = false;
    return M1_OK;
}

m1_status MixedModel::step(const double* dts, const m1_solve_params& sp, m1_step_stats* st)
{
    M1_TRY(validate_params(sp));
    for (int i = 0; i < hi.cap; ++i)
        if (hi.used[i] && !(dts[i] > 0)) return M1_ERR_INVALID_ARG;
    for (int i = 0; i < lo.cap; ++i)
        if (lo.used[i]) M1_TRY(lo.set_dt(i, dts[i]));
    Params p{ sp.nu0, sp.nu_l, sp.m_pseudo, sp.m_coarse, sp.cycle };
    M1_TRY(build_graph(p));
    M1_TRY(hi.begin_step(dts, sp));
    cudaStream_t s = hi.stream;
    M1_CK(cudaEventRecord(hi.ev0, s));
    const WorkList t0 = hi.strips[0].view(), c0 = hi.chunks[0].view();
    launch_make_rhs<double>(hi.d, c0, hi.ctl, 0, s);
    launch_dw_split(hi.d, hi.dwd, c0, s);
    launch_norm_state<double>(hi.d, t0, hi.ctl, hi.partb, s);
    launch_defect(hi.d, lo.d, t0, hi.ctl, hi.part, s, p.nu0 > 0);
    launch_finalize<double>(hi.ctl, hi.d, hi.cap, hi.part, hi.partb, FIN_INIT, 0, hi.bctl, s);
    M1_CK(cudaGetLastError());
    for (int i = 0; i < hi.cap; ++i)
        if (hi.used[i]) { hi.dt_rhs[i] = dts[i]; hi.rhs_valid[i] = 1; }
    long long launched = 0;
    M1_TRY(run_until_done(graph, 1, sp.max_cycles, s, hi.bctl, hi.done_h, hi.poll, &launched));
    M1_CK(cudaMemcpyAsync(hi.ctl_h, hi.ctl, sizeof(Ctl) * hi.cap, cudaMemcpyDeviceToHost, s));
    M1_CK(cudaEventRecord(hi.ev1, s));
    M1_CK(cudaEventSynchronize(hi.ev1));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, hi.ev0, hi.ev1);
    bool all_ok = true;
    int k = 0;
    for (int i = 0; i < hi.cap; ++i) {
        if (!hi.used[i]) continue;
        const Ctl& c = hi.ctl_h[i];
        hi.last_cycles[i] = c.kappa;
        all_ok = all_ok && c.status == CTL_OK;
        if (st) {
            m1_step_stats& o = st[k];
            o.cycles = c.kappa;
            o.res0 = c.res0;
            o.res = c.kappa > 0 ? c.res : c.res0;
            o.dtau_final = c.dtau;
            o.sweeps = (long long)c.kappa * (lo.L == 1 ? p.nu0 : 2 * p.nu0);
            o.ms = ms;
            o.status = c.status;
            o.newton_fail = c.newton_fail;
            o.damped = c.damped;
            // accumulate, defects, finalize; the first fine sweep is the defects'
            o.launches = 4 + launched * (lo.kernels_per_cycle(p) + 4 - (p.nu0 > 0 ? 1 : 0));
        }
        ++k;
    }
    return all_ok ? M1_OK : M1_ERR_NOT_CONVERGED;
}

// Algorithm 1 in mixed precision: b = (E, F, C_v T) of the current state v, the
// FP64 defect r = b - A(v), `sweeps` FP32 Jacobi sweeps of the correction
// equation A32(w + e) - A32(w) = r from e = 0 (w = fl32(v)), then v += e in FP64.
m1_status MixedModel::jacobi(int i, double dt, int sweeps)
{
    if (hi.cap != 1 || i != 0 || !hi.used[0] || !(dt > 0) || sweeps < 0) return M1_ERR_INVALID_ARG;
    M1_TRY(hi.set_dt(0, dt));
    M1_TRY(lo.set_dt(0, dt));
    M1_TRY(hi.set_ctl_simple(0, 0.0, 0.5, 0.5));
    cudaStream_t s = hi.stream;
    launch_make_rhs<double>(hi.d, hi.chunks[0].view(), hi.ctl, 0, s);
    launch_defect(hi.d, lo.d, hi.strips[0].view(), hi.ctl, hi.part, s, false);
    int cur = 0;
    lo.sweeps_fine(cur, sweeps, s);
    launch_accumulate(hi.d, lo.d, hi.chunks[0].view(), hi.ctl, cur, s);
    M1_CK(cudaGetLastError());
    hi.dt_rhs[0] = dt;
    hi.rhs_valid[0] = 1;
    return M1_OK;
}

MixedModel::~MixedModel()
{
    if (graph) cudaGraphExecDestroy(graph);
}

m1_status make_model(const std::vector<m1_grid_desc>& descs, cudaStream_t s,
                     std::unique_ptr<Model>& out)
{
    if (descs.empty()) return M1_ERR_INVALID_ARG;
    for (const auto& d : descs) {
        M1_TRY(validate_desc(&d));
        if (d.lmax != descs[0].lmax || d.precision != descs[0].precision) return M1_ERR_INVALID_ARG;
    }
    if (descs[0].precision == M1_MIXED) {
        std::unique_ptr<MixedModel> m(new MixedModel());
        m1_status st = m->create(descs, s);
        out = std::move(m);
        return st;
    }
    std::unique_ptr<PlainModel> m(new PlainModel());
    m1_status st = m->create(descs, s);
    out = std::move(m);
    return st;
}

template <typename R>
m1_status make_op_engine(const m1_grid_desc* desc, int lmax, const double* inflow,
                         std::unique_ptr<Engine<R>>& out)
{
    m1_grid_desc g = *desc;
    g.lmax = lmax;
    M1_TRY(validate_desc(&g));
    out.reset(new Engine<R>());
    M1_TRY(out->init(1, lmax, false, nullptr, 0));
    int slot;
    M1_TRY(out->add_slot(g, &slot));
    M1_TRY(out->rebuild());
    if (inflow) {
        const int Lp = std::max(g.nx, g.dim == 2 ? g.ny : 1);
        for (int w = 0; w < 4; ++w)
            if (g.bc[w] == M1_BC_INFLOW)
                M1_TRY(out->set_inflow(0, w, inflow + (size_t)(w * 3) * Lp,
                                       inflow + (size_t)(w * 3 + 1) * Lp,
                                       inflow + (size_t)(w * 3 + 2) * Lp));
    }
    return M1_OK;
}

}  // namespace m1

using m1::Model;

extern "C" {

const char* m1_last_error(void) { return m1::g_err; }

m1_status m1_default_params(m1_solve_params* p)
{
    if (!p) return M1_ERR_INVALID_ARG;
    p->nu0 = 3; p->nu_l = 1; p->m_pseudo = 3; p->m_coarse = 3;
    p->dtau0 = 1e-3; p->grow = 1.1; p->shrink = 0.5; p->eps_i = 1e-2; p->eps_d = 1e-4;
    p->tol = 1e-8; p->dtau_min = 1e-12; p->dtau_max = 1e6; p->theta_ex = 0.5; p->theta_c = 0.5;
    p->max_cycles = 20000;
    p->dtau_rule = M1_DTAU_ABS;
    p->cycle = M1_CYCLE_V;
    return M1_OK;
}

m1_status m1_create_grid(const m1_grid_desc* desc, void* cuda_stream, m1_grid_t* out)
{
    if (!out || !desc) return M1_ERR_INVALID_ARG;
    *out = nullptr;
    M1_TRY(m1::validate_desc(desc));
    std::unique_ptr<Model> model;
    m1_status s = m1::make_model({ *desc }, static_cast<cudaStream_t>(cuda_stream), model);
    if (s != M1_OK) return s;
    m1_grid* g = new m1_grid;
    g->model = std::move(model);
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
    return g->model->set_state(0, E, Fx, Fy, T, sig_a, sig_s, on_device);
}

m1_status m1_set_inflow(m1_grid_t g, int side, const double* E, const double* Fx, const double* Fy)
{
    if (!g) return M1_ERR_INVALID_ARG;
    return g->model->set_inflow(0, side, E, Fx, Fy);
}

m1_status m1_get_state(m1_grid_t g, double* E, double* Fx, double* Fy, double* T, int on_device)
{
    if (!g) return M1_ERR_INVALID_ARG;
    return g->model->get_state(0, E, Fx, Fy, T, on_device);
}

m1_status m1_implicit_step(m1_grid_t g, double dt, const m1_solve_params* params,
                           m1_step_stats* stats)
{
    if (!g) return M1_ERR_INVALID_ARG;
    m1_solve_params p;
    if (params) p = *params; else m1_default_params(&p);
    return g->model->step(&dt, p, stats);
}

m1_status m1_jacobi(m1_grid_t g, double dt, int sweeps)
{
    if (!g) return M1_ERR_INVALID_ARG;
    return g->model->jacobi(0, dt, sweeps);
}

m1_status m1_residual_norm(m1_grid_t g, double dt, double* out)
{
    if (!g) return M1_ERR_INVALID_ARG;
    return g->model->residual_norm(0, dt, out);
}

m1_status m1_step_history(m1_grid_t g, double* hist, double* dtau, int len)
{
    if (!g) return M1_ERR_INVALID_ARG;
    return g->model->history(0, hist, dtau, len);
}

m1_status m1_create_batch(const m1_grid_desc* descs, int count, void* cuda_stream, m1_batch_t* out)
{
    if (!out || !descs || count < 1) return M1_ERR_INVALID_ARG;
    *out = nullptr;
    std::vector<m1_grid_desc> v(descs, descs + count);
    std::unique_ptr<Model> model;
    m1_status s = m1::make_model(v, static_cast<cudaStream_t>(cuda_stream), model);
    if (s != M1_OK) return s;
    m1_batch* b = new m1_batch;
    b->model = std::move(model);
    b->count = count;
    *out = b;
    return M1_OK;
}

m1_status m1_destroy_batch(m1_batch_t b)
{
    if (!b) return M1_ERR_INVALID_ARG;
    delete b;
    return M1_OK;
}

m1_status m1_batch_set_state(m1_batch_t b, int index, const double* E, const double* Fx,
                             const double* Fy, const double* T, const double* sig_a,
                             const double* sig_s, int on_device)
{
    if (!b || index < 0 || index >= b->count) return M1_ERR_INVALID_ARG;
    return b->model->set_state(index, E, Fx, Fy, T, sig_a, sig_s, on_device);
}

m1_status m1_batch_set_inflow(m1_batch_t b, int index, int side, const double* E, const double* Fx,
                              const double* Fy)
{
    if (!b || index < 0 || index >= b->count) return M1_ERR_INVALID_ARG;
    return b->model->set_inflow(index, side, E, Fx, Fy);
}

m1_status m1_batch_get_state(m1_batch_t b, int index, double* E, double* Fx, double* Fy, double* T,
                             int on_device)
{
    if (!b || index < 0 || index >= b->count) return M1_ERR_INVALID_ARG;
    return b->model->get_state(index, E, Fx, Fy, T, on_device);
}

m1_status m1_batch_implicit_step(m1_batch_t b, const double* dt, const m1_solve_params* params,
                                 m1_step_stats* stats)
{
    if (!b || !dt) return M1_ERR_INVALID_ARG;
    m1_solve_params p;
    if (params) p = *params; else m1_default_params(&p);
    return b->model->step(dt, p, stats);
}

m1_status m1_op_level(const m1_grid_desc* desc, const double* inflow, double dt, const double* sig,
                      const double* state, const double* rhs, int mode, double dtau, double theta,
                      double* out, double* norm)
{
    if (!desc || !sig || !state || !out || !(dt > 0)) return M1_ERR_INVALID_ARG;
    if (mode != M1_OP_APPLY && !rhs) return M1_ERR_INVALID_ARG;
    if (desc->precision == M1_FP64) {
        std::unique_ptr<m1::Engine<double>> e;
        M1_TRY(m1::make_op_engine(desc, 1, inflow, e));
        return e->op_level(dt, sig, state, rhs, mode, dtau, theta, out, norm);
    }
    std::unique_ptr<m1::Engine<float>> e;
    M1_TRY(m1::make_op_engine(desc, 1, inflow, e));
    return e->op_level(dt, sig, state, rhs, mode, dtau, theta, out, norm);
}

m1_status m1_op_restrict(const m1_grid_desc* fine, const double* inflow, const double* state,
                         const double* resid, double* coarse_state, double* coarse_resid)
{
    if (!fine || !state || !resid || !coarse_state || !coarse_resid) return M1_ERR_INVALID_ARG;
    if (fine->precision == M1_FP64) {
        std::unique_ptr<m1::Engine<double>> e;
        M1_TRY(m1::make_op_engine(fine, 2, inflow, e));
        return e->op_restrict(state, resid, coarse_state, coarse_resid);
    }
    std::unique_ptr<m1::Engine<float>> e;
    M1_TRY(m1::make_op_engine(fine, 2, inflow, e));
    return e->op_restrict(state, resid, coarse_state, coarse_resid);
}

m1_status m1_op_prolong_correct(const m1_grid_desc* fine, const double* uc, const double* vc,
                                const double* uf, double theta, double* out, int* damped)
{
    if (!fine || !uc || !vc || !uf || !out) return M1_ERR_INVALID_ARG;
    if (fine->precision == M1_FP64) {
        std::unique_ptr<m1::Engine<double>> e;
        M1_TRY(m1::make_op_engine(fine, 2, nullptr, e));
        return e->op_prolong(uc, vc, uf, theta, out, damped);
    }
    std::unique_ptr<m1::Engine<float>> e;
    M1_TRY(m1::make_op_engine(fine, 2, nullptr, e));
    return e->op_prolong(uc, vc, uf, theta, out, damped);
}

m1_status m1_dw_split(const double* x, long long n, float* hi, float* lo)
{
    if (n < 0 || (n > 0 && (!x || !hi || !lo))) return M1_ERR_INVALID_ARG;
    for (long long i = 0; i < n; ++i) {
        const m1::DW d = m1::dw_split(x[i]);
        hi[i] = d.hi;
        lo[i] = d.lo;
    }
    return M1_OK;
}

m1_status m1_f32_widen(const float* x, long long n, double* y)
{
    if (n < 0 || (n > 0 && (!x || !y))) return M1_ERR_INVALID_ARG;
    for (long long i = 0; i < n; ++i) y[i] = m1::widen(x[i]);
    return M1_OK;
}

}  // extern "C"
