// The implicit M1 step in three dimensions: Algorithm 4 (Appendix A) on a 3D
// level hierarchy, with the 2D path's readings on three axes.
//
// Levels 0 .. L_max - 1, each axis halved per level (Section 4.2; L_max counts
// the grids, Table 4).  Per level: the restricted iterate v, the ping-pong
// iterate u[0], u[1], the right-hand side f (b at level 0, the FAS right-hand
// side f = A(v) + r above, Eq. (24)), the residual r, the closure array P and
// the opacities.  A cycle (V, W or F, the recursion of the 2D path) is emitted
// once per (dt, parameters) into a CUDA graph and relaunched until the control
// block on the device says done; the stop test and the dtau_im control
// (Algorithm 4) never leave the device, and every kernel of a cycle queued
// past convergence returns at once, so the cycle count is the oracle's.
//
// Fine level: nu0 Jacobi sweeps (closure pass + operator pass each), the
// residual and its restriction, the coarse-grid corrections, the damped
// prolongation (Eq. (34)), nu0 sweeps, then v <- u.  The norm of b - A(v) that
// ends a cycle is formed by the first sweep of the next one, which reads v and
// evaluates b + N(v) anyway (one closure and one operator pass fewer per
// cycle); if that cycle converged the rest of the launch returns at once and v
// is the result.
// Coarse level l: on a fresh visit f_l = A(v_l) + r_l and u_l = v_l; m
// pseudo-time steps (Eq. (30), Algorithm 3; the coarsest level m_coarse and
// nothing else), the residual, restriction, corrections, prolongation and m
// pseudo-time steps.
#include <m1.h>

#include <algorithm>
#include <cstring>
#include <memory>
#include <vector>

#include "m1_3d.cuh"
#include "m1_engine.h"

namespace m1 {
namespace {

struct Lev3 {
    G3 g{};
    double h[3] = { 0, 0, 0 };
    size_t n = 0;
    EF *v = nullptr, *u[2] = { nullptr, nullptr }, *f = nullptr, *r = nullptr;
    double *vT = nullptr, *uT[2] = { nullptr, nullptr }, *fT = nullptr, *rT = nullptr;
    P6* P = nullptr;
    Sig2<double>* sig = nullptr;
    double* prof = nullptr;                 // [6][4][fstride] inflow profiles (inflow walls only)
};

size_t face_max3(const int n[3])
{
    const size_t a = (size_t)n[1] * n[2], b = (size_t)n[0] * n[2], c = (size_t)n[0] * n[1];
    return std::max(a, std::max(b, c));
}

struct Grid3 {
    m1_grid3_desc desc{};
    int L = 0;
    cudaStream_t stream = nullptr, cap_stream = nullptr;
    bool own_stream = false;
    std::vector<Lev3> lv;
    std::vector<void*> mem;
    double* stage = nullptr;                // 5 n0 doubles: host planes in and out
    double *part = nullptr, *partb = nullptr;
    Ctl* ctl = nullptr;
    Ctl* ctl_h = nullptr;                   // pinned mirror
    BatchCtl* bctl = nullptr;
    int* done_h = nullptr;                  // pinned, two slots
    int* bad = nullptr;
    cudaEvent_t poll[2] = { nullptr, nullptr }, ev0 = nullptr, ev1 = nullptr;
    double *hist = nullptr, *dtau_hist = nullptr;
    int hist_len = 0;
    cudaGraphExec_t graph = nullptr;
    double graph_dt = 0.0;
    Params gparams{};
    long long kernels_per_cycle = 0;
    bool state_set = false, inflow_set = false, has_inflow = false;
    int last_cycles = 0;
    std::vector<int> cur;                   // per level: the u buffer holding the iterate

    ~Grid3()
    {
        if (stream) cudaStreamSynchronize(stream);
        if (graph) cudaGraphExecDestroy(graph);
        for (void* p : mem) cudaFree(p);
        if (ctl_h) cudaFreeHost(ctl_h);
        if (done_h) cudaFreeHost(done_h);
        for (auto e : poll)
            if (e) cudaEventDestroy(e);
        if (ev0) cudaEventDestroy(ev0);
        if (ev1) cudaEventDestroy(ev1);
        if (cap_stream) cudaStreamDestroy(cap_stream);
        if (own_stream && stream) cudaStreamDestroy(stream);
    }

    template <typename T>
    m1_status alloc(T** p, size_t count)
    {
        void* q = nullptr;
        M1_CK(cudaMalloc(&q, sizeof(T) * std::max<size_t>(count, 1)));
        mem.push_back(q);
        *p = static_cast<T*>(q);
        return M1_OK;
    }

    m1_status init(const m1_grid3_desc& d, int lmax, cudaStream_t s);
    void set_dt(double dt);
    void emit_sweeps_fine(int nsweeps, cudaStream_t s);
    void emit_pseudo(int l, int steps, cudaStream_t s);
    void emit_visit(int l, bool fresh, int shape, const Params& p, cudaStream_t s);
    void emit_corrections(int l, int shape, const Params& p, cudaStream_t s);
    void emit_cycle(const Params& p, cudaStream_t s);
    m1_status build_graph(const Params& p, double dt);
    m1_status set_state(const double* state, const double* sig, int on_device);
    m1_status set_inflow(const double* faces);
    m1_status get_state(double* state, int on_device);
    m1_status step(double dt, const m1_solve_params& sp, m1_step_stats* st);
    m1_status history(double* hs, double* dt, int len);
};

m1_status Grid3::init(const m1_grid3_desc& d, int lmax, cudaStream_t s)
{
    desc = d;
    L = lmax;
    if (s) {
        stream = s;
    } else {
        M1_CK(cudaStreamCreateWithFlags(&stream, cudaStreamNonBlocking));
        own_stream = true;
    }
    M1_CK(cudaStreamCreateWithFlags(&cap_stream, cudaStreamNonBlocking));
    lv.resize(L);
    cur.assign(L, 0);
    for (int w = 0; w < 6; ++w) has_inflow = has_inflow || d.bc[w] == M1_BC_INFLOW;
    const int n0[3] = { d.nx, d.ny, d.nz };
    const double len[3] = { d.lx, d.ly, d.lz };
    for (int l = 0; l < L; ++l) {
        Lev3& q = lv[l];
        for (int a = 0; a < 3; ++a) {
            q.g.n[a] = n0[a] >> l;
            q.h[a] = len[a] / q.g.n[a];
        }
        for (int w = 0; w < 6; ++w) q.g.bc[w] = (int)d.bc[w];
        q.g.c = d.c; q.g.a_r = d.a_r; q.g.c_v = d.c_v;
        q.g.ic2 = 1.0 / (d.c * d.c);
        q.g.vol = q.h[0] * q.h[1] * q.h[2];
        q.n = (size_t)q.g.n[0] * q.g.n[1] * q.g.n[2];
        M1_TRY(alloc(&q.v, q.n)); M1_TRY(alloc(&q.vT, q.n));
        for (int b = 0; b < 2; ++b) { M1_TRY(alloc(&q.u[b], q.n)); M1_TRY(alloc(&q.uT[b], q.n)); }
        M1_TRY(alloc(&q.f, q.n)); M1_TRY(alloc(&q.fT, q.n));
        M1_TRY(alloc(&q.r, q.n)); M1_TRY(alloc(&q.rT, q.n));
        M1_TRY(alloc(&q.P, q.n));
        M1_TRY(alloc(&q.sig, q.n));
        if (has_inflow) {
            q.g.fstride = (int)face_max3(q.g.n);
            M1_TRY(alloc(&q.prof, (size_t)6 * 4 * q.g.fstride));
            M1_CK(cudaMemsetAsync(q.prof, 0, sizeof(double) * 6 * 4 * q.g.fstride, stream));
            for (int w = 0; w < 6; ++w)
                q.g.in[w] = d.bc[w] == M1_BC_INFLOW ? q.prof + (size_t)w * 4 * q.g.fstride : nullptr;
        }
    }
    M1_TRY(alloc(&stage, 5 * lv[0].n));
    M1_TRY(alloc(&part, kMaxBlocks3));
    M1_TRY(alloc(&partb, kMaxBlocks3));
    M1_TRY(alloc(&ctl, 1));
    M1_TRY(alloc(&bctl, 1));
    M1_TRY(alloc(&bad, 1));
    hist_len = 20001;
    M1_TRY(alloc(&hist, hist_len));
    M1_TRY(alloc(&dtau_hist, hist_len));
    M1_CK(cudaHostAlloc(&ctl_h, sizeof(Ctl), cudaHostAllocDefault));
    M1_CK(cudaHostAlloc(&done_h, 2 * sizeof(int), cudaHostAllocDefault));
    for (auto& e : poll) M1_CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    M1_CK(cudaEventCreate(&ev0));
    M1_CK(cudaEventCreate(&ev1));
    return M1_OK;
}

// The constants of every level that depend on the time step.
void Grid3::set_dt(double dt)
{
    for (Lev3& q : lv) {
        q.g.cdt = q.g.c * dt;
        q.g.diag = 1.0;
        for (int a = 0; a < 3; ++a) {
            q.g.diag += q.g.c * dt / q.h[a];
            q.g.beta[a] = dt / (2.0 * q.h[a]);
        }
    }
}

// ---- the cycle, emitted into a graph --------------------------------------------
// nsweeps fine Jacobi sweeps; the first one of a cycle (reading v) also forms
// the norm of b - A(v), the stop test of the previous cycle (a deferred
// finalize follows it).
void Grid3::emit_sweeps_fine(int nsweeps, cudaStream_t s)
{
    Lev3& q = lv[0];
    for (int k = 0; k < nsweeps; ++k) {
        const bool first = cur[0] < 0;
        const EF* src = first ? q.v : q.u[cur[0]];
        const double* srcT = first ? q.vT : q.uT[cur[0]];
        const int dst = cur[0] == 0 ? 1 : 0;
        launch3_closure(q.g, src, q.P, q.n, ctl, s);
        launch3_op(first ? OP3K_JACOBI_NORM : OP3K_JACOBI, q.g, src, srcT, q.P, q.sig, q.f, q.fT,
                   q.u[dst], q.uT[dst], q.n, ctl, first ? part : nullptr, s);
        kernels_per_cycle += 2;
        if (first) {
            launch3_finalize(ctl, bctl, part, nullptr, blocks3(q.n), FIN3_DEFER, s);
            kernels_per_cycle += 1;
        }
        cur[0] = dst;
    }
}

void Grid3::emit_pseudo(int l, int steps, cudaStream_t s)
{
    Lev3& q = lv[l];
    for (int k = 0; k < steps; ++k) {
        const int a = cur[l], b = a ^ 1;
        launch3_closure(q.g, q.u[a], q.P, q.n, ctl, s);
        launch3_op(OP3K_PSEUDO, q.g, q.u[a], q.uT[a], q.P, q.sig, q.f, q.fT, q.u[b], q.uT[b], q.n,
                   ctl, nullptr, s);
        kernels_per_cycle += 2;
        cur[l] = b;
    }
}

void Grid3::emit_corrections(int l, int shape, const Params& p, cudaStream_t s)
{
    if (l + 1 == L - 1 || shape == M1_CYCLE_V) {
        emit_visit(l + 1, true, shape, p, s);
    } else if (shape == M1_CYCLE_W) {
        emit_visit(l + 1, true, M1_CYCLE_W, p, s);
        emit_visit(l + 1, false, M1_CYCLE_W, p, s);
    } else {
        emit_visit(l + 1, true, M1_CYCLE_F, p, s);
        emit_visit(l + 1, false, M1_CYCLE_V, p, s);
    }
}

void Grid3::emit_visit(int l, bool fresh, int shape, const Params& p, cudaStream_t s)
{
    Lev3& q = lv[l];
    if (fresh) {
        launch3_closure(q.g, q.v, q.P, q.n, ctl, s);
        launch3_op(OP3K_FAS, q.g, q.v, q.vT, q.P, q.sig, q.r, q.rT, q.f, q.fT, q.n, ctl, nullptr, s);
        launch3_copy(q.v, q.vT, q.u[0], q.uT[0], q.n, ctl, s);
        kernels_per_cycle += 3;
        cur[l] = 0;
    }
    if (l == L - 1) {
        emit_pseudo(l, p.mc, s);
        return;
    }
    emit_pseudo(l, p.m, s);
    Lev3& c = lv[l + 1];
    const int a = cur[l];
    launch3_closure(q.g, q.u[a], q.P, q.n, ctl, s);
    launch3_op(OP3K_RESID, q.g, q.u[a], q.uT[a], q.P, q.sig, q.f, q.fT, q.r, q.rT, q.n, ctl,
               nullptr, s);
    launch3_restrict(q.g, c.g, q.u[a], q.uT[a], q.r, q.rT, c.v, c.vT, c.r, c.rT, ctl, s);
    kernels_per_cycle += 3;
    emit_corrections(l, shape, p, s);
    launch3_prolong(c.g, q.g, c.u[cur[l + 1]], c.uT[cur[l + 1]], c.v, c.vT, q.u[a], q.uT[a], ctl, s);
    kernels_per_cycle += 1;
    emit_pseudo(l, p.m, s);
}

void Grid3::emit_cycle(const Params& p, cudaStream_t s)
{
    Lev3& q = lv[0];
    cur[0] = -1;                                    // the first sweep reads v
    emit_sweeps_fine(p.nu0, s);
    if (L > 1) {
        Lev3& c = lv[1];
        const int a = cur[0];
        launch3_closure(q.g, q.u[a], q.P, q.n, ctl, s);
        launch3_op(OP3K_RESID, q.g, q.u[a], q.uT[a], q.P, q.sig, q.f, q.fT, q.r, q.rT, q.n, ctl,
                   nullptr, s);
        launch3_restrict(q.g, c.g, q.u[a], q.uT[a], q.r, q.rT, c.v, c.vT, c.r, c.rT, ctl, s);
        kernels_per_cycle += 3;
        emit_corrections(0, p.cycle, p, s);
        launch3_prolong(c.g, q.g, c.u[cur[1]], c.uT[cur[1]], c.v, c.vT, q.u[a], q.uT[a], ctl, s);
        kernels_per_cycle += 1;
        emit_sweeps_fine(p.nu0, s);
    }
    // end of the cycle: v <- u; its residual norm, stop test and dtau_im update
    // come with the next cycle's first sweep (a step takes one graph launch
    // more than it has cycles)
    launch3_copy(q.u[cur[0]], q.uT[cur[0]], q.v, q.vT, q.n, ctl, s);
    kernels_per_cycle += 1;
}

m1_status Grid3::build_graph(const Params& p, double dt)
{
    if (graph && gparams == p && graph_dt == dt) return M1_OK;
    if (graph) { cudaGraphExecDestroy(graph); graph = nullptr; }
    cudaGraph_t g = nullptr;
    kernels_per_cycle = 0;
    M1_CK(cudaStreamBeginCapture(cap_stream, cudaStreamCaptureModeThreadLocal));
    emit_cycle(p, cap_stream);
    cudaError_t e = cudaStreamEndCapture(cap_stream, &g);
    if (e != cudaSuccess) { set_err(e, "cudaStreamEndCapture"); return M1_ERR_CUDA; }
    e = cudaGraphInstantiate(&graph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) { set_err(e, "cudaGraphInstantiate"); graph = nullptr; return M1_ERR_CUDA; }
    gparams = p;
    graph_dt = dt;
    return M1_OK;
}

// ---- state in and out ------------------------------------------------------------
m1_status Grid3::set_state(const double* state, const double* sig, int on_device)
{
    if (!state || !sig) return M1_ERR_INVALID_ARG;
    Lev3& q = lv[0];
    const double* sp = state;
    if (!on_device) {
        M1_CK(cudaMemcpyAsync(stage, state, sizeof(double) * 5 * q.n, cudaMemcpyHostToDevice, stream));
        sp = stage;
    }
    launch3_pack(sp, q.v, q.vT, q.n, stream);
    const double* gp = sig;
    if (!on_device) {
        M1_CK(cudaMemcpyAsync(stage, sig, sizeof(double) * 2 * q.n, cudaMemcpyHostToDevice, stream));
        gp = stage;
    }
    launch3_pack_sig(gp, q.sig, q.n, stream);
    for (int l = 1; l < L; ++l) launch3_restrict_sig(lv[l - 1].g, lv[l].g, lv[l - 1].sig, lv[l].sig, stream);
    M1_CK(cudaMemsetAsync(bad, 0, sizeof(int), stream));
    launch3_check(q.g, q.v, q.vT, q.sig, q.n, bad, stream);
    M1_CK(cudaGetLastError());
    int b = 0;
    M1_CK(cudaMemcpyAsync(&b, bad, sizeof(int), cudaMemcpyDeviceToHost, stream));
    M1_CK(cudaStreamSynchronize(stream));
    state_set = b == 0;
    return b ? M1_ERR_NONADMISSIBLE_INPUT : M1_OK;
}

// Profiles of every inflow wall at every level: the caller's fine profiles at
// level 0; a coarse level's are the full-weighting restriction (1/4, 1/2, 1/4,
// ends copied) of the level below along each tangential axis in turn (first
// the lower axis, then the higher one).
m1_status Grid3::set_inflow(const double* faces)
{
    if (!faces || !has_inflow) return M1_ERR_INVALID_ARG;
    const size_t fs0 = face_max3(lv[0].g.n);
    std::vector<double> fine(faces, faces + 6 * 4 * fs0), coarse, tmp, col_f, col_c;
    for (int l = 0; l < L; ++l) {
        Lev3& q = lv[l];
        const size_t fs = (size_t)q.g.fstride;
        if (l > 0) {
            const Lev3& p = lv[l - 1];
            const size_t fsp = (size_t)p.g.fstride;
            coarse.assign(6 * 4 * fs, 0.0);
            for (int w = 0; w < 6; ++w) {
                if (desc.bc[w] != M1_BC_INFLOW) continue;
                const int d = w / 2, ta = d == 0 ? 1 : 0, tb = d == 2 ? 1 : 2;
                const int nfa = p.g.n[ta], nfb = p.g.n[tb], nca = q.g.n[ta], ncb = q.g.n[tb];
                for (int fld = 0; fld < 4; ++fld) {
                    const double* f = fine.data() + ((size_t)w * 4 + fld) * fsp;
                    double* o = coarse.data() + ((size_t)w * 4 + fld) * fs;
                    tmp.assign((size_t)nca * nfb, 0.0);
                    for (int ib = 0; ib < nfb; ++ib)
                        restrict_profile(f + (size_t)ib * nfa, nfa, tmp.data() + (size_t)ib * nca, nca);
                    col_f.resize(nfb);
                    col_c.resize(ncb);
                    for (int ia = 0; ia < nca; ++ia) {
                        for (int ib = 0; ib < nfb; ++ib) col_f[ib] = tmp[(size_t)ib * nca + ia];
                        restrict_profile(col_f.data(), nfb, col_c.data(), ncb);
                        for (int ib = 0; ib < ncb; ++ib) o[(size_t)ib * nca + ia] = col_c[ib];
                    }
                }
            }
            fine.swap(coarse);
        }
        M1_CK(cudaMemcpyAsync(q.prof, fine.data(), sizeof(double) * 6 * 4 * fs,
                              cudaMemcpyHostToDevice, stream));
        M1_CK(cudaStreamSynchronize(stream));
    }
    inflow_set = true;
    return M1_OK;
}

m1_status Grid3::get_state(double* state, int on_device)
{
    if (!state) return M1_ERR_INVALID_ARG;
    Lev3& q = lv[0];
    double* dst = on_device ? state : stage;
    launch3_unpack(q.v, q.vT, dst, q.n, stream);
    M1_CK(cudaGetLastError());
    if (!on_device)
        M1_CK(cudaMemcpyAsync(state, stage, sizeof(double) * 5 * q.n, cudaMemcpyDeviceToHost, stream));
    M1_CK(cudaStreamSynchronize(stream));
    return M1_OK;
}

// ---- one implicit step --------------------------------------------------------------
m1_status Grid3::step(double dt, const m1_solve_params& sp, m1_step_stats* st)
{
    M1_TRY(validate_params(sp));
    if (!(dt > 0) || !state_set || (has_inflow && !inflow_set)) return M1_ERR_INVALID_ARG;
    set_dt(dt);
    const Params p{ sp.nu0, sp.nu_l, sp.m_pseudo, sp.m_coarse, sp.cycle };
    M1_TRY(build_graph(p, dt));
    Ctl c = make_ctl(sp, lv[0].g.diag);
    c.hist = hist;
    c.dtau_hist = dtau_hist;
    c.hist_len = hist_len;
    *ctl_h = c;
    const BatchCtl b{ 0, 1, 0, 0 };
    M1_CK(cudaMemcpyAsync(ctl, ctl_h, sizeof(Ctl), cudaMemcpyHostToDevice, stream));
    M1_CK(cudaMemcpyAsync(bctl, &b, sizeof(BatchCtl), cudaMemcpyHostToDevice, stream));
    M1_CK(cudaEventRecord(ev0, stream));
    Lev3& q = lv[0];
    const int np = blocks3(q.n);
    launch3_rhs(q.g, q.v, q.vT, q.f, q.fT, q.n, stream);
    launch3_closure(q.g, q.v, q.P, q.n, ctl, stream);
    launch3_op(OP3K_RESID, q.g, q.v, q.vT, q.P, q.sig, q.f, q.fT, q.r, q.rT, q.n, ctl, part, stream);
    launch3_norm_state(q.g, q.f, q.fT, partb, q.n, stream);
    launch3_finalize(ctl, bctl, part, partb, np, FIN3_INIT, stream);
    M1_CK(cudaGetLastError());
    long long launched = 0;
    M1_TRY(run_until_done(graph, 1, sp.max_cycles, stream, bctl, done_h, poll, &launched));
    M1_CK(cudaEventRecord(ev1, stream));
    M1_CK(cudaMemcpyAsync(ctl_h, ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, stream));
    M1_CK(cudaStreamSynchronize(stream));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, ev0, ev1);
    const Ctl& r = *ctl_h;
    last_cycles = r.kappa;
    if (st) {
        st->cycles = r.kappa;
        st->res0 = r.res0;
        st->res = r.kappa > 0 ? r.res : r.res0;
        st->dtau_final = r.dtau;
        st->sweeps = (long long)r.kappa * (L == 1 ? p.nu0 : 2 * p.nu0);
        st->ms = ms;
        st->status = r.status;
        st->newton_fail = r.newton_fail;
        st->damped = r.damped;
        st->launches = 5 + launched * kernels_per_cycle;
    }
    return r.status == CTL_OK ? M1_OK : M1_ERR_NOT_CONVERGED;
}

m1_status Grid3::history(double* hs, double* dt, int len)
{
    const int n = std::min(len, std::min(last_cycles + 1, hist_len));
    if (n <= 0) return M1_OK;
    if (hs) M1_CK(cudaMemcpy(hs, hist, sizeof(double) * n, cudaMemcpyDeviceToHost));
    if (dt && n > 1) M1_CK(cudaMemcpy(dt, dtau_hist, sizeof(double) * (n - 1), cudaMemcpyDeviceToHost));
    return M1_OK;
}

m1_status validate_desc3(const m1_grid3_desc* d, int lmax)
{
    if (!d || lmax < 1 || lmax > 20) return M1_ERR_INVALID_ARG;
    if (d->nx < 1 || d->ny < 1 || d->nz < 1 || !(d->lx > 0) || !(d->ly > 0) || !(d->lz > 0) ||
        !(d->c > 0) || !(d->a_r > 0) || !(d->c_v > 0))
        return M1_ERR_INVALID_ARG;
    const long long div = 1LL << (lmax - 1);
    if (d->nx % div || d->ny % div || d->nz % div) return M1_ERR_INVALID_ARG;
    if ((long long)d->nx * d->ny * d->nz > (1LL << 31)) return M1_ERR_INVALID_ARG;
    for (int w = 0; w < 6; ++w)
        if (d->bc[w] < M1_BC_PERIODIC || d->bc[w] > M1_BC_INFLOW) return M1_ERR_INVALID_ARG;
    for (int a = 0; a < 3; ++a)   // periodic walls come in pairs
        if ((d->bc[2 * a] == M1_BC_PERIODIC) != (d->bc[2 * a + 1] == M1_BC_PERIODIC))
            return M1_ERR_INVALID_ARG;
    return M1_OK;
}

}  // namespace
}  // namespace m1

struct m1_grid3 {
    std::unique_ptr<m1::Grid3> g;
};

extern "C" {

m1_status m1_create_grid3(const m1_grid3_desc* desc, int lmax, void* cuda_stream, m1_grid3_t* out)
{
    if (!out) return M1_ERR_INVALID_ARG;
    *out = nullptr;
    M1_TRY(m1::validate_desc3(desc, lmax));
    auto g = std::make_unique<m1::Grid3>();
    M1_TRY(g->init(*desc, lmax, static_cast<cudaStream_t>(cuda_stream)));
    m1_grid3* h = new m1_grid3;
    h->g = std::move(g);
    *out = h;
    return M1_OK;
}

m1_status m1_destroy_grid3(m1_grid3_t g)
{
    if (!g) return M1_ERR_INVALID_ARG;
    delete g;
    return M1_OK;
}

m1_status m1_grid3_set_state(m1_grid3_t g, const double* state, const double* sig, int on_device)
{
    if (!g) return M1_ERR_INVALID_ARG;
    return g->g->set_state(state, sig, on_device);
}

m1_status m1_grid3_set_inflow(m1_grid3_t g, const double* faces)
{
    if (!g) return M1_ERR_INVALID_ARG;
    return g->g->set_inflow(faces);
}

m1_status m1_grid3_get_state(m1_grid3_t g, double* state, int on_device)
{
    if (!g) return M1_ERR_INVALID_ARG;
    return g->g->get_state(state, on_device);
}

m1_status m1_grid3_implicit_step(m1_grid3_t g, double dt, const m1_solve_params* params,
                                 m1_step_stats* stats)
{
    if (!g) return M1_ERR_INVALID_ARG;
    m1_solve_params p;
    if (params) p = *params; else m1_default_params(&p);
    return g->g->step(dt, p, stats);
}

m1_status m1_grid3_step_history(m1_grid3_t g, double* hist, double* dtau, int len)
{
    if (!g) return M1_ERR_INVALID_ARG;
    return g->g->history(hist, dtau, len);
}

}  // extern "C"
