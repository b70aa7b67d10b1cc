// Serving: a request loop that runs implicit M1 steps of many simulations on one
// GPU with continuous batching.
//
// A request is a caller's grid (its state already set) and a number of steps.
// Requests go to one of two lanes by size: small ones (at most `small_cells`
// fine cells) and large ones.  Each lane is an engine of its own, driven by a
// scheduler thread of its own on a stream of its own (the small lane's at the
// highest stream priority), so a small request's V-cycle never waits for the
// levels of the largest instances, and the host work of one lane (admission
// copies that wait for its stream) never holds up the other: the two lanes'
// kernels interleave on the GPU.  Within a lane the scheduler admits queued
// requests in arrival order into free slots while all admitted level
// hierarchies of both lanes fit the HBM budget (the state is copied device to
// device; it stays resident for all of the request's steps) and launches
// V-cycle graphs over every active slot, one cycle per batch.  After queueing
// batch b it copies the control blocks asynchronously into a pinned snapshot,
// then waits for the snapshot of batch b - 1 and handles it while b runs: a
// slot whose step converged starts its next step (queued behind b), or, after
// its last step, its result is copied back into the caller's grid and its slot
// and budget are freed; queued requests join between batches.  A snapshot
// taken before a slot's step was started says nothing about that step and is
// ignored for it.  Instances never share arithmetic, so a request's result is
// the same served alone or in a mix.  Step latency is the host time from the
// start of a step to the handling of the snapshot that sees it converged.
#include <m1.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include "m1_engine.h"

namespace {

using m1::Ctl;
using m1::Model;

double now_s()
{
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

struct Request {
    unsigned long long ticket = 0;
    m1_grid* grid = nullptr;
    int nsteps = 0;
    double dt = 0.0;
    m1_solve_params params{};
    size_t bytes = 0;
    int lane = 0;
    int slot = -1;
    long long started_at = 0;     // batches of its lane queued before the current step started
    int steps_done = 0;
    int status = M1_PENDING;
    bool finished = false;
    double t_step = 0.0;
    m1_step_stats last{};
};

// One engine with its slots, queue, stream and snapshot pipeline.
struct Lane {
    std::unique_ptr<Model> model;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    std::deque<std::shared_ptr<Request>> queue;
    std::vector<std::shared_ptr<Request>> slot_req;
    Ctl* snap[2] = { nullptr, nullptr };
    cudaEvent_t snap_ev[2] = { nullptr, nullptr };
    long long batches = 0;        // batches queued so far
    long long handled = 0;        // batches whose snapshot has been handled

    bool active() const
    {
        for (auto& r : slot_req)
            if (r) return true;
        return false;
    }
    int free_slots() const
    {
        int n = 0;
        for (auto& r : slot_req) n += r ? 0 : 1;
        return n;
    }
};

}  // namespace

struct m1_server {
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::map<unsigned long long, std::shared_ptr<Request>> reqs;
    Lane lanes[2];
    m1::Params structure{};
    int precision = 0, L = 0, max_slots = 0, device = 0;
    size_t budget = 0, used = 0, peak = 0;
    long long small_cells = 0;
    int poll_cycles = 1;
    bool stop = false;
    int error = M1_OK;
    unsigned long long next_ticket = 1;
    // statistics
    std::vector<double> latencies_ms;
    long long steps_done = 0, requests_done = 0, cycles = 0;
    double t_first = 0.0, t_last = 0.0;
    std::thread th[2];

    ~m1_server();
    void loop(int k);
    m1_status admit_and_start(Lane& ln, std::vector<std::shared_ptr<Request>>& admit);
    m1_status launch_batch(Lane& ln);
    m1_status handle_snapshot(Lane& ln, long long b);
};

m1_server::~m1_server()
{
    for (Lane& ln : lanes) {
        if (ln.stream) cudaStreamSynchronize(ln.stream);   // no snapshot copy in flight
        ln.model.reset();
        for (int k = 0; k < 2; ++k) {
            if (ln.snap_ev[k]) cudaEventDestroy(ln.snap_ev[k]);
            if (ln.snap[k]) cudaFreeHost(ln.snap[k]);
        }
        if (ln.own_stream && ln.stream) cudaStreamDestroy(ln.stream);
    }
}

m1_status m1_server::admit_and_start(Lane& ln, std::vector<std::shared_ptr<Request>>& admit)
{
    std::vector<int> slots;
    std::vector<double> dts;
    std::vector<m1_solve_params> ps;
    for (auto& r : admit) {
        int slot = -1;
        M1_TRY(ln.model->sv_add(r->grid->model->desc0(), &slot));
        r->slot = slot;
        std::lock_guard<std::mutex> lk(mu);
        ln.slot_req[slot] = r;
    }
    M1_TRY(ln.model->sv_rebuild());
    for (auto& r : admit) {
        M1_TRY(ln.model->sv_copy_in(r->slot, *r->grid->model));
        slots.push_back(r->slot);
        dts.push_back(r->dt);
        ps.push_back(r->params);
    }
    M1_TRY(ln.model->sv_begin(slots, dts, ps));
    const double t = now_s();
    for (auto& r : admit) { r->t_step = t; r->started_at = ln.batches; }
    return M1_OK;
}

// Queue a batch of V-cycles over every active slot of the lane and an
// asynchronous snapshot of its control blocks.
m1_status m1_server::launch_batch(Lane& ln)
{
    M1_TRY(ln.model->sv_cycles(structure, poll_cycles));
    const long long b = ++ln.batches;
    const int nb = (int)(b & 1);
    M1_CK(cudaMemcpyAsync(ln.snap[nb], ln.model->sv_ctl(), sizeof(Ctl) * max_slots,
                          cudaMemcpyDeviceToHost, ln.model->sv_stream()));
    M1_CK(cudaEventRecord(ln.snap_ev[nb], ln.model->sv_stream()));
    std::lock_guard<std::mutex> lk(mu);
    cycles += (long long)poll_cycles * ln.model->sv_graph_cycles();
    return M1_OK;
}

// Per-slot bookkeeping from the snapshot taken after batch b of a lane (its
// copy has completed).
m1_status m1_server::handle_snapshot(Lane& ln, long long b)
{
    ln.handled = b;
    const Ctl* ctl = ln.snap[(int)(b & 1)];
    const double t = now_s();
    std::vector<int> restart;
    std::vector<double> rdts;
    std::vector<m1_solve_params> rps;
    bool removed = false;
    for (int s = 0; s < max_slots; ++s) {
        auto r = ln.slot_req[s];
        if (!r || b <= r->started_at || !ctl[s].active || !ctl[s].done) continue;
        M1_TRY(ln.model->sv_settle(s, ctl[s].result_buf));
        const Ctl& c = ctl[s];
        m1_step_stats st{};
        st.cycles = c.kappa;
        st.res0 = c.res0;
        st.res = c.kappa > 0 ? c.res : c.res0;
        st.dtau_final = c.dtau;
        st.sweeps = (long long)c.kappa * (L == 1 ? structure.nu0 : 2 * structure.nu0);
        st.ms = 1e3 * (t - r->t_step);
        st.status = c.status;
        st.newton_fail = c.newton_fail;
        st.damped = c.damped;
        const bool ok = c.status == m1::CTL_OK;
        bool last;
        {
            std::lock_guard<std::mutex> lk(mu);
            r->last = st;
            r->steps_done += 1;
            latencies_ms.push_back(st.ms);
            steps_done += 1;
            t_last = t;
            last = !ok || r->steps_done >= r->nsteps;
        }
        if (!last) {
            restart.push_back(s);
            rdts.push_back(r->dt);
            rps.push_back(r->params);
            continue;
        }
        M1_TRY(ln.model->sv_copy_out(s, *r->grid->model));
        M1_TRY(ln.model->sv_remove(s));
        removed = true;
        {
            std::lock_guard<std::mutex> lk(mu);
            ln.slot_req[s].reset();
            used -= r->bytes;
            r->status = ok ? M1_OK : M1_ERR_NOT_CONVERGED;
            r->finished = true;
            requests_done += 1;
        }
        cv_done.notify_all();
    }
    if (removed) M1_TRY(ln.model->sv_rebuild());
    if (!restart.empty()) {
        M1_TRY(ln.model->sv_begin(restart, rdts, rps));
        const double t2 = now_s();
        for (int s : restart) { ln.slot_req[s]->t_step = t2; ln.slot_req[s]->started_at = ln.batches; }
    }
    return M1_OK;
}

void m1_server::loop(int k)
{
    cudaSetDevice(device);
    Lane& ln = lanes[k];
    for (;;) {
        std::vector<std::shared_ptr<Request>> admit;
        const bool active = ln.active();
        {
            std::unique_lock<std::mutex> lk(mu);
            if (error != M1_OK) break;
            if (stop && ln.queue.empty() && !active) break;
            // admission in arrival order while a slot is free and the budget allows
            int free_slots = ln.free_slots();
            while (!ln.queue.empty() && free_slots > 0 && used + ln.queue.front()->bytes <= budget) {
                auto r = ln.queue.front();
                ln.queue.pop_front();
                used += r->bytes;
                peak = std::max(peak, used);
                admit.push_back(r);
                --free_slots;
            }
            if (admit.empty() && !active) {
                cv_work.wait_for(lk, std::chrono::milliseconds(20));
                continue;
            }
            if (t_first == 0.0) t_first = now_s();
        }
        m1_status st = M1_OK;
        if (!admit.empty()) st = admit_and_start(ln, admit);
        // queue batch b, then handle the snapshot of batch b - 1 while b runs
        if (st == M1_OK && ln.active()) st = launch_batch(ln);
        const long long prev = ln.batches - 1;
        if (st == M1_OK && prev > ln.handled) {
            const cudaError_t e = cudaEventSynchronize(ln.snap_ev[(int)(prev & 1)]);
            if (e != cudaSuccess) { m1::set_err(e, "cudaEventSynchronize"); st = M1_ERR_CUDA; }
            else st = handle_snapshot(ln, prev);
        }
        if (st != M1_OK) {
            std::lock_guard<std::mutex> lk(mu);
            if (error == M1_OK) error = st;
            for (auto& kv : reqs)
                if (!kv.second->finished) { kv.second->status = st; kv.second->finished = true; }
            for (Lane& other : lanes) other.queue.clear();
            stop = true;
            cv_done.notify_all();
            break;
        }
    }
    cv_work.notify_all();
}

extern "C" {

m1_status m1_server_create(size_t hbm_budget_bytes, int max_slots, int lmax, int precision,
                           const m1_solve_params* structure, long long small_cells,
                           void* cuda_stream, m1_server_t* out)
{
    if (!out || max_slots < 1 || lmax < 1 || lmax > 20 || hbm_budget_bytes == 0 || small_cells < 0 ||
        (precision != M1_FP64 && precision != M1_MIXED))
        return M1_ERR_INVALID_ARG;
    *out = nullptr;
    m1_solve_params p;
    if (structure) p = *structure; else m1_default_params(&p);
    M1_TRY(m1::validate_params(p));
    std::unique_ptr<m1_server> s(new m1_server());
    int lo_prio = 0, hi_prio = 0;
    M1_CK(cudaDeviceGetStreamPriorityRange(&lo_prio, &hi_prio));
    for (int k = 0; k < 2; ++k) {
        Lane& ln = s->lanes[k];
        if (k == 1 && cuda_stream) {
            ln.stream = static_cast<cudaStream_t>(cuda_stream);
        } else {
            // the small lane at the highest priority: its short cycles take SMs
            // as soon as the large lane's blocks free them
            M1_CK(cudaStreamCreateWithPriority(&ln.stream, cudaStreamNonBlocking,
                                               k == 0 ? hi_prio : lo_prio));
            ln.own_stream = true;
        }
        if (precision == M1_MIXED) ln.model.reset(new m1::MixedModel());
        else ln.model.reset(new m1::PlainModel());
        M1_TRY(ln.model->sv_init(max_slots, lmax, ln.stream));
        ln.slot_req.assign(max_slots, nullptr);
        for (int b = 0; b < 2; ++b) {
            if (cudaMallocHost(&ln.snap[b], sizeof(m1::Ctl) * max_slots) != cudaSuccess ||
                cudaEventCreateWithFlags(&ln.snap_ev[b], cudaEventDisableTiming) != cudaSuccess)
                return M1_ERR_OOM;
        }
    }
    s->structure = m1::Params{ p.nu0, p.nu_l, p.m_pseudo, p.m_coarse, p.cycle };
    s->precision = precision;
    s->L = lmax;
    s->max_slots = max_slots;
    s->budget = hbm_budget_bytes;
    s->small_cells = small_cells;
    cudaGetDevice(&s->device);
    m1_server* raw = s.release();
    for (int k = 0; k < 2; ++k) raw->th[k] = std::thread([raw, k] { raw->loop(k); });
    *out = raw;
    return M1_OK;
}

m1_status m1_serve_submit(m1_server_t s, m1_grid_t g, int nsteps, double dt,
                          const m1_solve_params* params, unsigned long long* ticket)
{
    if (!s || !g || !ticket || nsteps < 1 || !(dt > 0)) return M1_ERR_INVALID_ARG;
    const m1_grid_desc& d = g->model->desc0();
    if (g->model->precision() != s->precision || d.lmax != s->L) return M1_ERR_INVALID_ARG;
    auto r = std::make_shared<Request>();
    r->grid = g;
    r->nsteps = nsteps;
    r->dt = dt;
    if (params) r->params = *params; else m1_default_params(&r->params);
    M1_TRY(m1::validate_params(r->params));
    if (r->params.nu0 != s->structure.nu0 || r->params.m_pseudo != s->structure.m ||
        r->params.m_coarse != s->structure.mc || r->params.cycle != s->structure.cycle)
        return M1_ERR_INVALID_ARG;
    r->lane = (long long)d.nx * (d.dim == 2 ? d.ny : 1) <= s->small_cells ? 0 : 1;
    r->bytes = s->lanes[r->lane].model->sv_bytes(d);
    if (r->bytes > s->budget) return M1_ERR_REJECTED;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->stop) return s->error != M1_OK ? (m1_status)s->error : M1_ERR_REJECTED;
        r->ticket = s->next_ticket++;
        s->reqs[r->ticket] = r;
        s->lanes[r->lane].queue.push_back(r);
        *ticket = r->ticket;
    }
    s->cv_work.notify_all();
    return M1_OK;
}

m1_status m1_serve_poll(m1_server_t s, unsigned long long ticket, int* steps_done,
                        m1_step_stats* last)
{
    if (!s) return M1_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return M1_ERR_INVALID_ARG;
    const Request& r = *it->second;
    if (steps_done) *steps_done = r.steps_done;
    if (last) *last = r.last;
    return r.finished ? (m1_status)r.status : M1_PENDING;
}

m1_status m1_serve_wait(m1_server_t s, unsigned long long ticket, double timeout_s)
{
    if (!s) return M1_ERR_INVALID_ARG;
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return M1_ERR_INVALID_ARG;
    auto r = it->second;
    const bool done = s->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s),
                                          [&] { return r->finished; });
    if (!done) return M1_ERR_TIMEOUT;
    return (m1_status)r->status;
}

m1_status m1_server_get_stats(m1_server_t s, m1_server_stats* out)
{
    if (!s || !out) return M1_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    m1_server_stats st{};
    st.requests_done = s->requests_done;
    st.steps_done = s->steps_done;
    st.cycles = s->cycles;
    st.wall_s = s->t_last > s->t_first ? s->t_last - s->t_first : 0.0;
    st.solves_per_s = st.wall_s > 0 ? s->steps_done / st.wall_s : 0.0;
    st.bytes_in_use = (long long)s->used;
    st.bytes_peak = (long long)s->peak;
    int active = 0, queued = 0;
    for (const Lane& ln : s->lanes) {
        for (auto& r : ln.slot_req) active += r ? 1 : 0;
        queued += (int)ln.queue.size();
    }
    st.active = active;
    st.queued = queued;
    if (!s->latencies_ms.empty()) {
        std::vector<double> v = s->latencies_ms;
        std::sort(v.begin(), v.end());
        auto pct = [&](double q) {
            const double x = q * (double)(v.size() - 1);
            const size_t i = (size_t)x;
            const double f = x - (double)i;
            return i + 1 < v.size() ? v[i] * (1 - f) + v[i + 1] * f : v[i];
        };
        st.p50_ms = pct(0.50);
        st.p99_ms = pct(0.99);
        double sum = 0.0;
        for (double x : v) sum += x;
        st.mean_ms = sum / (double)v.size();
    }
    *out = st;
    return M1_OK;
}

m1_status m1_server_destroy(m1_server_t s)
{
    if (!s) return M1_ERR_INVALID_ARG;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv_work.notify_all();
    for (auto& t : s->th)
        if (t.joinable()) t.join();
    const m1_status err = (m1_status)s->error;
    delete s;
    return err;
}

}  // extern "C"
