// Host-side engine of libm1 (definitions in m1_api.cu).
//
// Engine<R>: a fixed number of slots, each holding one instance's level
// hierarchy (all instances share the level count L and the precision R; sizes,
// dimension, walls and time steps are per instance).  Device descriptors are
// laid out [level][slot]; work lists per level enumerate (slot, warp strip) and
// (slot, 256-cell chunk) items of the used slots.  A single grid is an engine
// with one slot, a batch an engine with one slot per instance; the server adds
// and removes slots between V-cycles.
#pragma once
#include <m1.h>

#include <memory>
#include <vector>

#include "m1_kernels.cuh"

namespace m1 {

void set_err(cudaError_t e, const char* what);
void set_error_text(const char* msg);

#define M1_CK(call)                                                                                \
    do {                                                                                           \
        cudaError_t e_ = (call);                                                                   \
        if (e_ != cudaSuccess) {                                                                   \
            ::m1::set_err(e_, #call);                                                              \
            return e_ == cudaErrorMemoryAllocation ? M1_ERR_OOM : M1_ERR_CUDA;                     \
        }                                                                                          \
    } while (0)

#define M1_TRY(expr)                                                                               \
    do {                                                                                           \
        m1_status s_ = (expr);                                                                     \
        if (s_ != M1_OK) return s_;                                                                \
    } while (0)

struct Params {
    int nu0, nu_l, m, mc, cycle;
    bool operator==(const Params& o) const
    {
        return nu0 == o.nu0 && nu_l == o.nu_l && m == o.m && mc == o.mc && cycle == o.cycle;
    }
};

// A device work list and its host mirror.
struct DevList {
    int2* items = nullptr;
    int* count = nullptr;
    int capacity = 0;
    int n = 0;
    std::vector<int2> host;
    WorkList view() const { return WorkList{ items, count, capacity }; }
};

m1_status validate_desc(const m1_grid_desc* d);
// Rows of a sweep strip for a 2D level (kind 0: FP64, 1: FP32), from the
// autotuner's table (m1_tune.cu) or the default rule.
int strip_rows(int kind, int nx, int ny);
// Whether an FP32 correction-form level of this size stages its strip rows
// through shared memory by asynchronous copies (autotuned; default: no).
int strip_ring(int nx, int ny);
m1_status validate_params(const m1_solve_params& sp);
Ctl make_ctl(const m1_solve_params& sp, double diag0);
m1_status run_until_done(cudaGraphExec_t graph, int graph_cycles, int max_cycles,
                         cudaStream_t stream, BatchCtl* bctl, int* done_h, cudaEvent_t* poll,
                         long long* launched_out);
void restrict_profile(const double* fine, int nf, double* coarse, int nc);

template <typename R>
struct Engine {
    int cap = 0, L = 0;
    bool delta = false;                     // correction form (mixed path's FP32 hierarchy)
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    cudaStream_t cap_stream = nullptr;
    std::vector<m1_grid_desc> desc;         // per slot
    std::vector<char> used;
    std::vector<std::vector<void*>> mem;    // per-slot device allocations
    std::vector<void*> common;              // engine-wide device allocations
    std::vector<Level<R>> h;                // host descriptors [level * cap + slot]
    Level<R>* d = nullptr;                  // device descriptors
    std::vector<std::vector<double>> prof;  // inflow profiles [level * cap + slot]
    std::vector<DevList> strips, chunks;    // work lists per level: warp strips, 256-cell chunks
    DevList init_strips, init_chunks;       // scratch lists for one slot
    int* init_slots = nullptr;
    Ctl* ctl = nullptr;                     // device control blocks [cap]
    Ctl* ctl_h = nullptr;                   // pinned mirror
    BatchCtl* bctl = nullptr;
    BatchCtl* bctl_h = nullptr;
    int* done_h = nullptr;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    cudaEvent_t poll[2] = { nullptr, nullptr };
    double* hist = nullptr;
    double* dtau_hist = nullptr;
    int hist_len = 0;
    double* part = nullptr;                 // per-strip norm partials (level 0, all slots)
    double* partb = nullptr;
    int part_cap = 0;
    double* stage = nullptr;                // planar FP64 staging, 6 * stage_n
    size_t stage_n = 0;
    Sig2<R>* sig_stage = nullptr;
    unsigned int* bad = nullptr;
    unsigned int* bad_h = nullptr;
    std::vector<double> dt_set, dt_rhs;
    std::vector<char> rhs_valid;
    std::vector<int> last_cycles;
    cudaGraphExec_t graph = nullptr;
    Params gparams{};
    int graph_cycles = 1;
    bool graph_dirty = true;
    std::vector<char> ring;                 // per level: the sweeps take the cp.async kernel
    std::vector<char> list_sig;             // which work lists were non-empty at capture
    // double-word copies of each slot's level-0 iterate, right-hand side and
    // opacities (the mixed path's FP64 level: its defect in double words)
    bool dw = false;
    DwLevel* dwd = nullptr;                 // device table [cap]
    std::vector<DwLevel> dwh;               // host mirror

    ~Engine();
    std::vector<DevList*> all_lists();
    m1_status calloc_common(void** p, size_t bytes);
    m1_status slot_alloc(int i, void** p, size_t bytes);
    m1_status init(int capacity, int levels, bool correction_form, cudaStream_t s, int history_len);
    m1_status enable_dw();
    m1_status add_slot(const m1_grid_desc& dsc, int* out);
    m1_status remove_slot(int i);
    m1_status ensure_stage(size_t n);
    m1_status upload_list(DevList& l);
    m1_status rebuild();
    m1_status set_dt(int i, double dt);
    m1_status pack_into(int i, Cell4<R>* dst, const double* E, const double* Fx, const double* Fy,
                        const double* T, int dev);
    m1_status unpack_from(const Cell4<R>* src, int n, double* E, double* Fx, double* Fy, double* T,
                          int dev);
    m1_status set_state(int i, const double* E, const double* Fx, const double* Fy, const double* T,
                        const double* sa, const double* ss, int dev);
    m1_status set_inflow(int i, int side, const double* E, const double* Fx, const double* Fy);
    m1_status get_state(int i, double* E, double* Fx, double* Fy, double* T, int dev);
    void sweeps_fine(int& cur, int count, cudaStream_t s);
    void fas_rhs(int l, cudaStream_t s);
    void pseudo(int l, int& cur, int m, bool from_v, cudaStream_t s, bool fas = false);
    // first_done (the FP32 engine of the mixed model): the defect kernels have
    // already formed the first fine sweep into buffer 1, so the cycle starts there
    void record_cycle(const Params& p, int& cur0, cudaStream_t s, bool tail = true,
                      bool first_done = false);
    void visit(const Params& p, int l, bool fresh, int shape, std::vector<int>& cur, cudaStream_t s);
    void corrections(const Params& p, int l, int shape, std::vector<int>& cur, cudaStream_t s);
    long long kernels_per_cycle(const Params& p) const;
    m1_status build_graph(const Params& p);
    m1_status begin_step(const double* dts, const m1_solve_params& sp);
    m1_status step(const double* dts, const m1_solve_params& sp, m1_step_stats* st);
    m1_status residual_norm(int i, double dt, double* out);
    m1_status history(int i, double* hs, double* dt, int len);
    m1_status set_ctl_simple(int i, double dtau, double theta_ex, double theta_c);
    m1_status jacobi(int i, double dt, int sweeps);
    m1_status pack_planar(Cell4<R>* dst, int n, const double* planar);
    m1_status unpack_planar(const Cell4<R>* src, int n, double* planar);
    m1_status op_level(double dt, const double* sig, const double* state, const double* rhs,
                       int mode, double dtau, double theta, double* out, double* norm);
    m1_status op_restrict(const double* state, const double* resid, double* cs, double* cr);
    m1_status op_prolong(const double* uc, const double* vc, const double* uf, double theta,
                         double* out, int* damped);
    // serving
    size_t slot_bytes(const m1_grid_desc& g) const;
    m1_status set_init_lists(const std::vector<int>& slots);
    m1_status copy_slot_in(int slot, Engine<R>& src);
    m1_status copy_slot_out(int slot, Engine<R>& dst);
    m1_status settle(int slot, int result_buf);
};

// One or more instances behind the C ABI: the plain FP64 engine, or the mixed
// pair (FP64 fine level + FP32 correction-form hierarchy).
struct Model {
    virtual ~Model() = default;
    virtual m1_status set_state(int i, const double* E, const double* Fx, const double* Fy,
                                const double* T, const double* sa, const double* ss, int dev) = 0;
    virtual m1_status set_inflow(int i, int side, const double* E, const double* Fx,
                                 const double* Fy) = 0;
    virtual m1_status get_state(int i, double* E, double* Fx, double* Fy, double* T, int dev) = 0;
    virtual m1_status step(const double* dts, const m1_solve_params& p, m1_step_stats* st) = 0;
    virtual m1_status residual_norm(int i, double dt, double* out) = 0;
    virtual m1_status history(int i, double* hist, double* dtau, int len) = 0;
    virtual m1_status jacobi(int i, double dt, int sweeps) = 0;
    virtual const m1_grid_desc& desc0() const = 0;
    virtual int precision() const = 0;
    // serving: slots added and removed between V-cycles of a running engine
    virtual m1_status sv_init(int cap, int L, cudaStream_t s) = 0;
    virtual size_t sv_bytes(const m1_grid_desc& d) const = 0;
    virtual m1_status sv_add(const m1_grid_desc& d, int* slot) = 0;
    virtual m1_status sv_remove(int slot) = 0;
    virtual m1_status sv_rebuild() = 0;
    virtual m1_status sv_copy_in(int slot, Model& src) = 0;
    virtual m1_status sv_copy_out(int slot, Model& dst) = 0;
    virtual m1_status sv_begin(const std::vector<int>& slots, const std::vector<double>& dts,
                               const std::vector<m1_solve_params>& ps) = 0;
    virtual m1_status sv_cycles(const Params& p, int n) = 0;
    virtual m1_status sv_settle(int slot, int result_buf) = 0;
    virtual Ctl* sv_ctl() = 0;                           // device control blocks [cap]
    virtual cudaStream_t sv_stream() = 0;
    virtual int sv_graph_cycles() const { return 1; }   // V-cycles per graph launch
};

struct PlainModel : Model {
    Engine<double> e;
    m1_status create(const std::vector<m1_grid_desc>& descs, cudaStream_t s);
    m1_status set_state(int i, const double* E, const double* Fx, const double* Fy, const double* T,
                        const double* sa, const double* ss, int dev) override
    {
        return e.set_state(i, E, Fx, Fy, T, sa, ss, dev);
    }
    m1_status set_inflow(int i, int side, const double* E, const double* Fx,
                         const double* Fy) override
    {
        return e.set_inflow(i, side, E, Fx, Fy);
    }
    m1_status get_state(int i, double* E, double* Fx, double* Fy, double* T, int dev) override
    {
        return e.get_state(i, E, Fx, Fy, T, dev);
    }
    m1_status step(const double* dts, const m1_solve_params& p, m1_step_stats* st) override
    {
        return e.step(dts, p, st);
    }
    m1_status residual_norm(int i, double dt, double* out) override
    {
        return e.residual_norm(i, dt, out);
    }
    m1_status history(int i, double* hs, double* dt, int len) override
    {
        return e.history(i, hs, dt, len);
    }
    m1_status jacobi(int i, double dt, int sweeps) override { return e.jacobi(i, dt, sweeps); }
    const m1_grid_desc& desc0() const override { return e.desc[0]; }
    int precision() const override { return M1_FP64; }
    m1_status sv_init(int cap, int L, cudaStream_t s) override { return e.init(cap, L, false, s, 0); }
    size_t sv_bytes(const m1_grid_desc& d) const override { return e.slot_bytes(d); }
    m1_status sv_add(const m1_grid_desc& d, int* slot) override { return e.add_slot(d, slot); }
    m1_status sv_remove(int slot) override { return e.remove_slot(slot); }
    m1_status sv_rebuild() override { return e.rebuild(); }
    m1_status sv_copy_in(int slot, Model& src) override;
    m1_status sv_copy_out(int slot, Model& dst) override;
    m1_status sv_begin(const std::vector<int>& slots, const std::vector<double>& dts,
                       const std::vector<m1_solve_params>& ps) override;
    m1_status sv_cycles(const Params& p, int n) override;
    m1_status sv_settle(int slot, int rb) override { return e.settle(slot, rb); }
    Ctl* sv_ctl() override { return e.ctl; }
    cudaStream_t sv_stream() override { return e.stream; }
    int sv_graph_cycles() const override { return e.graph_cycles; }
};

struct MixedModel : Model {
    Engine<double> hi;   // FP64 fine level: v^n, b, opacities, residual, norms, accumulation
    Engine<float> lo;    // FP32 hierarchy in correction form
    cudaGraphExec_t graph = nullptr;
    Params gparams{};
    ~MixedModel() override;
    m1_status create(const std::vector<m1_grid_desc>& descs, cudaStream_t s);
    m1_status set_state(int i, const double* E, const double* Fx, const double* Fy, const double* T,
                        const double* sa, const double* ss, int dev) override;
    m1_status set_inflow(int i, int side, const double* E, const double* Fx,
                         const double* Fy) override;
    m1_status get_state(int i, double* E, double* Fx, double* Fy, double* T, int dev) override
    {
        return hi.get_state(i, E, Fx, Fy, T, dev);
    }
    void record_cycle(const Params& p, cudaStream_t s);
    m1_status build_graph(const Params& p);
    m1_status step(const double* dts, const m1_solve_params& p, m1_step_stats* st) override;
    m1_status residual_norm(int i, double dt, double* out) override
    {
        return hi.residual_norm(i, dt, out);
    }
    m1_status history(int i, double* hs, double* dt, int len) override
    {
        return hi.history(i, hs, dt, len);
    }
    m1_status jacobi(int i, double dt, int sweeps) override;
    const m1_grid_desc& desc0() const override { return lo.desc[0]; }
    int precision() const override { return M1_MIXED; }
    m1_status sv_init(int cap, int L, cudaStream_t s) override;
    size_t sv_bytes(const m1_grid_desc& d) const override;
    m1_status sv_add(const m1_grid_desc& d, int* slot) override;
    m1_status sv_remove(int slot) override;
    m1_status sv_rebuild() override;
    m1_status sv_copy_in(int slot, Model& src) override;
    m1_status sv_copy_out(int slot, Model& dst) override;
    m1_status sv_begin(const std::vector<int>& slots, const std::vector<double>& dts,
                       const std::vector<m1_solve_params>& ps) override;
    m1_status sv_cycles(const Params& p, int n) override;
    m1_status sv_settle(int, int) override { return M1_OK; }
    Ctl* sv_ctl() override { return hi.ctl; }
    cudaStream_t sv_stream() override { return hi.stream; }
};

m1_status make_model(const std::vector<m1_grid_desc>& descs, cudaStream_t s,
                     std::unique_ptr<Model>& out);

}  // namespace m1

// The opaque handles of the C ABI.
struct m1_grid {
    std::unique_ptr<m1::Model> model;
};

struct m1_batch {
    std::unique_ptr<m1::Model> model;
    int count = 0;
};
