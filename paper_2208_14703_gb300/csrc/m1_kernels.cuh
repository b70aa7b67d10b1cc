// Host-side launchers of the M1 multigrid kernels (definitions in m1_kernels.cu).
// Every launcher takes the device array of one level's descriptors (indexed by
// instance), a work list over that level and the instances' control blocks.
#pragma once
#include "m1_device.cuh"
#include "m1_dw.cuh"

namespace m1 {

enum ApplyMode { APPLY_RESID = 0, APPLY_FAS = 1, APPLY_A = 2 };
// FIN_INIT: r_0 and ||b|| of a new step.  FIN_CYCLE: the residual after a
// cycle, stop test and dtau.  FIN_DEFER: the same for the residual of the state
// a cycle left, computed by the next cycle's first fine sweep (the first such
// norm of a step is r_0 again and only clears the pending flag).
enum FinMode { FIN_INIT = 0, FIN_CYCLE = 1, FIN_DEFER = 2 };

template <typename R>
void launch_sweep(const Level<R>* lv, WorkList wl, Ctl* ctls, bool pseudo, int in_buf,
                  int out_buf, cudaStream_t s, bool delta = false, bool ring = false,
                  double* partials = nullptr, bool fas = false);
template <typename R>
void launch_apply(const Level<R>* lv, WorkList wl, Ctl* ctls, int mode, int state_buf,
                  double* partials, int write_r, cudaStream_t s, bool delta = false);
template <typename R>
void launch_norm_state(const Level<R>* lv, WorkList wl, const Ctl* ctls, double* partials,
                       cudaStream_t s);
template <typename R>
void launch_restrict(const Level<R>* lvf, const Level<R>* lvc, WorkList wl, Ctl* ctls,
                     int fine_buf, cudaStream_t s, bool delta = false);
template <typename R>
void launch_restrict_sig(const Level<R>* lvf, const Level<R>* lvc, WorkList wl, cudaStream_t s);
template <typename R>
void launch_prolong(const Level<R>* lvc, const Level<R>* lvf, WorkList wl, Ctl* ctls,
                    int coarse_buf, int fine_buf, cudaStream_t s, bool delta = false);
template <typename R>
void launch_make_rhs(const Level<R>* lv, WorkList wl, const Ctl* ctls, int buf, cudaStream_t s);
template <typename R>
void launch_finalize(Ctl* ctls, const Level<R>* lv0, int nslots, const double* part,
                     const double* partb, int mode, int cur, BatchCtl* bctl, cudaStream_t s,
                     const int* slot_ids = nullptr);
template <typename R>
void launch_pack_state(const double* E, const double* Fx, const double* Fy, const double* T,
                       double tscale, Cell4<R>* out, int n, cudaStream_t s);
template <typename R>
void launch_unpack_state(const Cell4<R>* in, double* E, double* Fx, double* Fy, double* T, int n,
                         cudaStream_t s);
template <typename R>
void launch_pack_sig(const double* sa, const double* ss, Sig2<R>* out, int n, cudaStream_t s);
template <typename R>
void launch_check_state(const Cell4<R>* st, const Sig2<R>* sig, int n, double c, unsigned int* bad,
                        cudaStream_t s);

// FP32 correction form, coarse level: A(w) -> aw and f = [A(w + v) - A(w)] + r.
void launch_fas_aw32(const Level<float>* lv, WorkList wl, Ctl* ctls, cudaStream_t s);
// The FP64 defect and the next FP32 cycle's problem (w = fl32(v), g = fl32(r));
// first_sweep: also that cycle's first fine sweep from e = 0, into buffer 1
// (else e = 0 in buffer 0).
void launch_defect(const Level<double>* lv64, const Level<float>* lv32, WorkList wl, Ctl* ctls,
                   double* partials, cudaStream_t s, bool first_sweep);
// the defect in double-word FP32, for the instances whose control block chose it
void launch_defect_dw(const Level<double>* lv64, const Level<float>* lv32, const DwLevel* dwd,
                      WorkList wl, Ctl* ctls, double* partials, cudaStream_t s, bool first_sweep);
// double-word copies of the fine level's iterate, right-hand side and opacities
void launch_dw_split(const Level<double>* lv, const DwLevel* dwd, WorkList wl, cudaStream_t s);
// the double-word residual r = b - A(u) of level-0 state u alone (written in FP64),
// for checks; scratch: n double-word cells
void launch_residual_dw(const Level<double>* lv, const Cell4<double>* u, DW4* scratch, int n,
                        WorkList wl, double* partials, cudaStream_t s);
void launch_accumulate(const Level<double>* lv64, const Level<float>* lv32, WorkList wl,
                       Ctl* ctls, int buf, cudaStream_t s, const DwLevel* dwd = nullptr);

}  // namespace m1
