// Host-side launchers of the M1 multigrid kernels (definitions in m1_kernels.cu).
#pragma once
#include "m1_device.cuh"

namespace m1 {

enum ApplyMode { APPLY_RESID = 0, APPLY_FAS = 1, APPLY_A = 2 };
enum FinMode { FIN_INIT = 0, FIN_CYCLE = 1 };

template <typename R>
void launch_sweep(const Level<R>* dL, const Level<R>& hL, bool pseudo, int in_buf, int out_buf,
                  Ctl* ctl, cudaStream_t s, bool delta = false);
template <typename R>
void launch_apply(const Level<R>* dL, const Level<R>& hL, int mode, int state_buf,
                  double* partials, int write_r, Ctl* ctl, cudaStream_t s, bool delta = false);
template <typename R>
void launch_norm_state(const Level<R>* dL, const Level<R>& hL, const Cell4<R>* st,
                       double* partials, cudaStream_t s);
template <typename R>
void launch_restrict(const Level<R>* dLf, const Level<R>* dLc, const Level<R>& hLc, int fine_buf,
                     Ctl* ctl, cudaStream_t s, bool delta = false);
template <typename R>
void launch_restrict_sig(const Level<R>* dLf, const Level<R>* dLc, const Level<R>& hLc,
                         cudaStream_t s);
template <typename R>
void launch_prolong(const Level<R>* dLc, const Level<R>* dLf, const Level<R>& hLf, int coarse_buf,
                    int fine_buf, Ctl* ctl, cudaStream_t s, bool delta = false);
template <typename R>
void launch_make_rhs(const Level<R>* dL, const Level<R>& hL, int buf, cudaStream_t s);
void launch_finalize(Ctl* ctl, const double* part, int np, const double* partb, int npb, int mode,
                     int cur, cudaStream_t s);
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

void launch_defect(const Level<double>* L64, const Level<double>& h64, const Level<float>* L32,
                   double* partials, Ctl* ctl, cudaStream_t s);
void launch_accumulate(const Level<double>* L64, const Level<double>& h64, const Level<float>* L32,
                       int buf, Ctl* ctl, cudaStream_t s);

}  // namespace m1
