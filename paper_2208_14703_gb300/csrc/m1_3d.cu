// Kernels of the 3D path (the 2D method on three axes; per-cell arithmetic in
// m1_3d.cuh) and the single-level entry point m1_op_level3.
//
// FP64 is what bounds these kernels on GB300 (two FP64 operations per clock per
// SM), so a cell's closure is evaluated once per pass: a first pass writes the
// pressure tensor P of every cell, the operator pass reads the six neighbours'
// (E, F) and P instead of re-evaluating six closures per cell.  The tensor costs
// 48 bytes per cell of traffic, far inside the bandwidth an FP64-bound kernel
// leaves unused.  Every kernel is cell-parallel (a grid-stride loop over a
// grid of at most 152 x 8 blocks); the norm partials are one per block, each a
// fixed-order sum, so norms are bitwise repeatable.
#include <m1.h>

#include <cstdio>

#include "m1_3d.cuh"

namespace m1 {
void set_err(cudaError_t e, const char* what);
void set_error_text(const char* msg);

namespace {

__device__ __forceinline__ bool skip3(const Ctl* ctl) { return ctl && ctl->done; }

// Fixed-order block sum (thread t's own sum, then a fixed tree); thread 0 gets it.
__device__ __forceinline__ double block_sum3(double v, double* red)
{
    red[threadIdx.x] = v;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    return red[0];
}

__global__ void __launch_bounds__(kThreads3) k_closure3(G3 g, const EF* __restrict__ u,
                                                        P6* __restrict__ P, size_t n,
                                                        const Ctl* __restrict__ ctl)
{
    if (skip3(ctl)) return;
    for (size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x; q < n;
         q += (size_t)gridDim.x * blockDim.x)
        P[q] = closure3(u[q], g.ic2);
}

// One cell-parallel pass: the neighbour terms of Eq. (9) on the three axes, then
// A(u) = D(u) - N (APPLY), b - A(u) (RESID, with the cell's norm contribution),
// A(u) + b (FAS, Eq. (24)), the Jacobi update D^{-1}(b + N) (JACOBI, Eq. (10);
// JACOBI_NORM also forms the norm contribution of b - A(u) = (b + N) - D(u) of
// its input, with the residual's expressions), or one pseudo-time step with
// source f = b (PSEUDO, Eq. (30)): the explicit half u~ = u + tau f,
// tau = min(dtau, theta tau*) (tau* the largest admissible step along f), then
// one Jacobi sweep of u' + dtau A(u') = u~ from u.
template <int MODE>
__global__ void __launch_bounds__(kThreads3) k_op3(G3 g, const EF* __restrict__ u,
                                                   const double* __restrict__ T,
                                                   const P6* __restrict__ P,
                                                   const Sig2<double>* __restrict__ sig,
                                                   const EF* __restrict__ b,
                                                   const double* __restrict__ bT,
                                                   EF* __restrict__ out,
                                                   double* __restrict__ outT, size_t n,
                                                   Ctl* __restrict__ ctl, double* __restrict__ part)
{
    __shared__ double red[kThreads3];
    if (skip3(ctl)) return;
    const double c = g.c;
    double dtau = 0.0, theta = 0.0;
    if (MODE == OP3K_PSEUDO) { dtau = ctl->dtau; theta = ctl->theta_ex; }
    double nrm = 0.0;
    unsigned int fails = 0;
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
        if (MODE == OP3K_APPLY || MODE == OP3K_RESID || MODE == OP3K_FAS) {
            const double T2 = Tc * Tc;
            const double src = ka * (uc.E - g.a_r * T2 * T2);
            EF a;
            a.E = g.diag * uc.E + src - N[0];
            for (int m = 0; m < 3; ++m) a.F[m] = (g.diag + kt) * uc.F[m] - N[1 + m];
            double aT = g.c_v * Tc - src;
            if (MODE == OP3K_RESID) {
                const EF bb = b[q];
                a.E = bb.E - a.E;
                for (int m = 0; m < 3; ++m) a.F[m] = bb.F[m] - a.F[m];
                aT = bT[q] - aT;
                nrm += a.E * a.E + (a.F[0] * a.F[0] + a.F[1] * a.F[1] + a.F[2] * a.F[2]) * g.ic2 +
                       aT * aT;
            } else if (MODE == OP3K_FAS) {
                const EF bb = b[q];
                a.E += bb.E;
                for (int m = 0; m < 3; ++m) a.F[m] += bb.F[m];
                aT += bT[q];
            }
            out[q] = a;
            outT[q] = aT;
        } else {
            const EF bb = b[q];
            double bE, bF[3], bTq;
            bool ok;
            EF o;
            double oT;
            if (MODE == OP3K_JACOBI || MODE == OP3K_JACOBI_NORM) {
                bE = bb.E + N[0];
                for (int m = 0; m < 3; ++m) bF[m] = bb.F[m] + N[1 + m];
                bTq = bT[q];
                if (MODE == OP3K_JACOBI_NORM) {
                    const double T2 = Tc * Tc;
                    const double src = ka * (uc.E - g.a_r * T2 * T2);
                    const double rE = bb.E - (g.diag * uc.E + src - N[0]);
                    double rF2 = 0.0;
                    for (int m = 0; m < 3; ++m) {
                        const double rF = bb.F[m] - ((g.diag + kt) * uc.F[m] - N[1 + m]);
                        rF2 += rF * rF;
                    }
                    const double rT = bTq - (g.c_v * Tc - src);
                    nrm += rE * rE + rF2 * g.ic2 + rT * rT;
                }
                local_solve3(0.0, 1.0, g, ka, kt, bE, bF, bTq, o, oT, ok);
            } else {
                const double fT = bT[q];
                const double tau = fmin(dtau, theta * max_step3(uc, Tc, bb, fT, c));
                bE = fma(dtau, N[0], fma(tau, bb.E, uc.E));
                for (int m = 0; m < 3; ++m) bF[m] = fma(dtau, N[1 + m], fma(tau, bb.F[m], uc.F[m]));
                bTq = fma(tau, fT, Tc);
                local_solve3(1.0, dtau, g, ka, kt, bE, bF, bTq, o, oT, ok);
            }
            if (!ok) ++fails;
            out[q] = o;
            outT[q] = oT;
        }
    }
    if ((MODE == OP3K_JACOBI || MODE == OP3K_JACOBI_NORM || MODE == OP3K_PSEUDO) && fails && ctl)
        atomicAdd(&ctl->newton_fail, fails);
    if ((MODE == OP3K_RESID || MODE == OP3K_JACOBI_NORM) && part) {
        const double s = block_sum3(nrm, red);
        if (threadIdx.x == 0) part[blockIdx.x] = s * g.vol;
    }
}

// Section 4.2, Eq. (21) on three axes: coarse cell (ic, jc, kc) gathers the 27
// fine cells 2ic-1 .. 2ic+1 (per axis) with weights 1/4, 1/2, 1/4 per axis; the
// iterate with the state wall rules, the residual with the difference rules.
__global__ void __launch_bounds__(kThreads3) k_restrict3(G3 gf, G3 gc, const EF* __restrict__ u,
                                                         const double* __restrict__ uT,
                                                         const EF* __restrict__ r,
                                                         const double* __restrict__ rT,
                                                         EF* __restrict__ vc,
                                                         double* __restrict__ vcT,
                                                         EF* __restrict__ rc,
                                                         double* __restrict__ rcT,
                                                         const Ctl* __restrict__ ctl)
{
    if (skip3(ctl)) return;
    const double w[3] = { 0.25, 0.5, 0.25 };
    const size_t nc = (size_t)gc.n[0] * gc.n[1] * gc.n[2];
    for (size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x; q < nc;
         q += (size_t)gridDim.x * blockDim.x) {
        const int ic = (int)(q % gc.n[0]);
        const int jc = (int)((q / gc.n[0]) % gc.n[1]);
        const int kc = (int)(q / ((size_t)gc.n[0] * gc.n[1]));
        EF av = { 0.0, { 0.0, 0.0, 0.0 } }, ar = { 0.0, { 0.0, 0.0, 0.0 } };
        double avT = 0.0, arT = 0.0;
        for (int cz = -1; cz <= 1; ++cz)
            for (int by = -1; by <= 1; ++by)
                for (int ax = -1; ax <= 1; ++ax) {
                    const double wt = w[ax + 1] * w[by + 1] * w[cz + 1];
                    const int i = 2 * ic + ax, j = 2 * jc + by, k = 2 * kc + cz;
                    EF s;
                    double sT;
                    fetch3(gf, u, uT, i, j, k, K3_STATE, s, sT);
                    av.E += wt * s.E;
                    for (int a = 0; a < 3; ++a) av.F[a] += wt * s.F[a];
                    avT += wt * sT;
                    fetch3(gf, r, rT, i, j, k, K3_DIFF, s, sT);
                    ar.E += wt * s.E;
                    for (int a = 0; a < 3; ++a) ar.F[a] += wt * s.F[a];
                    arT += wt * sT;
                }
        vc[q] = av;
        vcT[q] = avT;
        rc[q] = ar;
        rcT[q] = arT;
    }
}

__global__ void __launch_bounds__(kThreads3) k_restrict_sig3(G3 gf, G3 gc,
                                                             const Sig2<double>* __restrict__ sf,
                                                             Sig2<double>* __restrict__ sc)
{
    const double w[3] = { 0.25, 0.5, 0.25 };
    const size_t nc = (size_t)gc.n[0] * gc.n[1] * gc.n[2];
    for (size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x; q < nc;
         q += (size_t)gridDim.x * blockDim.x) {
        const int ic = (int)(q % gc.n[0]);
        const int jc = (int)((q / gc.n[0]) % gc.n[1]);
        const int kc = (int)(q / ((size_t)gc.n[0] * gc.n[1]));
        double a = 0.0, b = 0.0;
        for (int cz = -1; cz <= 1; ++cz)
            for (int by = -1; by <= 1; ++by)
                for (int ax = -1; ax <= 1; ++ax) {
                    const double wt = w[ax + 1] * w[by + 1] * w[cz + 1];
                    const Sig2<double> s =
                        sf[fetch_scalar3(gf, 2 * ic + ax, 2 * jc + by, 2 * kc + cz)];
                    a += wt * s.sa;
                    b += wt * s.ss;
                }
        sc[q] = Sig2<double>{ a, b };
    }
}

// Algorithm 4's prolongation with Eq. (34): u += P(u_c - v_c), fine cell 2i
// taking coarse i and 2i + 1 half of coarse i and i + 1 per axis (Fig. 1, the
// tensor product: weights 1, 1/2, 1/4, 1/8), coarse ghosts by the difference
// rules; a cell whose target is not admissible moves theta_c min(1, tau*) of
// the way instead (tau* the largest admissible fraction) and is counted.
__global__ void __launch_bounds__(kThreads3) k_prolong3(G3 gc, G3 gf, const EF* __restrict__ uc,
                                                        const double* __restrict__ ucT,
                                                        const EF* __restrict__ vc,
                                                        const double* __restrict__ vcT,
                                                        EF* __restrict__ uf,
                                                        double* __restrict__ ufT,
                                                        Ctl* __restrict__ ctl)
{
    if (skip3(ctl)) return;
    const double theta = ctl->theta_c, c = gf.c;
    const size_t nf = (size_t)gf.n[0] * gf.n[1] * gf.n[2];
    unsigned int damped = 0;
    for (size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x; q < nf;
         q += (size_t)gridDim.x * blockDim.x) {
        const int i = (int)(q % gf.n[0]);
        const int j = (int)((q / gf.n[0]) % gf.n[1]);
        const int k = (int)(q / ((size_t)gf.n[0] * gf.n[1]));
        const int base[3] = { i / 2, j / 2, k / 2 }, odd[3] = { i % 2, j % 2, k % 2 };
        const double wt = (odd[0] ? 0.5 : 1.0) * (odd[1] ? 0.5 : 1.0) * (odd[2] ? 0.5 : 1.0);
        EF pe = { 0.0, { 0.0, 0.0, 0.0 } };
        double peT = 0.0;
        for (int cz = 0; cz <= odd[2]; ++cz)
            for (int by = 0; by <= odd[1]; ++by)
                for (int ax = 0; ax <= odd[0]; ++ax) {
                    EF a, b;
                    double aT, bT;
                    fetch3(gc, uc, ucT, base[0] + ax, base[1] + by, base[2] + cz, K3_DIFF, a, aT);
                    fetch3(gc, vc, vcT, base[0] + ax, base[1] + by, base[2] + cz, K3_DIFF, b, bT);
                    pe.E += wt * (a.E - b.E);
                    for (int m = 0; m < 3; ++m) pe.F[m] += wt * (a.F[m] - b.F[m]);
                    peT += wt * (aT - bT);
                }
        const EF u = uf[q];
        const double uT = ufT[q];
        EF t;
        t.E = u.E + pe.E;
        for (int m = 0; m < 3; ++m) t.F[m] = u.F[m] + pe.F[m];
        double tT = uT + peT;
        if (!admissible3(t, tT, c)) {
            const double th = theta * fmin(1.0, max_step3(u, uT, pe, peT, c));
            t.E = u.E + th * pe.E;
            for (int m = 0; m < 3; ++m) t.F[m] = u.F[m] + th * pe.F[m];
            tT = uT + th * peT;
            ++damped;
        }
        uf[q] = t;
        ufT[q] = tT;
    }
    if (damped) atomicAdd(&ctl->damped, damped);
}

__global__ void k_copy3(const EF* __restrict__ src, const double* __restrict__ srcT,
                        EF* __restrict__ dst, double* __restrict__ dstT, size_t n,
                        const Ctl* __restrict__ ctl)
{
    if (skip3(ctl)) return;
    for (size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x; q < n;
         q += (size_t)gridDim.x * blockDim.x) {
        dst[q] = src[q];
        dstT[q] = srcT[q];
    }
}

// Right-hand side of Algorithm 4: b = (E^n, F^n, C_v T^n).
__global__ void k_rhs3(G3 g, const EF* __restrict__ u, const double* __restrict__ uT,
                       EF* __restrict__ b, double* __restrict__ bT, size_t n)
{
    for (size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x; q < n;
         q += (size_t)gridDim.x * blockDim.x) {
        b[q] = u[q];
        bT[q] = g.c_v * uT[q];
    }
}

// Per-block partials of ||x||^2 = sum h^3 (E^2 + |F|^2 / c^2 + T^2).
__global__ void __launch_bounds__(kThreads3) k_norm_state3(G3 g, const EF* __restrict__ x,
                                                           const double* __restrict__ xT,
                                                           double* __restrict__ part, size_t n)
{
    __shared__ double red[kThreads3];
    double s = 0.0;
    for (size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x; q < n;
         q += (size_t)gridDim.x * blockDim.x) {
        const EF a = x[q];
        const double t = xT[q];
        s += a.E * a.E + (a.F[0] * a.F[0] + a.F[1] * a.F[1] + a.F[2] * a.F[2]) * g.ic2 + t * t;
    }
    s = block_sum3(s, red);
    if (threadIdx.x == 0) part[blockIdx.x] = s * g.vol;
}

__device__ void mark_done3(Ctl* ctl, BatchCtl* bctl, int status)
{
    ctl->done = 1;
    ctl->status = status;
    if (bctl) {
        const int n = atomicAdd(&bctl->n_done, 1) + 1;
        if (n >= bctl->n_active) bctl->all_done = 1;
    }
}

// One block: the fixed-order sum of the norm partials, then the control logic
// of Algorithm 4 (the rules of the 2D path): INIT records ||r_0|| and ||b|| and
// stops at once below the rounding floor; CYCLE counts the cycle, records the
// residual, stops at tol ||r_0|| or max_cycles, else updates dtau_im.  DEFER is
// CYCLE for a norm formed by the next cycle's first sweep: the first one of a
// step (the norm of v^n again, flagged by INIT) is skipped.
__global__ void __launch_bounds__(kThreads3) k_finalize3(Ctl* __restrict__ ctl,
                                                         BatchCtl* __restrict__ bctl,
                                                         const double* __restrict__ part,
                                                         const double* __restrict__ partb, int np,
                                                         int mode)
{
    __shared__ double red[kThreads3];
    if (mode != FIN3_INIT && ctl->done) return;
    if (mode == FIN3_DEFER) {
        const int first = ctl->pending_r0;
        __syncthreads();
        if (first) {
            if (threadIdx.x == 0) ctl->pending_r0 = 0;
            return;
        }
    }
    double a = 0.0, b = 0.0;
    for (int k = threadIdx.x; k < np; k += blockDim.x) a += part[k];
    const double s = block_sum3(a, red);
    __syncthreads();
    double sb = 0.0;
    if (mode == FIN3_INIT) {
        for (int k = threadIdx.x; k < np; k += blockDim.x) b += partb[k];
        sb = block_sum3(b, red);
    }
    if (threadIdx.x != 0) return;
    const double res = sqrt(s);
    if (mode == FIN3_INIT) {
        ctl->res0 = res; ctl->res = res; ctl->res_prev = res;
        ctl->bnorm = sqrt(sb);
        ctl->dtau = ctl->dtau0;
        ctl->kappa = 0;
        ctl->status = CTL_NOT_CONVERGED;
        ctl->pending_r0 = 1;
        if (ctl->hist_len > 0) ctl->hist[0] = res;
        if (res <= ctl->res0_floor * ctl->bnorm) mark_done3(ctl, bctl, CTL_OK);
        return;
    }
    const int kappa = ++ctl->kappa;
    ctl->res = res;
    if (kappa < ctl->hist_len) { ctl->hist[kappa] = res; ctl->dtau_hist[kappa - 1] = ctl->dtau; }
    if (res <= ctl->tol * ctl->res0) { mark_done3(ctl, bctl, CTL_OK); return; }
    const double delta =
        (ctl->dtau_rule ? ctl->res_prev - res : fabs(res - ctl->res_prev)) / ctl->res0;
    double dtau = ctl->dtau;
    if (delta > ctl->eps_i) dtau *= ctl->grow;
    if (delta < ctl->eps_d) dtau *= ctl->shrink;
    dtau = dtau < ctl->dtau_min ? ctl->dtau_min : (dtau > ctl->dtau_max ? ctl->dtau_max : dtau);
    ctl->dtau = dtau;
    ctl->res_prev = res;
    if (kappa >= ctl->max_cycles) mark_done3(ctl, bctl, CTL_NOT_CONVERGED);
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

__global__ void k_check3(G3 g, const EF* __restrict__ u, const double* __restrict__ T,
                         const Sig2<double>* __restrict__ sig, size_t n, int* __restrict__ bad)
{
    bool b = false;
    for (size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x; q < n;
         q += (size_t)gridDim.x * blockDim.x) {
        const EF e = u[q];
        const double t = T[q];
        const Sig2<double> s = sig[q];
        const double f2 = e.F[0] * e.F[0] + e.F[1] * e.F[1] + e.F[2] * e.F[2];
        const bool ok = isfinite(e.E) && isfinite(f2) && isfinite(t) && e.E > 0.0 && t > 0.0 &&
                        f2 <= g.c * g.c * e.E * e.E * (1.0 + Slack<double>::v) &&
                        isfinite(s.sa) && isfinite(s.ss) && s.sa >= 0.0 && s.ss >= 0.0;
        b = b || !ok;
    }
    if (b) *bad = 1;
}

}  // namespace

void launch3_closure(const G3& g, const EF* u, P6* P, size_t n, const Ctl* ctl, cudaStream_t s)
{
    k_closure3<<<blocks3(n), kThreads3, 0, s>>>(g, u, P, n, ctl);
}

void launch3_op(int mode, const G3& g, const EF* u, const double* uT, const P6* P,
                const Sig2<double>* sig, const EF* b, const double* bT, EF* out, double* outT,
                size_t n, Ctl* ctl, double* part, cudaStream_t s)
{
    const int nb = blocks3(n);
    switch (mode) {
    case OP3K_APPLY:
        k_op3<OP3K_APPLY><<<nb, kThreads3, 0, s>>>(g, u, uT, P, sig, b, bT, out, outT, n, ctl, part);
        break;
    case OP3K_RESID:
        k_op3<OP3K_RESID><<<nb, kThreads3, 0, s>>>(g, u, uT, P, sig, b, bT, out, outT, n, ctl, part);
        break;
    case OP3K_JACOBI:
        k_op3<OP3K_JACOBI><<<nb, kThreads3, 0, s>>>(g, u, uT, P, sig, b, bT, out, outT, n, ctl, part);
        break;
    case OP3K_JACOBI_NORM:
        k_op3<OP3K_JACOBI_NORM><<<nb, kThreads3, 0, s>>>(g, u, uT, P, sig, b, bT, out, outT, n, ctl,
                                                         part);
        break;
    case OP3K_FAS:
        k_op3<OP3K_FAS><<<nb, kThreads3, 0, s>>>(g, u, uT, P, sig, b, bT, out, outT, n, ctl, part);
        break;
    default:
        k_op3<OP3K_PSEUDO><<<nb, kThreads3, 0, s>>>(g, u, uT, P, sig, b, bT, out, outT, n, ctl, part);
        break;
    }
}

void launch3_restrict(const G3& gf, const G3& gc, const EF* u, const double* uT, const EF* r,
                      const double* rT, EF* vc, double* vcT, EF* rc, double* rcT, const Ctl* ctl,
                      cudaStream_t s)
{
    const size_t nc = (size_t)gc.n[0] * gc.n[1] * gc.n[2];
    k_restrict3<<<blocks3(nc), kThreads3, 0, s>>>(gf, gc, u, uT, r, rT, vc, vcT, rc, rcT, ctl);
}

void launch3_restrict_sig(const G3& gf, const G3& gc, const Sig2<double>* sf, Sig2<double>* sc,
                          cudaStream_t s)
{
    const size_t nc = (size_t)gc.n[0] * gc.n[1] * gc.n[2];
    k_restrict_sig3<<<blocks3(nc), kThreads3, 0, s>>>(gf, gc, sf, sc);
}

void launch3_prolong(const G3& gc, const G3& gf, const EF* uc, const double* ucT, const EF* vc,
                     const double* vcT, EF* uf, double* ufT, Ctl* ctl, cudaStream_t s)
{
    const size_t nf = (size_t)gf.n[0] * gf.n[1] * gf.n[2];
    k_prolong3<<<blocks3(nf), kThreads3, 0, s>>>(gc, gf, uc, ucT, vc, vcT, uf, ufT, ctl);
}

void launch3_copy(const EF* src, const double* srcT, EF* dst, double* dstT, size_t n,
                  const Ctl* ctl, cudaStream_t s)
{
    k_copy3<<<blocks3(n), kThreads3, 0, s>>>(src, srcT, dst, dstT, n, ctl);
}

void launch3_rhs(const G3& g, const EF* u, const double* uT, EF* b, double* bT, size_t n,
                 cudaStream_t s)
{
    k_rhs3<<<blocks3(n), kThreads3, 0, s>>>(g, u, uT, b, bT, n);
}

void launch3_norm_state(const G3& g, const EF* x, const double* xT, double* part, size_t n,
                        cudaStream_t s)
{
    k_norm_state3<<<blocks3(n), kThreads3, 0, s>>>(g, x, xT, part, n);
}

void launch3_finalize(Ctl* ctl, BatchCtl* bctl, const double* part, const double* partb, int np,
                      int mode, cudaStream_t s)
{
    k_finalize3<<<1, kThreads3, 0, s>>>(ctl, bctl, part, partb, np, mode);
}

void launch3_pack(const double* planes, EF* ef, double* T, size_t n, cudaStream_t s)
{
    k_pack3<<<blocks3(n), kThreads3, 0, s>>>(planes, ef, T, n);
}

void launch3_unpack(const EF* ef, const double* T, double* planes, size_t n, cudaStream_t s)
{
    k_unpack3<<<blocks3(n), kThreads3, 0, s>>>(ef, T, planes, n);
}

void launch3_pack_sig(const double* planes, Sig2<double>* sig, size_t n, cudaStream_t s)
{
    k_pack_sig3<<<blocks3(n), kThreads3, 0, s>>>(planes, sig, n);
}

void launch3_check(const G3& g, const EF* u, const double* T, const Sig2<double>* sig, size_t n,
                   int* bad, cudaStream_t s)
{
    k_check3<<<blocks3(n), kThreads3, 0, s>>>(g, u, T, sig, n, bad);
}

}  // namespace m1

namespace {

using m1::EF;
using m1::G3;
using m1::P6;
using m1::Sig2;

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
    g.vol = h[0] * h[1] * h[2];

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

    // caller planes -> device layout
    auto pack = [&](const double* src, EF* ef, double* T) -> cudaError_t {
        const double* planes = src;
        if (!on_device) {
            const cudaError_t e = cudaMemcpyAsync(stage, src, 5 * n * sizeof(double),
                                                  cudaMemcpyHostToDevice, s);
            if (e != cudaSuccess) return e;
            planes = stage;
        }
        m1::launch3_pack(planes, ef, T, n, s);
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
        m1::launch3_pack_sig(planes, sg, n, s);
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
    const int kmode = mode == M1_OP3_APPLY ? m1::OP3K_APPLY
                    : mode == M1_OP3_RESIDUAL ? m1::OP3K_RESID : m1::OP3K_JACOBI;
    for (int it = 0; it < passes; ++it) {
        m1::launch3_closure(g, cur, P, n, nullptr, s);
        m1::launch3_op(kmode, g, cur, curT, P, sg, b, bT, nxt, nxtT, n, nullptr, nullptr, s);
        M1_CK3(cudaGetLastError());
        EF* t = cur; cur = nxt; nxt = t;
        double* tt = curT; curT = nxtT; nxtT = tt;
    }
    if (ms) M1_CK3(cudaEventRecord(ev.e[1], s));

    // device layout -> caller planes
    double* dst = on_device ? out : stage;
    m1::launch3_unpack(cur, curT, dst, n, s);
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
