// Device-side data structures and per-cell arithmetic of the 3D path: the 2D
// method (Bloch, Tremblin, Gonzalez & Audit, arXiv:2208.14703) on three axes.
// The Rusanov faces of Eq. (6) on x, y and z, the 3x3 pressure tensor of
// Eq. (5), the [EXT] sources and local E-T solve of the 2D path with three flux
// components, and the tensor-product transfers of Section 4.2 (R = 2^-3 P^T).
//
// Layout.  A state is two arrays: EF {E, Fx, Fy, Fz} (32 bytes, one vector
// access per cell) and T (8 bytes); index (k * ny + j) * nx + i.  The closure
// of every cell of the operand is written once per pass to a P6 array (48
// bytes), which the operator pass reads for the six face neighbours.
#pragma once
#include <cuda_runtime.h>

#include "m1_device.cuh"

namespace m1 {

struct alignas(32) EF { double E, F[3]; };                       // energy and flux of a cell
struct P6 { double xx, xy, xz, yy, yz, zz; };                    // symmetric pressure tensor

// One 3D level as the kernels see it.  Walls: 0 x low, 1 x high, 2 y low,
// 3 y high, 4 z low, 5 z high.  An inflow wall's profile holds the prescribed
// E, Fx, Fy, Fz of its face cells, field f at in[w] + f * fstride, the face
// cell (a, b) over the wall's two tangential axes a < b at index b * n_a + a.
struct G3 {
    int n[3];
    int bc[6];
    double c, a_r, c_v, ic2, diag, cdt;
    double beta[3];                                              // dt / (2 h_d)
    double vol;                                                  // hx hy hz (norm weight)
    const double* in[6];                                         // inflow profiles, or null
    int fstride;
};

constexpr int kThreads3 = 256;
constexpr int kMaxBlocks3 = 152 * 8;
enum { K3_STATE = 0, K3_DIFF = 1 };

__host__ __device__ inline int blocks3(size_t n)
{
    const size_t b = (n + kThreads3 - 1) / kThreads3;
    return (int)(b < (size_t)kMaxBlocks3 ? (b > 0 ? b : 1) : kMaxBlocks3);
}

__device__ __forceinline__ double P_at(const P6& p, int a, int b)
{
    if (a > b) { const int t = a; a = b; b = t; }
    if (a == 0) return b == 0 ? p.xx : (b == 1 ? p.xy : p.xz);
    if (a == 1) return b == 1 ? p.yy : p.yz;
    return p.zz;
}

// Eq. (5) in the algebraically equal form of the 2D path:
// P = E (s - 1)/3 I + 3/(2 + s) F F^T / (c^2 E), s = sqrt(4 - 3 f^2), f^2 clamped to 1.
__device__ __forceinline__ P6 closure3(const EF& u, double ic2)
{
    const double iE = Fm<double>::rcp(u.E);
    const double px = u.F[0] * iE, py = u.F[1] * iE, pz = u.F[2] * iE;
    double a = fma(fma(pz, pz, fma(py, py, px * px)), -3.0 * ic2, 4.0);
    a = a > 1.0 ? a : 1.0;
    const double s = Fm<double>::sqrt(a);
    const double Eiso = u.E * fma(s, 1.0 / 3.0, -1.0 / 3.0);
    const double q = Fm<double>::rcp(2.0 + s) * (3.0 * ic2);
    const double qx = q * px, qy = q * py, qz = q * pz;
    return P6{ fma(qx, u.F[0], Eiso), qx * u.F[1], qx * u.F[2],
               fma(qy, u.F[1], Eiso), qy * u.F[2], fma(qz, u.F[2], Eiso) };
}

__device__ __forceinline__ size_t at3(const G3& g, int i, int j, int k)
{
    return ((size_t)k * g.n[1] + j) * g.n[0] + i;
}

// The two axes tangential to a wall on axis d, in increasing order.
__device__ __forceinline__ void tangential3(int d, int& a, int& b)
{
    a = d == 0 ? 1 : 0;
    b = d == 2 ? 1 : 2;
}

// Prescribed E, F of the inflow wall on axis d, side `hi`, at the face cell
// under position p (tangential coordinates clamped to the grid).
__device__ __forceinline__ void inflow_at(const G3& g, int d, int hi, const int p[3], EF& o)
{
    int ta, tb;
    tangential3(d, ta, tb);
    const int ia = p[ta] < 0 ? 0 : (p[ta] >= g.n[ta] ? g.n[ta] - 1 : p[ta]);
    const int ib = p[tb] < 0 ? 0 : (p[tb] >= g.n[tb] ? g.n[tb] - 1 : p[tb]);
    const double* prof = g.in[2 * d + hi];
    const size_t f = (size_t)ib * g.n[ta] + ia;
    o.E = prof[f];
    o.F[0] = prof[(size_t)g.fstride + f];
    o.F[1] = prof[2 * (size_t)g.fstride + f];
    o.F[2] = prof[3 * (size_t)g.fstride + f];
}

// A cell at any position one layer around the grid, with the wall rules:
// periodic wrap; reflecting = mirror with the wall-normal flux negated; Neumann
// = copy; inflow = the prescribed E, F at the clamped tangential position with
// T from the mirror cell, and zero everywhere for differences (kind K3_DIFF).
// Edges and corners resolve the axes in order x, y, z and apply the walls'
// rules in the reverse order (the x wall's rule last, on top), the position an
// inflow profile is read at being the one with the lower axes already resolved.
__device__ __forceinline__ void fetch3(const G3& g, const EF* __restrict__ u,
                                       const double* __restrict__ T, int i, int j, int k, int kind,
                                       EF& o, double& oT)
{
    int p[3] = { i, j, k };
    int rule[3] = { -1, -1, -1 };
    int at[3][3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if (p[a] >= 0 && p[a] < g.n[a]) continue;
        const int hi = p[a] < 0 ? 0 : 1;
        const int bc = g.bc[2 * a + hi];
        if (bc == BC_PERIODIC) {
            p[a] = hi ? p[a] - g.n[a] : p[a] + g.n[a];
            continue;
        }
        at[a][0] = p[0]; at[a][1] = p[1]; at[a][2] = p[2];
        p[a] = hi ? 2 * g.n[a] - 1 - p[a] : -1 - p[a];
        rule[a] = bc;
    }
    const size_t q = at3(g, p[0], p[1], p[2]);
    o = u[q];
    oT = T[q];
#pragma unroll
    for (int a = 2; a >= 0; --a) {
        if (rule[a] == BC_REFLECT) {
            o.F[a] = -o.F[a];
        } else if (rule[a] == BC_INFLOW) {
            if (kind == K3_DIFF) {
                o.E = o.F[0] = o.F[1] = o.F[2] = 0.0;
                oT = 0.0;
            } else {
                inflow_at(g, a, at[a][a] < 0 ? 0 : 1, at[a], o);
            }
        }
    }
}

// A scalar (opacity) one layer around the grid: wrap or mirror per axis.
__device__ __forceinline__ size_t fetch_scalar3(const G3& g, int i, int j, int k)
{
    int p[3] = { i, j, k };
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if (p[a] >= 0 && p[a] < g.n[a]) continue;
        if (g.bc[2 * a + (p[a] < 0 ? 0 : 1)] == BC_PERIODIC)
            p[a] = p[a] < 0 ? p[a] + g.n[a] : p[a] - g.n[a];
        else
            p[a] = p[a] < 0 ? -1 - p[a] : 2 * g.n[a] - 1 - p[a];
    }
    return at3(g, p[0], p[1], p[2]);
}

// The face neighbour of cell (i, j, k) across axis d on side `side` (-1 / +1)
// with its pressure tensor: from the closure array, the entries that pair the
// wall-normal axis with another negated at a reflecting wall (the closure of
// the mirrored state), or the closure of the prescribed state at an inflow wall.
__device__ __forceinline__ void neighbour3(const G3& g, const EF* __restrict__ u,
                                           const P6* __restrict__ P, int i, int j, int k, int d,
                                           int side, EF& nb, P6& pn)
{
    int p[3] = { i, j, k };
    p[d] += side;
    int rule = -1;
    if (p[d] < 0 || p[d] >= g.n[d]) {
        const int bc = g.bc[2 * d + (side < 0 ? 0 : 1)];
        if (bc == BC_PERIODIC) {
            p[d] = p[d] < 0 ? p[d] + g.n[d] : p[d] - g.n[d];
        } else if (bc == BC_INFLOW) {
            inflow_at(g, d, side < 0 ? 0 : 1, p, nb);
            pn = closure3(nb, g.ic2);
            return;
        } else {
            p[d] = p[d] < 0 ? -1 - p[d] : 2 * g.n[d] - 1 - p[d];
            rule = bc;
        }
    }
    const size_t q = at3(g, p[0], p[1], p[2]);
    nb = u[q];
    pn = P[q];
    if (rule == BC_REFLECT) {
        nb.F[d] = -nb.F[d];
        if (d == 0) { pn.xy = -pn.xy; pn.xz = -pn.xz; }
        else if (d == 1) { pn.xy = -pn.xy; pn.yz = -pn.yz; }
        else { pn.xz = -pn.xz; pn.yz = -pn.yz; }
    }
}

// Local solve D^{-1} of one cell with the backward-Euler sources (the 2D
// local_solve with three flux components):
//   (w0 + w1 diag) E + w1 ka (E - a_r T^4) = bE,  (w0 + w1 (diag + kt)) F = bF,
//   (w0 + w1 C_v) T - w1 ka (E - a_r T^4) = bT.
// (w0, w1) = (0, 1): Jacobi (Algorithm 1); (1, dtau): implicit pseudo-time step
// (Eq. (30)).  E eliminated, the quartic in T solved as in 2D, E recovered.
__device__ __forceinline__ void local_solve3(double w0, double w1, const G3& g, double ka,
                                             double kt, double bE, const double bF[3], double bT,
                                             EF& o, double& oT, bool& ok)
{
    const double A = w0 + w1 * g.diag, k = w1 * ka, C = w0 + w1 * g.c_v;
    const double dF = w0 + w1 * (g.diag + kt);
    ok = true;
    if (k == 0.0) {
        const double iF = Fm<double>::rcp(dF);
        for (int m = 0; m < 3; ++m) o.F[m] = bF[m] * iF;
        oT = bT / C;
        o.E = bE / A;
        return;
    }
    // one reciprocal for both denominators, as in the 2D local solve
    const double dE = A + k;
    const double ip = Fm<double>::rcp(dF * dE);
    const double iF = dE * ip, iAk = dF * ip;
    for (int m = 0; m < 3; ++m) o.F[m] = bF[m] * iF;
    const double kk = k * iAk;
    const double K = (A * g.a_r) * kk;
    const double R = fma(kk, bE, bT);
    oT = Quartic<double>::solve(C, K, R, ok);
    const double T2 = oT * oT;
    o.E = fma(g.a_r * kk, T2 * T2, bE * iAk);
}

// Largest tau >= 0 with (u, T) + tau (d, dT) admissible (E > 0, T > 0,
// |F| <= c E): the linear E and T bounds and the first positive root of
// |F + tau dF|^2 = c^2 (E + tau dE)^2; +inf when none applies.
__device__ __forceinline__ double max_step3(const EF& u, double T, const EF& d, double dT, double c)
{
    double tau = INFINITY;
    if (d.E < 0.0) tau = fmin(tau, -u.E / d.E);
    if (dT < 0.0) tau = fmin(tau, -T / dT);
    double a = -c * c * d.E * d.E, b = -c * c * u.E * d.E, c0 = -c * c * u.E * u.E;
    for (int q = 0; q < 3; ++q) {
        a += d.F[q] * d.F[q];
        b += u.F[q] * d.F[q];
        c0 += u.F[q] * u.F[q];
    }
    if (c0 > 0.0) c0 = 0.0;
    const double disc = b * b - a * c0;
    double t = INFINITY;
    if (a > 0.0) {
        const double sd = sqrt(disc);
        t = b <= 0.0 ? (-b + sd) / a : -c0 / (b + sd);
    } else if (a < 0.0) {
        if (b > 0.0 && disc >= 0.0) t = -c0 / (b + sqrt(disc));
    } else if (b > 0.0) {
        t = -c0 / (2.0 * b);
    }
    return fmin(tau, t);
}

__device__ __forceinline__ bool admissible3(const EF& s, double T, double c)
{
    return s.E > 0.0 && T > 0.0 &&
           s.F[0] * s.F[0] + s.F[1] * s.F[1] + s.F[2] * s.F[2] <=
               c * c * s.E * s.E * (1.0 + Slack<double>::v);
}

// ---------------------------------------------------------------------------
// Launchers (m1_3d.cu).  Every kernel of a cycle returns at once when the
// control block says done (ctl may be null outside a step).
enum Op3 { OP3K_APPLY = 0, OP3K_RESID = 1, OP3K_JACOBI = 2, OP3K_FAS = 3, OP3K_PSEUDO = 4,
            OP3K_JACOBI_NORM = 5 };

void launch3_closure(const G3& g, const EF* u, P6* P, size_t n, const Ctl* ctl, cudaStream_t s);
// APPLY: out = A(u); RESID: out = b - A(u) (+ per-block norm partials when part
// is not null); JACOBI: one sweep of A(u) = b; FAS: out = A(u) + b; PSEUDO: one
// pseudo-time step with source b (explicit limited half, then one Jacobi sweep
// of u + dtau A(u) = u~; dtau and theta from the control block); JACOBI_NORM:
// a Jacobi sweep that also writes the norm partials of b - A(u) of its input.
void launch3_op(int mode, const G3& g, const EF* u, const double* uT, const P6* P,
                const Sig2<double>* sig, const EF* b, const double* bT, EF* out, double* outT,
                size_t n, Ctl* ctl, double* part, cudaStream_t s);
void launch3_restrict(const G3& gf, const G3& gc, const EF* u, const double* uT, const EF* r,
                      const double* rT, EF* vc, double* vcT, EF* rc, double* rcT, const Ctl* ctl,
                      cudaStream_t s);
void launch3_restrict_sig(const G3& gf, const G3& gc, const Sig2<double>* sf, Sig2<double>* sc,
                          cudaStream_t s);
void launch3_prolong(const G3& gc, const G3& gf, const EF* uc, const double* ucT, const EF* vc,
                     const double* vcT, EF* uf, double* ufT, Ctl* ctl, cudaStream_t s);
void launch3_copy(const EF* src, const double* srcT, EF* dst, double* dstT, size_t n,
                  const Ctl* ctl, cudaStream_t s);
void launch3_rhs(const G3& g, const EF* u, const double* uT, EF* b, double* bT, size_t n,
                 cudaStream_t s);
void launch3_norm_state(const G3& g, const EF* x, const double* xT, double* part, size_t n,
                        cudaStream_t s);
enum { FIN3_INIT = 0, FIN3_CYCLE = 1, FIN3_DEFER = 2 };
void launch3_finalize(Ctl* ctl, BatchCtl* bctl, const double* part, const double* partb, int np,
                      int mode, cudaStream_t s);
void launch3_pack(const double* planes, EF* ef, double* T, size_t n, cudaStream_t s);
void launch3_unpack(const EF* ef, const double* T, double* planes, size_t n, cudaStream_t s);
void launch3_pack_sig(const double* planes, Sig2<double>* sig, size_t n, cudaStream_t s);
// Sets *bad to 1 if some cell is not admissible (E > 0, T > 0, |F| <= c E,
// finite) or has a negative or non-finite opacity.
void launch3_check(const G3& g, const EF* u, const double* T, const Sig2<double>* sig, size_t n,
                   int* bad, cudaStream_t s);

}  // namespace m1
