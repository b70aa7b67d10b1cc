// Kernels of the implicit M1 multigrid step (arXiv:2208.14703), FP64 and FP32.
//
//   k_sweep     one Jacobi sweep (Algorithm 1 / Eq. (10)); PSEUDO = true fuses
//               the explicit and implicit halves of the pseudo-time step
//               (Eq. (30), Algorithm 3) into the same sweep
//   k_apply     A(u) for the residual r = f - A(u) (Eq. (13)) with per-strip norm
//               partials, or the FAS right-hand side f = A(v) + r (Eq. (24))
//   k_restrict  full-weighting restriction of the iterate and residual (Eq. (21)/(22))
//   k_prolong   prolongation of the coarse correction (Eq. (14)/(18)) with the
//               per-cell damping of Eq. (34)
//   k_finalize  deterministic norm reduction, cycle counter, stop test and the
//               adaptive implicit pseudo-time step (Algorithm 4), per instance
//   k_defect, k_accumulate   FP64 ends of the mixed-precision cycle
//
// Every kernel walks a work list of (instance, strip) or (instance, 256-cell
// chunk) items with a fixed persistent grid, so one launch serves every
// instance of a batch at one level; an instance whose control block says done
// skips its items.  The stencil kernels give each warp a strip of 30 columns
// and march it up the rows with the staged rows (state and closure) in
// registers, so each staged cell's closure is evaluated once per strip.
#include <type_traits>

#include "m1_dw.cuh"
#include "m1_kernels.cuh"

namespace m1 {

template <typename R>
__device__ __forceinline__ void load_level(Level<R>& dst, const Level<R>* src)
{
    static_assert(sizeof(Level<R>) % 8 == 0, "level descriptor size");
    const unsigned long long* s = reinterpret_cast<const unsigned long long*>(src);
    unsigned long long* d = reinterpret_cast<unsigned long long*>(&dst);
    for (int k = threadIdx.x; k < (int)(sizeof(Level<R>) / 8); k += blockDim.x) d[k] = s[k];
}


// The explicit pseudo-time step length min(dtau, theta tau*) of Algorithm 3
// (tau* = the largest admissible step from u along f).  The admissible set is
// convex, so when u + (dtau / theta) f is admissible tau* >= dtau / theta and
// the step is dtau: the divisions and the square root of tau* are needed only
// in cells where the bound may bind.  s = dtau / theta is passed in (once per
// strip).
template <typename R>
__device__ __forceinline__ R limited_step(const Cell4<R>& u, const Cell4<R>& f, R dtau, R theta,
                                          R s, R c)
{
    const Cell4<R> p = { u.E + s * f.E, u.Fx + s * f.Fx, u.Fy + s * f.Fy, u.T + s * f.T };
    if (admissible_c2<R, false>(p, c * c)) return dtau;
    return fmin(dtau, theta * max_admissible_step(u, f, c));
}

// Sum of one double over the lanes of a warp in a fixed order (lane 0 holds it).
__device__ __forceinline__ double warp_sum(double v)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ bool skip(const Ctl* ctls, int inst)
{
    return ctls && (ctls[inst].done || !ctls[inst].active);
}

// 2^-k (0 <= k <= 4) built from its exponent: the transfer weights are products
// of 1/2 and 1/4, exact either way, and this keeps them off the FP64 pipe.
template <typename R>
__device__ __forceinline__ R pow2_neg(int k)
{
    if constexpr (sizeof(R) == 8) return __longlong_as_double((long long)(1023 - k) << 52);
    else return __int_as_float((127 - k) << 23);
}

// Work-list entry w, or (0, 0) past the allocation (entries up to the capacity
// are allocated).  The persistent loops read their first entry together with
// the count instead of after it: a small level's launch is a chain of
// dependent reads (list, descriptor, rows), and this takes one link out.
__device__ __forceinline__ int2 item_at(const WorkList& wl, int w)
{
    return w < wl.capacity ? wl.items[w] : make_int2(0, 0);
}

// ---------------------------------------------------------------------------
// One cell of a warp strip as its neighbours need it: the state (or, in the
// correction form, the correction e) and its closure P (or P(w + e) - P(w)),
// plus the temperature the cell's own update needs (u.T; correction form: the
// base w.T).
template <typename R>
struct Staged {
    R E, Fx, Fy, Pxx, Pxy, Pyy, T;
};

// The loads behind a staged cell (issued one row ahead of their use).
template <typename R>
struct Raw {
    Cell4<R> c, w;
};

template <typename R>
__device__ __forceinline__ Staged<R> shfl_staged(const Staged<R>& v, int from)
{
    Staged<R> o;
    o.E = __shfl_sync(0xffffffffu, v.E, from);
    o.Fx = __shfl_sync(0xffffffffu, v.Fx, from);
    o.Fy = __shfl_sync(0xffffffffu, v.Fy, from);
    o.Pxx = __shfl_sync(0xffffffffu, v.Pxx, from);
    o.Pxy = __shfl_sync(0xffffffffu, v.Pxy, from);
    o.Pyy = __shfl_sync(0xffffffffu, v.Pyy, from);
    o.T = v.T;
    return o;
}

// Cell (i, j) of state s (ghost rules of `fetch` outside the grid; `fast`:
// the whole row of the warp lies inside, plain loads).
template <typename R, bool DELTA>
__device__ __forceinline__ Raw<R> load_raw(const Level<R>& L, const Cell4<R>* __restrict__ s, int i,
                                           int j, bool fast)
{
    Raw<R> r;
    const size_t k = (size_t)j * L.nx + i;
    if (!DELTA) {
        r.c = fast ? s[k] : fetch(L, s, i, j, KIND_STATE);
    } else {
        r.w = fast ? L.w[k] : fetch(L, L.w, i, j, KIND_STATE);
        r.c = fast ? s[k] : fetch(L, s, i, j, KIND_DIFF);
    }
    return r;
}

template <typename R, bool DELTA>
__device__ __forceinline__ Staged<R> stage_raw(const Level<R>& L, const Raw<R>& r)
{
    Staged<R> o;
    o.E = r.c.E; o.Fx = r.c.Fx; o.Fy = r.c.Fy;
    if (!DELTA) {
        closure(r.c.E, r.c.Fx, r.c.Fy, L.ic2, o.Pxx, o.Pxy, o.Pyy);
        o.T = r.c.T;
    } else {
        closure_delta(r.w.E, r.w.Fx, r.w.Fy, r.c.E, r.c.Fx, r.c.Fy, L.ic2, o.Pxx, o.Pxy, o.Pyy);
        o.T = r.w.T;
    }
    return o;
}

// The pseudo-time constants of a sweep, read once per strip: dtau_im, theta_ex
// and dtau_im / theta_ex.
template <typename R>
struct Pseudo {
    R dtau, theta, s;
};

template <typename R>
__device__ __forceinline__ Pseudo<R> pseudo_of(const Ctl* ctl)
{
    const double dtau = ctl->dtau, theta = ctl->theta_ex;
    return Pseudo<R>{ (R)dtau, (R)theta, (R)(dtau / theta) };
}

// The update of one strip cell (lanes 1..30): neighbour operators of Eq. (9)
// from the staged west/east (shuffled) and south/north rows, then the local
// solve of a Jacobi sweep (Algorithm 1) or of the fused pseudo-time step
// (Eq. (30), Algorithm 3).  `u` is the cell's own iterate (the correction e in
// the correction form) and `wb` its base state (correction form only).
//
// NORM (fine Jacobi sweep only): also add the cell's weighted squared residual
// of the input state, r = b - A(u) = (b + N(u)) - D(u) (Eq. (13)), to *nrm: the
// neighbour terms N are the sweep's own, D(u) the local part, written as the
// residual kernel writes it.
//
// FAS (first pseudo-time step of a fresh coarse visit, plain form): the input is
// the restricted iterate v and `b_in` holds the restricted residual r; the
// step first forms the FAS right-hand side f = A(v) + r (Eq. (24)) from its own
// neighbour terms, as the FAS kernel writes it, stores it for the later steps
// and uses it.
template <typename R, bool PSEUDO, bool DELTA, bool NORM = false, bool FAS = false>
__device__ __forceinline__ void update_cell(const Level<R>& L, Ctl* ctl, const Staged<R>& wv,
                                            const Staged<R>& ev, const Staged<R>& prev,
                                            const Staged<R>& next, const Staged<R>& cur,
                                            const Cell4<R>& b_in, const Sig2<R>& sg, size_t k,
                                            int out_buf, bool two_d, const Cell4<R>& u,
                                            const Cell4<R>& wb, const Pseudo<R>& ps,
                                            double* nrm = nullptr)
{
    Cell4<R> b = b_in;
    const R c = L.c, bx = L.bx, by = L.by;
    R NE = bx * (c * (wv.E + ev.E) + (wv.Fx - ev.Fx));
    R NFx = c * bx * ((wv.Fx + ev.Fx) + c * (wv.Pxx - ev.Pxx));
    R NFy = c * bx * ((wv.Fy + ev.Fy) + c * (wv.Pxy - ev.Pxy));
    if (two_d) {
        NE += by * (c * (prev.E + next.E) + (prev.Fy - next.Fy));
        NFx += c * by * ((prev.Fx + next.Fx) + c * (prev.Pxy - next.Pxy));
        NFy += c * by * ((prev.Fy + next.Fy) + c * (prev.Pyy - next.Pyy));
    }
    const R ka = L.cdt * sg.sa, kt = L.cdt * (sg.sa + sg.ss);
    if constexpr (FAS && PSEUDO && !DELTA) {
        const R T2 = cur.T * cur.T;
        const R src_e = ka * (cur.E - L.a_r * T2 * T2);
        const Cell4<R> a = { L.diag * cur.E + src_e - NE, (L.diag + kt) * cur.Fx - NFx,
                             (L.diag + kt) * cur.Fy - NFy, L.c_v * cur.T - src_e };
        b = Cell4<R>{ a.E + b_in.E, a.Fx + b_in.Fx, a.Fy + b_in.Fy, a.T + b_in.T };
        L.f[k] = b;
    }
    if constexpr (NORM && !PSEUDO && !DELTA) {
        const R T2 = cur.T * cur.T;
        const R src_e = ka * (cur.E - L.a_r * T2 * T2);
        const Cell4<R> a = { L.diag * cur.E + src_e - NE, (L.diag + kt) * cur.Fx - NFx,
                             (L.diag + kt) * cur.Fy - NFy, L.c_v * cur.T - src_e };
        const Cell4<R> r = { b.E - a.E, b.Fx - a.Fx, b.Fy - a.Fy, b.T - a.T };
        *nrm += (double)r.E * r.E + ((double)r.Fx * r.Fx + (double)r.Fy * r.Fy) * (double)L.ic2 +
                (double)r.T * r.T;
    }
    bool ok;
    Cell4<R> out;
    if (!PSEUDO) {
        if (!DELTA)
            out = local_solve<R>(R(0), R(1), L.diag, ka, kt, L.c_v, L.a_r, b.E + NE, b.Fx + NFx,
                                 b.Fy + NFy, b.T, ok);
        else
            out = local_solve_delta<R>(R(0), R(1), L.diag, ka, kt, L.c_v, L.a_r, cur.T, b.E + NE,
                                       b.Fx + NFx, b.Fy + NFy, b.T, ok);
    } else {
        // explicit half: u~ = u + tau f, tau = min(dtau, theta tau*); implicit half:
        // one Jacobi sweep of u + dtau A(u) = u~ from the old iterate.
        const R dtau = ps.dtau, theta = ps.theta, dts = ps.s;
        if (!DELTA) {
            const R tau = limited_step(u, b, dtau, theta, dts, c);
            out = local_solve<R>(R(1), dtau, L.diag, ka, kt, L.c_v, L.a_r,
                                 u.E + tau * b.E + dtau * NE, u.Fx + tau * b.Fx + dtau * NFx,
                                 u.Fy + tau * b.Fy + dtau * NFy, u.T + tau * b.T, ok);
        } else {
            // u = w + e and f = A(w) + g: the full-form step u' + dtau A(u') = u + tau f
            // reads, for the correction,
            // e' + dtau (A(w+e') - A(w)) = e + tau g + (tau - dtau) A(w);
            // the last term is zero wherever the step is not limited
            const Cell4<R> aw = L.aw[k];
            const Cell4<R> full = { wb.E + u.E, wb.Fx + u.Fx, wb.Fy + u.Fy, wb.T + u.T };
            const Cell4<R> ff = { aw.E + b.E, aw.Fx + b.Fx, aw.Fy + b.Fy, aw.T + b.T };
            const R tau = limited_step(full, ff, dtau, theta, dts, c);
            const R lim = tau - dtau;
            out = local_solve_delta<R>(R(1), dtau, L.diag, ka, kt, L.c_v, L.a_r, wb.T,
                                       u.E + tau * b.E + lim * aw.E + dtau * NE,
                                       u.Fx + tau * b.Fx + lim * aw.Fx + dtau * NFx,
                                       u.Fy + tau * b.Fy + lim * aw.Fy + dtau * NFy,
                                       u.T + tau * b.T + lim * aw.T, ok);
        }
    }
    if (!ok) atomicAdd(&ctl->newton_fail, 1u);
    L.u[out_buf][k] = out;
}

// One Jacobi sweep (Algorithm 1) or one fused pseudo-time step (Eq. (30),
// Algorithm 3) of one (instance, strip) item by one warp, loads into registers.
//
// The warp takes a strip of 30 columns x L.sh rows (1D: 30 cells): lane l owns
// column x0 - 1 + l, and the warp marches up the rows keeping the staged rows
// j - 1, j, j + 1 in registers (the loads of row j + 2 and of the next own
// cells are issued before row j is updated); the west and east neighbours of a
// lane are its neighbour lanes (warp shuffles), so every staged cell's closure
// is evaluated once per strip (32/30 x (sh + 2)/sh evaluations per updated
// cell) with no shared-memory tile and no block barrier.  Lanes 1..30 update
// their cell.  Ghost rows and columns follow the rules of `fetch`.
template <typename R, bool PSEUDO, bool DELTA, bool NORM = false, bool FAS = false>
__device__ __forceinline__ double strip_regs(const Level<R>& L, Ctl* ctl, int2 it, int lane,
                                             const Cell4<R>* __restrict__ src, int out_buf)
{
    // the cell's right-hand side (FAS: the restricted residual)
    auto rhs = [&](size_t q) { return FAS ? L.r[q] : L.f[q]; };
    double nrm = 0.0;
    const int nx = L.nx, ny = L.ny, two_d = L.dim == 2;
    const int x0 = (it.y % L.sx) * kStripW, y0 = (it.y / L.sx) * L.sh;
    const int i = min(x0 - 1 + lane, nx);       // lanes past the east ghost repeat it
    const bool colfast = x0 >= 1 && x0 + kStripW + 1 <= nx;
    const bool own = lane >= 1 && lane <= kStripW && i < nx;
    const int rows = min(L.sh, ny - y0);
    const Pseudo<R> ps = PSEUDO ? pseudo_of<R>(ctl) : Pseudo<R>{};
    Staged<R> prev{}, cur, next{};
    Raw<R> rn{};
    if (two_d) {
        prev = stage_raw<R, DELTA>(L, load_raw<R, DELTA>(L, src, i, y0 - 1, colfast && y0 >= 1));
        rn = load_raw<R, DELTA>(L, src, i, y0 + 1, colfast && y0 + 1 < ny);
    }
    cur = stage_raw<R, DELTA>(L, load_raw<R, DELTA>(L, src, i, y0, colfast));
    size_t k = (size_t)y0 * nx + i;
    Cell4<R> bn{};
    Sig2<R> sn{};
    if (own) { bn = rhs(k); sn = L.sig[k]; }
    for (int r = 0; r < rows; ++r, k += nx) {
        const int j = y0 + r;
        if (two_d) {
            next = stage_raw<R, DELTA>(L, rn);
            if (r + 1 < rows) rn = load_raw<R, DELTA>(L, src, i, j + 2, colfast && j + 2 < ny);
        }
        const Cell4<R> b = bn;
        const Sig2<R> sg = sn;
        if (own && r + 1 < rows) { bn = rhs(k + nx); sn = L.sig[k + nx]; }
        const Staged<R> wv = shfl_staged(cur, (lane + 31) & 31);
        const Staged<R> ev = shfl_staged(cur, (lane + 1) & 31);
        if (own) {
            Cell4<R> u{}, wb{};
            if (PSEUDO) {
                if (!DELTA) { u = Cell4<R>{ cur.E, cur.Fx, cur.Fy, cur.T }; }
                else { u = src[k]; wb = L.w[k]; }
            }
            update_cell<R, PSEUDO, DELTA, NORM, FAS>(L, ctl, wv, ev, prev, next, cur, b, sg, k,
                                                     out_buf, two_d, u, wb, ps, &nrm);
        }
        prev = cur;
        cur = next;
    }
    return nrm;
}

// Copy the per-warp Level descriptor of item `inst` into shared memory.
template <typename R>
__device__ __forceinline__ void load_level_warp(Level<R>& L, const Level<R>* src, int lane)
{
    const unsigned long long* s = reinterpret_cast<const unsigned long long*>(src);
    unsigned long long* d = reinterpret_cast<unsigned long long*>(&L);
    for (int q = lane; q < (int)(sizeof(Level<R>) / 8); q += 32) d[q] = s[q];
    __syncwarp();
}

// Begin a warp's item of instance `inst`: the level descriptor is read (one
// word per lane) together with the instance's control flags, in one round trip,
// then stored to the warp's shared copy.  False (for the whole warp) when the
// instance is done or inactive.
template <typename R>
__device__ __forceinline__ bool enter_item(Level<R>& L, const Level<R>* src, const Ctl* ctls,
                                           int inst, int lane)
{
    static_assert(sizeof(Level<R>) % 8 == 0 && sizeof(Level<R>) <= 32 * 8, "one word per lane");
    constexpr int nwords = (int)(sizeof(Level<R>) / 8);
    const unsigned long long word =
        lane < nwords ? reinterpret_cast<const unsigned long long*>(src)[lane] : 0ull;
    if (skip(ctls, inst)) return false;
    if (lane < nwords) reinterpret_cast<unsigned long long*>(&L)[lane] = word;
    __syncwarp();
    return true;
}

// Persistent sweep over every listed (instance, strip): one warp per item.
// FP64 instances are held to 128 registers (8 blocks per SM): one register
// more (the pseudo-time variant) cost 4% of the FP64 step on GB300.
// NORM: the fine Jacobi sweep that also writes each strip's weighted residual
// norm partial of its input state (the stop test of the cycle that left it).
// FAS: the first pseudo-time step of a fresh coarse visit, which also forms the
// FAS right-hand side.
template <typename R, bool PSEUDO, bool DELTA = false, bool NORM = false, bool FAS = false>
__global__ void __launch_bounds__(kStripWarps * 32, (sizeof(R) == 8 ? 8 : 10)) k_sweep(const Level<R>* __restrict__ lv,
                                                            WorkList wl, Ctl* __restrict__ ctls,
                                                            int in_buf, int out_buf,
                                                            double* __restrict__ partials)
{
    __shared__ Level<R> Ls[kStripWarps];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    Level<R>& L = Ls[wib];
    const int w0 = blockIdx.x * kStripWarps + wib, ws = gridDim.x * kStripWarps;
    int2 nx = item_at(wl, w0);
    const int nw = *wl.count;
    for (int w = w0; w < nw; w += ws, nx = item_at(wl, w)) {
        const int2 it = nx;
        if (!enter_item(L, lv + it.x, ctls, it.x, lane)) continue;
        const Cell4<R>* __restrict__ src = in_buf < 0 ? L.v : L.u[in_buf];
        const double nrm =
            strip_regs<R, PSEUDO, DELTA, NORM, FAS>(L, ctls + it.x, it, lane, src, out_buf);
        if (NORM) {
            const double sum = warp_sum(nrm);
            if (lane == 0) partials[L.part_off + it.y] = sum * L.vol;
        }
        __syncwarp();
    }
}

// ---------------------------------------------------------------------------
// FP32 correction-form sweep with the strip rows staged through shared memory
// by asynchronous copies (cp.async), kRing - 1 rows ahead of their use, so that
// the loads of three rows are in flight per warp without holding registers.
// Cells outside the grid (ghost rows and columns) are filled by `fetch` with
// the wall rules and stored into the ring directly.
constexpr int kRing = 4;

struct RowSlot32 {
    Cell4<float> w[32], e[32], f[32];
    Sig2<float> sig[32];
};

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s), "l"(gmem) : "memory");
}

__device__ __forceinline__ void cp_async8(void* smem, const void* gmem)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(s), "l"(gmem) : "memory");
}

__device__ __forceinline__ void cp_commit()
{
    asm volatile("cp.async.commit_group;" ::: "memory");
}

template <int N>
__device__ __forceinline__ void cp_wait()
{
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Row q of the strip (lane's column i) into a ring slot: asynchronous copies of
// w, e and, for the lane's own cell, f and sigma; a cell outside the grid is
// fetched with the wall rules and stored directly.  Rows past `last` are not
// needed and leave an empty copy group.
__device__ __forceinline__ void issue_row32(const Level<float>& L,
                                            const Cell4<float>* __restrict__ src, RowSlot32& S,
                                            int i, int q, int last, int lane, bool own)
{
    if (q <= last) {
        if (q >= 0 && q < L.ny && i >= 0 && i < L.nx) {
            const size_t k = (size_t)q * L.nx + i;
            cp_async16(&S.w[lane], L.w + k);
            cp_async16(&S.e[lane], src + k);
            if (own) {
                cp_async16(&S.f[lane], L.f + k);
                cp_async8(&S.sig[lane], L.sig + k);
            }
        } else {
            S.w[lane] = fetch(L, L.w, i, q, KIND_STATE);
            S.e[lane] = fetch(L, src, i, q, KIND_DIFF);
        }
    }
    cp_commit();
}

// The 1D form of a strip (one row of 30 updated cells, no y neighbours).
template <bool PSEUDO>
__device__ __forceinline__ void row_1d32(const Level<float>& L, Ctl* ctl, int2 it, int lane,
                                         const Cell4<float>* __restrict__ src, int out_buf)
{
    const int nx = L.nx;
    const int x0 = it.y * kStripW;
    const int i = min(x0 - 1 + lane, nx);
    const bool own = lane >= 1 && lane <= kStripW && i < nx;
    const bool fast = x0 >= 1 && x0 + kStripW + 1 <= nx;
    const Pseudo<float> ps = PSEUDO ? pseudo_of<float>(ctl) : Pseudo<float>{};
    const Staged<float> cur = stage_raw<float, true>(L, load_raw<float, true>(L, src, i, 0, fast));
    const Staged<float> wv = shfl_staged(cur, (lane + 31) & 31);
    const Staged<float> ev = shfl_staged(cur, (lane + 1) & 31);
    if (own) {
        const size_t k = (size_t)i;
        Cell4<float> u{}, wb{};
        if (PSEUDO) { u = src[k]; wb = L.w[k]; }
        update_cell<float, PSEUDO, true>(L, ctl, wv, ev, cur, cur, cur, L.f[k], L.sig[k], k,
                                         out_buf, false, u, wb, ps);
    }
}

template <bool PSEUDO>
__device__ __forceinline__ void strip_ring32(const Level<float>& L, Ctl* ctl, int2 it, int lane,
                                             const Cell4<float>* __restrict__ src, int out_buf,
                                             RowSlot32* ring)
{
    const int nx = L.nx, ny = L.ny;
    const int x0 = (it.y % L.sx) * kStripW, y0 = (it.y / L.sx) * L.sh;
    const int i = min(x0 - 1 + lane, nx);       // lanes past the east ghost repeat it
    const bool own = lane >= 1 && lane <= kStripW && i < nx;
    const int rows = min(L.sh, ny - y0);
    const int last = y0 + rows;               // the last row the strip reads
    const Pseudo<float> ps = PSEUDO ? pseudo_of<float>(ctl) : Pseudo<float>{};
    // ring slot of row q: (q - y0 + 1) mod kRing
    for (int q = y0 - 1; q <= y0 + 2; ++q) issue_row32(L, src, ring[(q - y0 + 1) & 3], i, q, last,
                                                       lane, own);
    cp_wait<2>();                             // rows y0 - 1 and y0
    auto stage = [&](const RowSlot32& S) {
        Raw<float> r;
        r.w = S.w[lane];
        r.c = S.e[lane];
        return stage_raw<float, true>(L, r);
    };
    Staged<float> prev = stage(ring[0]), cur = stage(ring[1]), next{};
    size_t k = (size_t)y0 * nx + i;
    for (int r = 0; r < rows; ++r, k += nx) {
        cp_wait<1>();                         // row j + 1
        next = stage(ring[(r + 2) & 3]);
        issue_row32(L, src, ring[r & 3], i, y0 + r + 3, last, lane, own);
        const Staged<float> wv = shfl_staged(cur, (lane + 31) & 31);
        const Staged<float> ev = shfl_staged(cur, (lane + 1) & 31);
        if (own) {
            const RowSlot32& S = ring[(r + 1) & 3];
            const Cell4<float> b = S.f[lane];
            const Sig2<float> sg = S.sig[lane];
            Cell4<float> u{}, wb{};
            if (PSEUDO) { u = S.e[lane]; wb = S.w[lane]; }
            update_cell<float, PSEUDO, true>(L, ctl, wv, ev, prev, next, cur, b, sg, k, out_buf,
                                             true, u, wb, ps);
        }
        prev = cur;
        cur = next;
    }
    cp_wait<0>();                             // no copy outlives the item
}

template <bool PSEUDO>
__global__ void __launch_bounds__(kStripWarps * 32) k_sweep_ring32(const Level<float>* __restrict__ lv,
                                                                   WorkList wl,
                                                                   Ctl* __restrict__ ctls,
                                                                   int in_buf, int out_buf)
{
    __shared__ Level<float> Ls[kStripWarps];
    __shared__ RowSlot32 ring[kStripWarps][kRing];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    Level<float>& L = Ls[wib];
    const int w0 = blockIdx.x * kStripWarps + wib, ws = gridDim.x * kStripWarps;
    int2 nx = item_at(wl, w0);
    const int nw = *wl.count;
    for (int w = w0; w < nw; w += ws, nx = item_at(wl, w)) {
        const int2 it = nx;
        if (!enter_item(L, lv + it.x, ctls, it.x, lane)) continue;
        const Cell4<float>* __restrict__ src = in_buf < 0 ? L.v : L.u[in_buf];
        if (L.dim == 2) strip_ring32<PSEUDO>(L, ctls + it.x, it, lane, src, out_buf, ring[wib]);
        else row_1d32<PSEUDO>(L, ctls + it.x, it, lane, src, out_buf);
        __syncwarp();
    }
}


// Neighbour operators L and R of Eq. (9) of a strip cell from its staged west /
// east (shuffled) and south / north rows.
template <typename R>
__device__ __forceinline__ void strip_neighbours(const Level<R>& L, const Staged<R>& wv,
                                                 const Staged<R>& ev, const Staged<R>& prev,
                                                 const Staged<R>& next, bool two_d, R& NE,
                                                 R& NFx, R& NFy)
{
    const R c = L.c, bx = L.bx, by = L.by;
    NE = bx * (c * (wv.E + ev.E) + (wv.Fx - ev.Fx));
    NFx = c * bx * ((wv.Fx + ev.Fx) + c * (wv.Pxx - ev.Pxx));
    NFy = c * bx * ((wv.Fy + ev.Fy) + c * (wv.Pxy - ev.Pxy));
    if (two_d) {
        NE += by * (c * (prev.E + next.E) + (prev.Fy - next.Fy));
        NFx += c * by * ((prev.Fx + next.Fx) + c * (prev.Pxy - next.Pxy));
        NFy += c * by * ((prev.Fy + next.Fy) + c * (prev.Pyy - next.Pyy));
    }
}

// March one warp up an (instance, strip) item with the staged rows j - 1, j,
// j + 1 in registers (loads of row j + 2 issued before row j is used) and call
// cell(k, wv, ev, prev, next, cur) for each own cell (lanes 1..30 inside the
// grid).  The layout is the sweep's (strip_regs).
template <typename R, bool DELTA, typename F>
__device__ __forceinline__ void strip_march(const Level<R>& L, int2 it, int lane,
                                            const Cell4<R>* __restrict__ src, F&& cell)
{
    const int nx = L.nx, ny = L.ny, two_d = L.dim == 2;
    const int x0 = (it.y % L.sx) * kStripW, y0 = (it.y / L.sx) * L.sh;
    const int i = min(x0 - 1 + lane, nx);
    const bool colfast = x0 >= 1 && x0 + kStripW + 1 <= nx;
    const bool own = lane >= 1 && lane <= kStripW && i < nx;
    const int rows = min(L.sh, ny - y0);
    Staged<R> prev{}, cur, next{};
    Raw<R> rn{};
    if (two_d) {
        prev = stage_raw<R, DELTA>(L, load_raw<R, DELTA>(L, src, i, y0 - 1, colfast && y0 >= 1));
        rn = load_raw<R, DELTA>(L, src, i, y0 + 1, colfast && y0 + 1 < ny);
    }
    cur = stage_raw<R, DELTA>(L, load_raw<R, DELTA>(L, src, i, y0, colfast));
    size_t k = (size_t)y0 * nx + i;
    for (int r = 0; r < rows; ++r, k += nx) {
        const int j = y0 + r;
        if (two_d) {
            next = stage_raw<R, DELTA>(L, rn);
            if (r + 1 < rows) rn = load_raw<R, DELTA>(L, src, i, j + 2, colfast && j + 2 < ny);
        }
        const Staged<R> wv = shfl_staged(cur, (lane + 31) & 31);
        const Staged<R> ev = shfl_staged(cur, (lane + 1) & 31);
        if (own) cell(k, wv, ev, prev, next, cur);
        prev = cur;
        cur = next;
    }
}

template <typename R, int MODE, bool DELTA>
__device__ __forceinline__ double apply_item(const Level<R>& L, int2 it, int lane, int state_buf,
                                             int write_r)
{
    // state_buf: 0/1 the iterate, -1 the restricted iterate v, -2 the base w
    const Cell4<R>* __restrict__ src =
        state_buf == -2 ? L.w : (state_buf < 0 ? L.v : L.u[state_buf]);
    const bool two_d = L.dim == 2;
    double nrm = 0.0;
    strip_march<R, DELTA>(L, it, lane, src, [&](size_t k, const Staged<R>& wv,
                                                 const Staged<R>& ev, const Staged<R>& prev,
                                                 const Staged<R>& next, const Staged<R>& cur) {
        R NE, NFx, NFy;
        strip_neighbours(L, wv, ev, prev, next, two_d, NE, NFx, NFy);
        const Cell4<R> u = src[k];
        const Sig2<R> sg = L.sig[k];
        const R ka = L.cdt * sg.sa, kt = L.cdt * (sg.sa + sg.ss);
        R src_e;
        if (!DELTA) {
            const R T2 = u.T * u.T;
            src_e = ka * (u.E - L.a_r * T2 * T2);
        } else {
            // A(w + e) - A(w): source difference ka (e_E - a_r ((T + e_T)^4 - T^4))
            src_e = ka * (u.E - L.a_r * quartic_delta(cur.T, u.T));
        }
        Cell4<R> a;
        a.E = L.diag * u.E + src_e - NE;
        a.Fx = (L.diag + kt) * u.Fx - NFx;
        a.Fy = (L.diag + kt) * u.Fy - NFy;
        a.T = L.c_v * u.T - src_e;
        if (MODE == APPLY_RESID) {
            const Cell4<R> f = L.f[k];
            const Cell4<R> r = { f.E - a.E, f.Fx - a.Fx, f.Fy - a.Fy, f.T - a.T };
            if (write_r) L.r[k] = r;
            nrm += (double)r.E * r.E + ((double)r.Fx * r.Fx + (double)r.Fy * r.Fy) * (double)L.ic2 +
                   (double)r.T * r.T;
        } else if (MODE == APPLY_FAS) {
            const Cell4<R> r = L.r[k];
            L.f[k] = Cell4<R>{ a.E + r.E, a.Fx + r.Fx, a.Fy + r.Fy, a.T + r.T };
        } else if (state_buf == -2) {
            L.aw[k] = a;
        } else {
            L.r[k] = a;
        }
    });
    return nrm;
}

// A(u) of Eq. (12) (+ sources) at one level, per (instance, strip) item:
//   APPLY_RESID  r = f - A(u) (Eq. (13)), written to L.r if write_r, and the
//                weighted norm partial of the strip (partials != null)
//   APPLY_FAS    f = A(v) + r (Eq. (24))
//   APPLY_A      r = A(u), or aw = A(w) when state_buf = -2
// DELTA (correction form): u is a correction e around the base w and the
// operator is the difference A(w + e) - A(w).
template <typename R, int MODE, bool DELTA = false>
__global__ void __launch_bounds__(kStripWarps * 32) k_apply(const Level<R>* __restrict__ lv,
                                                            WorkList wl, Ctl* __restrict__ ctls,
                                                            int state_buf,
                                                            double* __restrict__ partials,
                                                            int write_r)
{
    __shared__ Level<R> Ls[kStripWarps];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    Level<R>& L = Ls[wib];
    const int w0 = blockIdx.x * kStripWarps + wib, ws = gridDim.x * kStripWarps;
    int2 nx = item_at(wl, w0);
    const int nw = *wl.count;
    for (int w = w0; w < nw; w += ws, nx = item_at(wl, w)) {
        const int2 it = nx;
        if (!enter_item(L, lv + it.x, ctls, it.x, lane)) continue;
        const double nrm = apply_item<R, MODE, DELTA>(L, it, lane, state_buf, write_r);
        if (MODE == APPLY_RESID && partials) {
            const double sum = warp_sum(nrm);
            if (lane == 0) partials[L.part_off + it.y] = sum * L.vol;
        }
        __syncwarp();
    }
}

// The coarse-level right-hand side of the correction form in one pass: the base
// operator A(w) (kept for the pseudo-time steps of the cycle) and the FAS
// right-hand side f = [A(w + v) - A(w)] + r of the restricted correction v
// (Eq. (24) in correction form).  Both come from the same staged rows: one load
// of w and v per cell feeds the closure of w and the closure difference.
__device__ __forceinline__ void fas_aw32_item(const Level<float>& L, int2 it, int lane)
{
    const int nx = L.nx, ny = L.ny;
    const bool two_d = L.dim == 2;
    const int x0 = (it.y % L.sx) * kStripW, y0 = (it.y / L.sx) * L.sh;
    const int i = min(x0 - 1 + lane, nx);
    const bool colfast = x0 >= 1 && x0 + kStripW + 1 <= nx;
    const bool own = lane >= 1 && lane <= kStripW && i < nx;
    const int rows = min(L.sh, ny - y0);
    auto stage2 = [&](const Raw<float>& r, Staged<float>& sw, Staged<float>& sd) {
        Raw<float> rw;
        rw.c = r.w;
        sw = stage_raw<float, false>(L, rw);
        sd = stage_raw<float, true>(L, r);
    };
    Staged<float> pw{}, cw, nw_{}, pd{}, cd, nd{};
    Raw<float> rn{};
    if (two_d) {
        stage2(load_raw<float, true>(L, L.v, i, y0 - 1, colfast && y0 >= 1), pw, pd);
        rn = load_raw<float, true>(L, L.v, i, y0 + 1, colfast && y0 + 1 < ny);
    }
    stage2(load_raw<float, true>(L, L.v, i, y0, colfast), cw, cd);
    size_t k = (size_t)y0 * nx + i;
    for (int r = 0; r < rows; ++r, k += nx) {
        const int j = y0 + r;
        if (two_d) {
            stage2(rn, nw_, nd);
            if (r + 1 < rows) rn = load_raw<float, true>(L, L.v, i, j + 2, colfast && j + 2 < ny);
        }
        const Staged<float> wvw = shfl_staged(cw, (lane + 31) & 31);
        const Staged<float> evw = shfl_staged(cw, (lane + 1) & 31);
        const Staged<float> wvd = shfl_staged(cd, (lane + 31) & 31);
        const Staged<float> evd = shfl_staged(cd, (lane + 1) & 31);
        if (own) {
            const Sig2<float> sg = L.sig[k];
            const float ka = L.cdt * sg.sa, kt = L.cdt * (sg.sa + sg.ss);
            const Cell4<float> wb = L.w[k], v = L.v[k];
            float NE, NFx, NFy;
            strip_neighbours(L, wvw, evw, pw, nw_, two_d, NE, NFx, NFy);
            const float T2 = wb.T * wb.T, sw = ka * (wb.E - L.a_r * T2 * T2);
            L.aw[k] = Cell4<float>{ L.diag * wb.E + sw - NE, (L.diag + kt) * wb.Fx - NFx,
                                    (L.diag + kt) * wb.Fy - NFy, L.c_v * wb.T - sw };
            strip_neighbours(L, wvd, evd, pd, nd, two_d, NE, NFx, NFy);
            const float sd = ka * (v.E - L.a_r * quartic_delta(wb.T, v.T));
            const Cell4<float> rr = L.r[k];
            L.f[k] = Cell4<float>{ (L.diag * v.E + sd - NE) + rr.E,
                                   ((L.diag + kt) * v.Fx - NFx) + rr.Fx,
                                   ((L.diag + kt) * v.Fy - NFy) + rr.Fy,
                                   (L.c_v * v.T - sd) + rr.T };
        }
        pw = cw; cw = nw_;
        pd = cd; cd = nd;
    }
}

__global__ void __launch_bounds__(kStripWarps * 32) k_fas_aw32(const Level<float>* __restrict__ lv,
                                                               WorkList wl,
                                                               Ctl* __restrict__ ctls)
{
    __shared__ Level<float> Ls[kStripWarps];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    Level<float>& L = Ls[wib];
    const int w0 = blockIdx.x * kStripWarps + wib, ws = gridDim.x * kStripWarps;
    int2 nx = item_at(wl, w0);
    const int nw = *wl.count;
    for (int w = w0; w < nw; w += ws, nx = item_at(wl, w)) {
        const int2 it = nx;
        if (!enter_item(L, lv + it.x, ctls, it.x, lane)) continue;
        fas_aw32_item(L, it, lane);
        __syncwarp();
    }
}

// Norm of the right-hand side f of each instance (for ||b||): per-strip partials.
template <typename R>
__global__ void __launch_bounds__(kStripWarps * 32) k_norm_state(const Level<R>* __restrict__ lv,
                                                                 WorkList wl,
                                                                 const Ctl* __restrict__ ctls,
                                                                 double* __restrict__ partials)
{
    __shared__ Level<R> Ls[kStripWarps];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    Level<R>& L = Ls[wib];
    const int w0 = blockIdx.x * kStripWarps + wib, ws = gridDim.x * kStripWarps;
    int2 nx = item_at(wl, w0);
    const int nw = *wl.count;
    for (int w = w0; w < nw; w += ws, nx = item_at(wl, w)) {
        const int2 it = nx;
        if (ctls && !ctls[it.x].active) continue;
        load_level_warp(L, lv + it.x, lane);
        const int x0 = (it.y % L.sx) * kStripW, y0 = (it.y / L.sx) * L.sh;
        const int i = x0 - 1 + lane;
        const int rows = min(L.sh, L.ny - y0);
        double nrm = 0.0;
        if (lane >= 1 && lane <= kStripW && i < L.nx)
            for (int r = 0; r < rows; ++r) {
                const Cell4<R> f = L.f[(size_t)(y0 + r) * L.nx + i];
                nrm += (double)f.E * f.E + ((double)f.Fx * f.Fx + (double)f.Fy * f.Fy) *
                       (double)L.ic2 + (double)f.T * f.T;
            }
        const double sum = warp_sum(nrm);
        if (lane == 0) partials[L.part_off + it.y] = sum * L.vol;
        __syncwarp();
    }
}

// ---------------------------------------------------------------------------
// Full weighting, coarse cell (ic, jc) <- fine cells 2ic-1..2ic+1 (x) and
// 2jc-1..2jc+1 (y, 2D only), weights 1/4, 1/2, 1/4 per axis: the iterate of
// buffer fine_buf, the residual and, in the correction form, the base w.
// FP32: row by row of the stencil, the sources of its three cells are mapped
// first (ghost rules of `fetch`) and their loads issued together, then the rules
// applied and the weighted values summed in the order of the stencil; the
// coarse FP32 levels are small and this takes the loads' latency off the chain.
// FP64 keeps one stencil point at a time: its restriction is bound by the FP64
// pipe, and the registers of the batched loads cost it occupancy (measured: the
// FP64 step 3.7% slower).  Both forms sum the same values in the same order.
template <typename R, bool DELTA>
__device__ __forceinline__ void restrict_cell(const Level<R>& Lf, const Level<R>& Lc, int kc,
                                              int fine_buf)
{
    const R wgt[3] = { R(0.25), R(0.5), R(0.25) };
    const int ic = kc % Lc.nx, jc = kc / Lc.nx;
    const Cell4<R>* __restrict__ us = Lf.u[fine_buf];
    Cell4<R> av = { 0, 0, 0, 0 }, ar = { 0, 0, 0, 0 }, aw = { 0, 0, 0, 0 };
    const int b0 = Lf.dim == 2 ? -1 : 0, b1 = Lf.dim == 2 ? 1 : 0;
    if constexpr (sizeof(R) == 8) {
        // the whole 3 x 3 (1D: 3) fine stencil inside the grid: plain loads
        const bool inside = 2 * ic >= 1 && 2 * ic + 1 < Lf.nx &&
                            (Lf.dim != 2 || (2 * jc >= 1 && 2 * jc + 1 < Lf.ny));
        auto get = [&](const Cell4<R>* arr, int i, int j, int kind) {
            return inside ? arr[(size_t)j * Lf.nx + i] : fetch(Lf, arr, i, j, kind);
        };
        for (int b = b0; b <= b1; ++b) {
            // weights 2^-(eb + ea): 1/4, 1/2, 1/4 per axis (1D: no y factor)
            const int eb = Lf.dim == 2 ? (b == 0 ? 1 : 2) : 0;
            const int jf = Lf.dim == 2 ? 2 * jc + b : 0;
            for (int a = -1; a <= 1; ++a) {
                const R wt = pow2_neg<R>(eb + (a == 0 ? 1 : 2));
                const Cell4<R> s = get(us, 2 * ic + a, jf, DELTA ? KIND_DIFF : KIND_STATE);
                const Cell4<R> r = get(Lf.r, 2 * ic + a, jf, KIND_DIFF);
                av.E += wt * s.E; av.Fx += wt * s.Fx; av.Fy += wt * s.Fy; av.T += wt * s.T;
                ar.E += wt * r.E; ar.Fx += wt * r.Fx; ar.Fy += wt * r.Fy; ar.T += wt * r.T;
                if (DELTA) {
                    const Cell4<R> q = get(Lf.w, 2 * ic + a, jf, KIND_STATE);
                    aw.E += wt * q.E; aw.Fx += wt * q.Fx; aw.Fy += wt * q.Fy; aw.T += wt * q.T;
                }
            }
        }
        Lc.v[kc] = av;
        Lc.r[kc] = ar;
        if (DELTA) Lc.w[kc] = aw;
        return;
    }
    for (int b = b0; b <= b1; ++b) {
        const R wy = Lf.dim == 2 ? wgt[b + 1] : R(1);
        const int jf = Lf.dim == 2 ? 2 * jc + b : 0;
        Ghost g[3];
        Cell4<R> s[3], r[3], q[3];
        for (int a = 0; a < 3; ++a) g[a] = ghost_map(Lf, 2 * ic + a - 1, jf);
        for (int a = 0; a < 3; ++a) {
            s[a] = us[g[a].k];
            r[a] = Lf.r[g[a].k];
            if (DELTA) q[a] = Lf.w[g[a].k];
        }
        for (int a = 0; a < 3; ++a) {
            const R wt = wy * wgt[a];
            // correction form: the correction has zero inflow ghosts, the base
            // carries the prescribed state
            const Cell4<R> sv = ghost_apply(Lf, s[a], g[a], DELTA ? KIND_DIFF : KIND_STATE);
            const Cell4<R> rv = ghost_apply(Lf, r[a], g[a], KIND_DIFF);
            av.E += wt * sv.E; av.Fx += wt * sv.Fx; av.Fy += wt * sv.Fy; av.T += wt * sv.T;
            ar.E += wt * rv.E; ar.Fx += wt * rv.Fx; ar.Fy += wt * rv.Fy; ar.T += wt * rv.T;
            if (DELTA) {
                const Cell4<R> qv = ghost_apply(Lf, q[a], g[a], KIND_STATE);
                aw.E += wt * qv.E; aw.Fx += wt * qv.Fx; aw.Fy += wt * qv.Fy; aw.T += wt * qv.T;
            }
        }
    }
    Lc.v[kc] = av;
    Lc.r[kc] = ar;
    if (DELTA) Lc.w[kc] = aw;
}

// Items are (instance, 256-cell chunk of the coarse level).
template <typename R, bool DELTA = false>
__global__ void __launch_bounds__(kThreads) k_restrict(const Level<R>* __restrict__ lvf,
                                                       const Level<R>* __restrict__ lvc,
                                                       WorkList wl, Ctl* __restrict__ ctls,
                                                       int fine_buf)
{
    __shared__ Level<R> Lf, Lc;
    const int w0 = blockIdx.x, ws = gridDim.x;
    int2 nx = item_at(wl, w0);
    const int nw = *wl.count;
    int inst = -1;
    for (int w = w0; w < nw; w += ws, nx = item_at(wl, w)) {
        const int2 it = nx;
        if (skip(ctls, it.x)) continue;
        if (it.x != inst) {                   // descriptors of a new instance
            __syncthreads();
            load_level(Lf, lvf + it.x);
            load_level(Lc, lvc + it.x);
            __syncthreads();
            inst = it.x;
        }
        const int kc = it.y * kThreads + threadIdx.x;
        if (kc < Lc.n) restrict_cell<R, DELTA>(Lf, Lc, kc, fine_buf);
    }
}

template <typename R>
__global__ void k_restrict_sig(const Level<R>* __restrict__ lvf, const Level<R>* __restrict__ lvc,
                               WorkList wl)
{
    __shared__ Level<R> Lf, Lc;
    const int w0 = blockIdx.x, ws = gridDim.x;
    int2 nx = item_at(wl, w0);
    const int nw = *wl.count;
    int inst = -1;
    const R wgt[3] = { R(0.25), R(0.5), R(0.25) };
    for (int w = w0; w < nw; w += ws, nx = item_at(wl, w)) {
        const int2 it = nx;
        if (it.x != inst) {                   // descriptors of a new instance
            __syncthreads();
            load_level(Lf, lvf + it.x);
            load_level(Lc, lvc + it.x);
            __syncthreads();
            inst = it.x;
        }
        const int kc = it.y * kThreads + threadIdx.x;
        if (kc < Lc.n) {
            const int ic = kc % Lc.nx, jc = kc / Lc.nx;
            Sig2<R> acc = { 0, 0 };
            const int b0 = Lf.dim == 2 ? -1 : 0, b1 = Lf.dim == 2 ? 1 : 0;
            for (int b = b0; b <= b1; ++b) {
                const R wy = Lf.dim == 2 ? wgt[b + 1] : R(1);
                const int jf = Lf.dim == 2 ? 2 * jc + b : 0;
                for (int a = -1; a <= 1; ++a) {
                    const Sig2<R> s = fetch_sig(Lf, Lf.sig, 2 * ic + a, jf);
                    acc.sa += wy * wgt[a + 1] * s.sa;
                    acc.ss += wy * wgt[a + 1] * s.ss;
                }
            }
            Lc.sig[kc] = acc;
        }
    }
}

// ---------------------------------------------------------------------------
// u_l += P(u_{l+1} - v_{l+1}) (fine 2i <- coarse i, fine 2i+1 <- half of coarse
// i and i+1; tensor product in 2D); a target outside the admissible set is
// replaced by u + theta_c min(1, tau*) P(e) (Eq. (34)).  One thread takes the
// 2 x 2 (1D: 2) fine cells of coarse cell kc: the differences of the coarse
// cells (ic + a, jc + b), a, b in {0, 1}, are formed once for all of them, and
// each fine cell (2ic + ox, 2jc + oy) sums its weighted differences (a <= ox,
// b <= oy) in the order b, then a, as a thread per fine cell would.
template <typename R, bool DELTA>
__device__ __forceinline__ void prolong_block(const Level<R>& Lc, const Level<R>& Lf, int kc,
                                              int coarse_buf, int fine_buf, Ctl* ctl)
{
    const bool two_d = Lf.dim == 2;
    const int ic = kc % Lc.nx, jc = two_d ? kc / Lc.nx : 0;
    const Cell4<R>* __restrict__ uc = Lc.u[coarse_buf];
    // the coarse cells read lie inside the grid: plain loads
    const bool inside = ic + 1 < Lc.nx && (!two_d || jc + 1 < Lc.ny);
    const int nb = two_d ? 2 : 1;
    Cell4<R> dc[2][2];
    for (int b = 0; b < nb; ++b)
        for (int a = 0; a < 2; ++a) {
            const size_t kk = (size_t)(jc + b) * Lc.nx + ic + a;
            const Cell4<R> cu = inside ? uc[kk] : fetch(Lc, uc, ic + a, jc + b, KIND_DIFF);
            const Cell4<R> cv = inside ? Lc.v[kk] : fetch(Lc, Lc.v, ic + a, jc + b, KIND_DIFF);
            dc[b][a] = Cell4<R>{ cu.E - cv.E, cu.Fx - cv.Fx, cu.Fy - cv.Fy, cu.T - cv.T };
        }
    Cell4<R>* __restrict__ uf = Lf.u[fine_buf];
    for (int oy = 0; oy < nb; ++oy)
        for (int ox = 0; ox < 2; ++ox) {
            const size_t k = (size_t)(2 * jc + oy) * Lf.nx + 2 * ic + ox;
            const R wt = pow2_neg<R>(ox + oy);   // 1, 1/2 or 1/4
            Cell4<R> pe = { 0, 0, 0, 0 };
            for (int b = 0; b <= oy; ++b)
                for (int a = 0; a <= ox; ++a) {
                    pe.E += wt * dc[b][a].E; pe.Fx += wt * dc[b][a].Fx;
                    pe.Fy += wt * dc[b][a].Fy; pe.T += wt * dc[b][a].T;
                }
            const Cell4<R> e = uf[k];
            Cell4<R> u = e;
            if (DELTA) {   // correction form: the admissible set constrains w + e
                const Cell4<R> wb = Lf.w[k];
                u.E += wb.E; u.Fx += wb.Fx; u.Fy += wb.Fy; u.T += wb.T;
            }
            const Cell4<R> tg = { u.E + pe.E, u.Fx + pe.Fx, u.Fy + pe.Fy, u.T + pe.T };
            R th = R(1);
            if (!admissible(tg, Lf.c)) {
                th = (R)ctl->theta_c * fmin(R(1), max_admissible_step(u, pe, Lf.c));
                atomicAdd(&ctl->damped, 1u);
            }
            uf[k] = Cell4<R>{ e.E + th * pe.E, e.Fx + th * pe.Fx, e.Fy + th * pe.Fy,
                              e.T + th * pe.T };
        }
}

// Items are (instance, 256-cell chunk of the coarse level).
template <typename R, bool DELTA = false>
__global__ void __launch_bounds__(kThreads) k_prolong(const Level<R>* __restrict__ lvc,
                                                      const Level<R>* __restrict__ lvf,
                                                      WorkList wl, Ctl* __restrict__ ctls,
                                                      int coarse_buf, int fine_buf)
{
    __shared__ Level<R> Lf, Lc;
    const int w0 = blockIdx.x, ws = gridDim.x;
    int2 nx = item_at(wl, w0);
    const int nw = *wl.count;
    int inst = -1;
    for (int w = w0; w < nw; w += ws, nx = item_at(wl, w)) {
        const int2 it = nx;
        if (skip(ctls, it.x)) continue;
        if (it.x != inst) {                   // descriptors of a new instance
            __syncthreads();
            load_level(Lf, lvf + it.x);
            load_level(Lc, lvc + it.x);
            __syncthreads();
            inst = it.x;
        }
        const int kc = it.y * kThreads + threadIdx.x;
        if (kc < Lc.n) prolong_block<R, DELTA>(Lc, Lf, kc, coarse_buf, fine_buf, ctls + it.x);
    }
}

// ---------------------------------------------------------------------------
// b = (E^n, F^n, C_v T^n) of the iterate in buffer `buf` (Algorithm 4).
template <typename R>
__global__ void k_make_rhs(const Level<R>* __restrict__ lv, WorkList wl,
                           const Ctl* __restrict__ ctls, int buf)
{
    __shared__ Level<R> L;
    const int w0 = blockIdx.x, ws = gridDim.x;
    int2 nx = item_at(wl, w0);
    const int nw = *wl.count;
    int inst = -1;
    for (int w = w0; w < nw; w += ws, nx = item_at(wl, w)) {
        const int2 it = nx;
        if (ctls && !ctls[it.x].active) continue;
        if (it.x != inst) {                   // descriptor of a new instance
            __syncthreads();
            load_level(L, lv + it.x);
            __syncthreads();
            inst = it.x;
        }
        const int k = it.y * kThreads + threadIdx.x;
        if (k < L.n) {
            Cell4<R> s = L.u[buf][k];
            s.T *= L.c_v;
            L.f[k] = s;
        }
    }
}

// Deterministic reduction of one instance's per-strip partials (fixed order:
// thread t sums entries t, t+256, ... then a fixed tree), then the control
// logic of Algorithm 4 for that instance.  One block per instance slot.
__device__ double block_reduce_fixed(const double* __restrict__ p, int n, double* red)
{
    double s = 0.0;
    for (int k = threadIdx.x; k < n; k += blockDim.x) s += p[k];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    double r = red[0];
    __syncthreads();
    return r;
}

__device__ void mark_done(Ctl* ctl, BatchCtl* bctl, int status)
{
    ctl->done = 1;
    ctl->status = status;
    if (bctl) {
        const int n = atomicAdd(&bctl->n_done, 1) + 1;
        if (n >= bctl->n_active) bctl->all_done = 1;
    }
}

template <typename R>
__global__ void __launch_bounds__(kThreads) k_finalize(Ctl* __restrict__ ctls,
                                                       const Level<R>* __restrict__ lv0,
                                                       const double* __restrict__ part,
                                                       const double* __restrict__ partb, int mode,
                                                       int cur, BatchCtl* __restrict__ bctl,
                                                       const int* __restrict__ slot_ids)
{
    __shared__ double red[kThreads];
    const int slot = slot_ids ? slot_ids[blockIdx.x] : (int)blockIdx.x;
    Ctl* ctl = ctls + slot;
    if (!ctl->active) return;
    if (mode != FIN_INIT && ctl->done) return;
    if (mode == FIN_DEFER) {
        const int first = ctl->pending_r0;
        __syncthreads();
        if (first) {
            if (threadIdx.x == 0) ctl->pending_r0 = 0;
            return;
        }
    }
    const Level<R>* L = lv0 + slot;
    const int off = L->part_off, np = L->strips;
    const double s = block_reduce_fixed(part + off, np, red);
    double sb = 0.0;
    if (mode == FIN_INIT) sb = block_reduce_fixed(partb + off, np, red);
    if (threadIdx.x != 0) return;
    const double res = sqrt(s);
    if (mode == FIN_INIT) {
        ctl->res0 = res; ctl->res = res; ctl->res_prev = res;
        ctl->bnorm = sqrt(sb);
        ctl->dtau = ctl->dtau0;
        ctl->kappa = 0;
        if (ctl->hist_len > 0) ctl->hist[0] = res;
        ctl->result_buf = cur;
        ctl->status = CTL_NOT_CONVERGED;
        ctl->pending_r0 = 1;
        ctl->defect_dw = ctl->tol * res > ctl->dw_floor * ctl->bnorm;
        if (res <= ctl->res0_floor * ctl->bnorm) mark_done(ctl, bctl, CTL_OK);
        return;
    }
    const int kappa = ++ctl->kappa;
    ctl->res = res;
    if (kappa < ctl->hist_len) { ctl->hist[kappa] = res; ctl->dtau_hist[kappa - 1] = ctl->dtau; }
    ctl->result_buf = cur;
    if (res <= ctl->tol * ctl->res0) { mark_done(ctl, bctl, CTL_OK); return; }
    const double delta =
        (ctl->dtau_rule ? ctl->res_prev - res : fabs(res - ctl->res_prev)) / ctl->res0;
    double dtau = ctl->dtau;
    if (delta > ctl->eps_i) dtau *= ctl->grow;
    if (delta < ctl->eps_d) dtau *= ctl->shrink;
    dtau = dtau < ctl->dtau_min ? ctl->dtau_min : (dtau > ctl->dtau_max ? ctl->dtau_max : dtau);
    ctl->dtau = dtau;
    ctl->res_prev = res;
    if (kappa >= ctl->max_cycles) mark_done(ctl, bctl, CTL_NOT_CONVERGED);
}

// ---------------------------------------------------------------------------
// Layout conversion: planar FP64 E | Fx | Fy | T (caller's arrays) <-> Cell4<R>.
template <typename R>
__global__ void k_pack_state(const double* __restrict__ E, const double* __restrict__ Fx,
                             const double* __restrict__ Fy, const double* __restrict__ T,
                             double tscale, Cell4<R>* __restrict__ out, int n)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    Cell4<R> c = { (R)E[k], (R)Fx[k], Fy ? (R)Fy[k] : R(0), (R)(T[k] * tscale) };
    out[k] = c;
}

template <typename R>
__global__ void k_unpack_state(const Cell4<R>* __restrict__ in, double* __restrict__ E,
                               double* __restrict__ Fx, double* __restrict__ Fy,
                               double* __restrict__ T, int n)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const Cell4<R> c = in[k];
    E[k] = c.E; Fx[k] = c.Fx;
    if (Fy) Fy[k] = c.Fy;
    T[k] = c.T;
}

template <typename R>
__global__ void k_pack_sig(const double* __restrict__ sa, const double* __restrict__ ss,
                           Sig2<R>* __restrict__ out, int n)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    Sig2<R> s = { (R)sa[k], (R)ss[k] };
    out[k] = s;
}

// Admissibility and finiteness check of an input state: counts bad cells.
template <typename R>
__global__ void k_check_state(const Cell4<R>* __restrict__ s, const Sig2<R>* __restrict__ sig,
                              int n, R c, unsigned int* __restrict__ bad)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const Cell4<R> u = s[k];
    bool ok = isfinite(u.E) && isfinite(u.Fx) && isfinite(u.Fy) && isfinite(u.T) && u.E > R(0) &&
              u.T > R(0) && u.Fx * u.Fx + u.Fy * u.Fy <= c * c * u.E * u.E * (R(1) + Slack<R>::v);
    if (sig) {
        const Sig2<R> g = sig[k];
        ok = ok && isfinite(g.sa) && isfinite(g.ss) && g.sa >= R(0) && g.ss >= R(0);
    }
    if (!ok) atomicAdd(bad, 1u);
}

// The first fine Jacobi sweep of the next FP32 cycle (Algorithm 1 in the
// correction form), formed by the defect kernels beside the cycle's FP32
// problem when `first_sweep` is set: from e = 0 every neighbour term vanishes
// exactly (each closure difference P(w + 0) - P(w) is zero), so the sweep is
// the cell's own local solve with right-hand side g, and its result goes to
// buffer 1, where the cycle's second sweep reads it.  The cycle then launches
// one fine sweep fewer.
__device__ __forceinline__ Cell4<float> first_sweep32(const Level<float>& M, const Cell4<float>& w,
                                                      const Cell4<float>& g, float sa, float ss,
                                                      Ctl* ctl)
{
    const float ka = M.cdt * sa, kt = M.cdt * (sa + ss);
    bool ok;
    const Cell4<float> e = local_solve_delta<float>(0.f, 1.f, M.diag, ka, kt, M.c_v, M.a_r, w.T,
                                                    g.E, g.Fx, g.Fy, g.T, ok);
    if (!ok) atomicAdd(&ctl->newton_fail, 1u);
    return e;
}

// ---------------------------------------------------------------------------
// Mixed precision: FP32 V-cycles in correction form inside FP64 defect
// correction.
//
// k_defect: per fine cell, r64 = b64 - A64(v64) in FP64 (norm partials for the
// stop test), and the FP32 fine problem of the next cycle in correction form:
// base state w = fl32(v64), initial correction e = 0, source g = fl32(r64)
// (the FP32 cycle solves A32(w + e) - A32(w) = r64 for e).
__global__ void __launch_bounds__(kStripWarps * 32) k_defect(const Level<double>* __restrict__ lv64,
                                                             const Level<float>* __restrict__ lv32,
                                                             WorkList wl, Ctl* __restrict__ ctls,
                                                             double* __restrict__ partials,
                                                             int first_sweep)
{
    __shared__ Level<double> Ls[kStripWarps];
    __shared__ Level<float> Ms[kStripWarps];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    Level<double>& L = Ls[wib];
    Level<float>& M = Ms[wib];
    const int w0 = blockIdx.x * kStripWarps + wib, ws = gridDim.x * kStripWarps;
    int2 nx = item_at(wl, w0);
    const int nw = *wl.count;
    for (int w = w0; w < nw; w += ws, nx = item_at(wl, w)) {
        const int2 it = nx;
        // k_defect_dw forms this instance's defect: skip before reading any descriptor
        if (ctls[it.x].defect_dw) continue;
        {
            constexpr int nm = (int)(sizeof(Level<float>) / 8);
            const unsigned long long wm =
                lane < nm ? reinterpret_cast<const unsigned long long*>(lv32 + it.x)[lane] : 0ull;
            if (!enter_item(L, lv64 + it.x, ctls, it.x, lane)) continue;
            if (lane < nm) reinterpret_cast<unsigned long long*>(&M)[lane] = wm;
            __syncwarp();
        }
        const bool two_d = L.dim == 2;
        double nrm = 0.0;
        strip_march<double, false>(L, it, lane, L.u[0], [&](size_t k, const Staged<double>& wv,
                                                             const Staged<double>& ev,
                                                             const Staged<double>& prev,
                                                             const Staged<double>& next,
                                                             const Staged<double>& cur) {
            double NE, NFx, NFy;
            strip_neighbours(L, wv, ev, prev, next, two_d, NE, NFx, NFy);
            const Cell4<double> u = { cur.E, cur.Fx, cur.Fy, cur.T };
            const Sig2<double> sg = L.sig[k];
            const double ka = L.cdt * sg.sa, kt = L.cdt * (sg.sa + sg.ss);
            const double T2 = u.T * u.T, se = ka * (u.E - L.a_r * T2 * T2);
            const Cell4<double> b = L.f[k];
            const double rE = b.E - (L.diag * u.E + se - NE);
            const double rFx = b.Fx - ((L.diag + kt) * u.Fx - NFx);
            const double rFy = b.Fy - ((L.diag + kt) * u.Fy - NFy);
            const double rT = b.T - (L.c_v * u.T - se);
            nrm += rE * rE + (rFx * rFx + rFy * rFy) * L.ic2 + rT * rT;
            const Cell4<float> w32 = { narrow(u.E), narrow(u.Fx), narrow(u.Fy), narrow(u.T) };
            const Cell4<float> g32 = { narrow(rE), narrow(rFx), narrow(rFy), narrow(rT) };
            M.w[k] = w32;
            M.f[k] = g32;
            if (first_sweep)
                M.u[1][k] = first_sweep32(M, w32, g32, narrow(sg.sa), narrow(sg.ss), ctls + it.x);
            else
                M.u[0][k] = Cell4<float>{ 0.f, 0.f, 0.f, 0.f };
        });
        const double sum = warp_sum(nrm);
        if (lane == 0) partials[L.part_off + it.y] = sum * L.vol;
        __syncwarp();
    }
}

// ---------------------------------------------------------------------------
// The defect in double-word FP32 (m1_dw.cuh): the same expressions as the FP64
// residual, each operation on hi + lo pairs of FP32 numbers (about 48 bits).
// The FP64 state, right-hand side and opacities are read and split into double
// words; constants of the level are split once per item.

struct StagedDW {
    DW E, Fx, Fy, Pxx, Pxy, Pyy, T;
};

struct LevelDW {
    DW c, bx, by, diag, a_r, c_v, cdt, m3ic2, q3ic2, third;
};

__device__ __forceinline__ LevelDW level_dw(const Level<double>& L)
{
    return LevelDW{ dw_from(L.c), dw_from(L.bx), dw_from(L.by), dw_from(L.diag), dw_from(L.a_r),
                    dw_from(L.c_v), dw_from(L.cdt), dw_from(-3.0 * L.ic2), dw_from(3.0 * L.ic2),
                    dw_from(1.0 / 3.0) };
}

// The closure of Eq. (5) in the form of closure(): s = sqrt(4 - 3 f^2) (f^2
// clamped to 1), P = (s - 1)/3 E I + 3/(2 + s) F F^T / (c^2 E).
__device__ __forceinline__ StagedDW stage_dw(const LevelDW& D, const DW4& c)
{
    StagedDW o;
    o.E = c.E; o.Fx = c.Fx; o.Fy = c.Fy; o.T = c.T;
    const DW iE = dw_rcp(o.E);
    const DW fx = o.Fx * iE, fy = o.Fy * iE;
    DW a = (fy * fy + fx * fx) * D.m3ic2 + 4.f;
    if (!(a > 1.f)) a = DW{ 1.f, 0.f };
    const DW s = dw_sqrt(a);
    const DW Eiso = o.E * ((s + (-1.f)) * D.third);
    const DW q = dw_rcp(s + 2.f) * D.q3ic2;
    const DW qx = q * fx, qy = q * fy;
    o.Pxx = qx * o.Fx + Eiso;
    o.Pxy = qx * o.Fy;
    o.Pyy = qy * o.Fy + Eiso;
    return o;
}

__device__ __forceinline__ DW shfl_dw(DW v, int from)
{
    return DW{ __shfl_sync(0xffffffffu, v.hi, from), __shfl_sync(0xffffffffu, v.lo, from) };
}

__device__ __forceinline__ StagedDW shfl_staged_dw(const StagedDW& v, int from)
{
    StagedDW o;
    o.E = shfl_dw(v.E, from); o.Fx = shfl_dw(v.Fx, from); o.Fy = shfl_dw(v.Fy, from);
    o.Pxx = shfl_dw(v.Pxx, from); o.Pxy = shfl_dw(v.Pxy, from); o.Pyy = shfl_dw(v.Pyy, from);
    o.T = v.T;
    return o;
}

// r = b - A(u) of one strip cell in double words (Eq. (13) with the [EXT]
// sources), from the staged neighbours, the cell's own state, its right-hand
// side and opacities (double words).
__device__ __forceinline__ void residual_dw(const LevelDW& D, const StagedDW& wv,
                                            const StagedDW& ev, const StagedDW& prev,
                                            const StagedDW& next, const StagedDW& cur, bool two_d,
                                            const DW4& b, const DW2& sg, DW& rE, DW& rFx, DW& rFy,
                                            DW& rT)
{
    const DW cbx = D.c * D.bx;
    DW NE = D.bx * (D.c * (wv.E + ev.E) + (wv.Fx - ev.Fx));
    DW NFx = cbx * ((wv.Fx + ev.Fx) + D.c * (wv.Pxx - ev.Pxx));
    DW NFy = cbx * ((wv.Fy + ev.Fy) + D.c * (wv.Pxy - ev.Pxy));
    if (two_d) {
        const DW cby = D.c * D.by;
        NE = NE + D.by * (D.c * (prev.E + next.E) + (prev.Fy - next.Fy));
        NFx = NFx + cby * ((prev.Fx + next.Fx) + D.c * (prev.Pxy - next.Pxy));
        NFy = NFy + cby * ((prev.Fy + next.Fy) + D.c * (prev.Pyy - next.Pyy));
    }
    const DW ka = D.cdt * sg.sa, dk = D.diag + D.cdt * (sg.sa + sg.ss);
    const DW T2 = cur.T * cur.T;
    const DW se = ka * (cur.E - D.a_r * (T2 * T2));
    rE = b.E - ((D.diag * cur.E + se) - NE);
    rFx = b.Fx - (dk * cur.Fx - NFx);
    rFy = b.Fy - (dk * cur.Fy - NFy);
    rT = b.T - (D.c_v * cur.T - se);
}

// A cell of a double-word state with the ghost rules of fetch(): periodic wrap,
// reflecting mirror with the wall-normal flux negated, Neumann copy, inflow the
// prescribed E, Fx, Fy (split from the FP64 profile) with T from the mirror
// cell; a corner resolves the y wall first, the x wall on top.
__device__ __forceinline__ DW4 fetch_dw(const Level<double>& L, const DW4* __restrict__ s, int i,
                                        int j)
{
    const int jo = j;
    int xrule = -1, xwall = 0, yrule = -1, ywall = 0;
    if (i < 0 || i >= L.nx) {
        xwall = i < 0 ? WALL_W : WALL_E;
        const int bc = L.bc[xwall];
        if (bc == BC_PERIODIC) i = i < 0 ? i + L.nx : i - L.nx;
        else { i = i < 0 ? -1 - i : 2 * L.nx - 1 - i; xrule = bc; }
    }
    if (j < 0 || j >= L.ny) {
        ywall = j < 0 ? WALL_S : WALL_N;
        const int bc = L.bc[ywall];
        if (bc == BC_PERIODIC) j = j < 0 ? j + L.ny : j - L.ny;
        else { j = j < 0 ? -1 - j : 2 * L.ny - 1 - j; yrule = bc; }
    }
    DW4 c = s[(size_t)j * L.nx + i];
    if (yrule == BC_REFLECT) c.Fy = -c.Fy;
    if (yrule == BC_INFLOW) {
        const double* p = L.inflow + (size_t)(ywall * 3) * L.prof_len;
        c.E = dw_from(p[i]); c.Fx = dw_from(p[L.prof_len + i]); c.Fy = dw_from(p[2 * L.prof_len + i]);
    }
    if (xrule == BC_REFLECT) c.Fx = -c.Fx;
    if (xrule == BC_INFLOW) {
        const int jj = jo < 0 ? 0 : (jo >= L.ny ? L.ny - 1 : jo);
        const double* p = L.inflow + (size_t)(xwall * 3) * L.prof_len;
        c.E = dw_from(p[jj]); c.Fx = dw_from(p[L.prof_len + jj]); c.Fy = dw_from(p[2 * L.prof_len + jj]);
    }
    return c;
}

__device__ __forceinline__ DW4 load_dw(const Level<double>& L, const DW4* __restrict__ s, int i,
                                       int j, bool fast)
{
    return fast ? s[(size_t)j * L.nx + i] : fetch_dw(L, s, i, j);
}

// The warp-strip march of strip_march over a double-word state.
template <typename F>
__device__ __forceinline__ void strip_march_dw(const Level<double>& L, const LevelDW& D, int2 it,
                                               int lane, const DW4* __restrict__ src, F&& cell)
{
    const int nx = L.nx, ny = L.ny, two_d = L.dim == 2;
    const int x0 = (it.y % L.sx) * kStripW, y0 = (it.y / L.sx) * L.sh;
    const int i = min(x0 - 1 + lane, nx);
    const bool colfast = x0 >= 1 && x0 + kStripW + 1 <= nx;
    const bool own = lane >= 1 && lane <= kStripW && i < nx;
    const int rows = min(L.sh, ny - y0);
    StagedDW prev{}, cur, next{};
    DW4 rn{};
    if (two_d) {
        prev = stage_dw(D, load_dw(L, src, i, y0 - 1, colfast && y0 >= 1));
        rn = load_dw(L, src, i, y0 + 1, colfast && y0 + 1 < ny);
    }
    cur = stage_dw(D, load_dw(L, src, i, y0, colfast));
    size_t k = (size_t)y0 * nx + i;
    for (int r = 0; r < rows; ++r, k += nx) {
        const int j = y0 + r;
        if (two_d) {
            next = stage_dw(D, rn);
            if (r + 1 < rows) rn = load_dw(L, src, i, j + 2, colfast && j + 2 < ny);
        }
        const StagedDW wv = shfl_staged_dw(cur, (lane + 31) & 31);
        const StagedDW ev = shfl_staged_dw(cur, (lane + 1) & 31);
        if (own) cell(k, wv, ev, prev, next, cur);
        prev = cur;
        cur = next;
    }
}

// Double-word copies of one slot's fine-level iterate, right-hand side and
// opacities (at the start of a step; the FP64 arrays stay the reference).
__global__ void __launch_bounds__(kThreads) k_dw_split(const Level<double>* __restrict__ lv,
                                                       const DwLevel* __restrict__ dwd, WorkList wl)
{
    __shared__ Level<double> L;
    const int w0 = blockIdx.x, ws = gridDim.x;
    int2 nx = item_at(wl, w0);
    const int nw = *wl.count;
    int inst = -1;
    for (int w = w0; w < nw; w += ws, nx = item_at(wl, w)) {
        const int2 it = nx;
        if (it.x != inst) {
            __syncthreads();
            load_level(L, lv + it.x);
            __syncthreads();
            inst = it.x;
        }
        const int k = it.y * kThreads + threadIdx.x;
        if (k < L.n) {
            const DwLevel D = dwd[it.x];
            const Cell4<double> u = L.u[0][k], b = L.f[k];
            const Sig2<double> g = L.sig[k];
            D.v[k] = dw4_from(u.E, u.Fx, u.Fy, u.T);
            D.b[k] = dw4_from(b.E, b.Fx, b.Fy, b.T);
            D.sig[k] = DW2{ dw_split(g.sa), dw_split(g.ss) };
        }
    }
}

// k_defect in double words: the same outputs (norm partials, and the FP32
// problem w = fl32(v), e = 0, g = fl32(r)) for the instances whose control
// block selected it (tol ||r_0|| far above the double-word noise floor).  It
// reads only the double-word copies of the iterate (kept by k_accumulate), the
// right-hand side and the opacities, so no FP64 operation is left per cell;
// the norm is summed in FP32 from the leading words (about 1e-7 relative, far
// inside what the stop test and the dtau_im control resolve).
__global__ void __launch_bounds__(kStripWarps * 32) k_defect_dw(const Level<double>* __restrict__ lv64,
                                                                const Level<float>* __restrict__ lv32,
                                                                const DwLevel* __restrict__ dwd,
                                                                WorkList wl, Ctl* __restrict__ ctls,
                                                                double* __restrict__ partials,
                                                                int first_sweep)
{
    __shared__ Level<double> Ls[kStripWarps];
    __shared__ Level<float> Ms[kStripWarps];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    Level<double>& L = Ls[wib];
    Level<float>& M = Ms[wib];
    const int w0 = blockIdx.x * kStripWarps + wib, ws = gridDim.x * kStripWarps;
    int2 nx = item_at(wl, w0);
    const int nw = *wl.count;
    for (int w = w0; w < nw; w += ws, nx = item_at(wl, w)) {
        const int2 it = nx;
        // k_defect forms this instance's defect: skip before reading any descriptor
        if (!ctls[it.x].defect_dw) continue;
        {
            constexpr int nm = (int)(sizeof(Level<float>) / 8);
            const unsigned long long wm =
                lane < nm ? reinterpret_cast<const unsigned long long*>(lv32 + it.x)[lane] : 0ull;
            if (!enter_item(L, lv64 + it.x, ctls, it.x, lane)) continue;
            if (lane < nm) reinterpret_cast<unsigned long long*>(&M)[lane] = wm;
            __syncwarp();
        }
        const LevelDW D = level_dw(L);
        const DwLevel S = dwd[it.x];
        const bool two_d = L.dim == 2;
        const float ic2 = (float)L.ic2;
        float nrm = 0.f;
        strip_march_dw(L, D, it, lane, S.v, [&](size_t k, const StagedDW& wv, const StagedDW& ev,
                                                 const StagedDW& prev, const StagedDW& next,
                                                 const StagedDW& cur) {
            DW rE, rFx, rFy, rT;
            const DW2 sg = S.sig[k];
            residual_dw(D, wv, ev, prev, next, cur, two_d, S.b[k], sg, rE, rFx, rFy, rT);
            nrm += rE.hi * rE.hi + (rFx.hi * rFx.hi + rFy.hi * rFy.hi) * ic2 + rT.hi * rT.hi;
            const Cell4<float> w32 = { cur.E.hi, cur.Fx.hi, cur.Fy.hi, cur.T.hi };
            const Cell4<float> g32 = { rE.hi, rFx.hi, rFy.hi, rT.hi };
            M.w[k] = w32;
            M.f[k] = g32;
            if (first_sweep)
                M.u[1][k] = first_sweep32(M, w32, g32, sg.sa.hi, sg.ss.hi, ctls + it.x);
            else
                M.u[0][k] = Cell4<float>{ 0.f, 0.f, 0.f, 0.f };
        });
        const double sum = warp_sum((double)nrm);
        if (lane == 0) partials[L.part_off + it.y] = sum * L.vol;
        __syncwarp();
    }
}

// The double-word residual alone, r = b - A(u) written in FP64 (hi + lo) with
// FP64 norm partials: a check of k_defect_dw's arithmetic (m1_op_level).  It
// splits the FP64 state, right-hand side and opacities as it reads them.
__global__ void __launch_bounds__(kStripWarps * 32) k_residual_dw(const Level<double>* __restrict__ lv,
                                                                  WorkList wl, DW4* __restrict__ sv,
                                                                  double* __restrict__ partials)
{
    __shared__ Level<double> Ls[kStripWarps];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    Level<double>& L = Ls[wib];
    const int w0 = blockIdx.x * kStripWarps + wib, ws = gridDim.x * kStripWarps;
    int2 nx = item_at(wl, w0);
    const int nw = *wl.count;
    for (int w = w0; w < nw; w += ws, nx = item_at(wl, w)) {
        const int2 it = nx;
        if (!enter_item(L, lv + it.x, nullptr, it.x, lane)) continue;
        const LevelDW D = level_dw(L);
        const bool two_d = L.dim == 2;
        double nrm = 0.0;
        strip_march_dw(L, D, it, lane, sv, [&](size_t k, const StagedDW& wv, const StagedDW& ev,
                                                const StagedDW& prev, const StagedDW& next,
                                                const StagedDW& cur) {
            const Cell4<double> b = L.f[k];
            const Sig2<double> g = L.sig[k];
            DW rE, rFx, rFy, rT;
            residual_dw(D, wv, ev, prev, next, cur, two_d, dw4_from(b.E, b.Fx, b.Fy, b.T),
                        DW2{ dw_split(g.sa), dw_split(g.ss) }, rE, rFx, rFy, rT);
            const Cell4<double> r = { dw_to_double(rE), dw_to_double(rFx), dw_to_double(rFy),
                                      dw_to_double(rT) };
            L.r[k] = r;
            nrm += r.E * r.E + (r.Fx * r.Fx + r.Fy * r.Fy) * L.ic2 + r.T * r.T;
        });
        const double sum = warp_sum(nrm);
        if (lane == 0 && partials) partials[L.part_off + it.y] = sum * L.vol;
        __syncwarp();
    }
}

// The double-word copy of a level-0 state (for k_residual_dw).
__global__ void k_split_state_dw(const Cell4<double>* __restrict__ u, DW4* __restrict__ out, int n)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n) out[k] = dw4_from(u[k].E, u[k].Fx, u[k].Fy, u[k].T);
}

// k_accumulate: v64 += e in FP64 (e = the FP32 cycle's correction in buffer
// `buf`); a cell whose update leaves the admissible set takes
// v64 + theta_c min(1, tau*) e instead (the damping rule of Eq. (34)).  For an
// instance whose defect is formed in double words, it also writes the
// double-word copy of the new iterate (dwd: per-slot copies, or null).
__global__ void __launch_bounds__(kThreads) k_accumulate(const Level<double>* __restrict__ lv64,
                                                         const Level<float>* __restrict__ lv32,
                                                         const DwLevel* __restrict__ dwd,
                                                         WorkList wl, Ctl* __restrict__ ctls,
                                                         int buf)
{
    __shared__ Level<double> L;
    __shared__ Level<float> M;
    const int w0 = blockIdx.x, ws = gridDim.x;
    int2 nx = item_at(wl, w0);
    const int nw = *wl.count;
    int inst = -1;
    double c2 = 0.0;
    for (int w = w0; w < nw; w += ws, nx = item_at(wl, w)) {
        const int2 it = nx;
        if (skip(ctls, it.x)) continue;
        Ctl* ctl = ctls + it.x;
        if (it.x != inst) {                   // descriptors of a new instance
            __syncthreads();
            load_level(L, lv64 + it.x);
            load_level(M, lv32 + it.x);
            __syncthreads();
            inst = it.x;
            c2 = L.c * L.c;
        }
        const int k = it.y * kThreads + threadIdx.x;
        if (k < L.n) {
            const Cell4<float> a = M.u[buf][k];
            Cell4<double> e = { widen(a.E), widen(a.Fx), widen(a.Fy), widen(a.T) };
            if (!(isfinite(a.E) && isfinite(a.Fx) && isfinite(a.Fy) && isfinite(a.T))) {
                // a correction the FP32 cycle could not form is dropped (counted)
                e.E = e.Fx = e.Fy = e.T = 0.0;
                atomicAdd(&ctl->newton_fail, 1u);
            }
            const Cell4<double> u = L.u[0][k];
            Cell4<double> tg = { u.E + e.E, u.Fx + e.Fx, u.Fy + e.Fy, u.T + e.T };
            if (!admissible_c2(tg, c2)) {
                const double th = ctl->theta_c * fmin(1.0, max_admissible_step(u, e, L.c));
                tg.E = u.E + th * e.E; tg.Fx = u.Fx + th * e.Fx;
                tg.Fy = u.Fy + th * e.Fy; tg.T = u.T + th * e.T;
                atomicAdd(&ctl->damped, 1u);
            }
            L.u[0][k] = tg;
            if (dwd && ctl->defect_dw) dwd[it.x].v[k] = dw4_from(tg.E, tg.Fx, tg.Fy, tg.T);
        }
    }
}

// ---------------------------------------------------------------------------
// Host launchers.
static inline int cdiv(int a, int b) { return (a + b - 1) / b; }
static inline int pgrid(const WorkList& wl)
{
    return wl.capacity < kPersistentBlocks ? (wl.capacity > 0 ? wl.capacity : 1) : kPersistentBlocks;
}

// Blocks of a persistent launch over a list of warp items.
static inline int pgrid_warps(const WorkList& wl)
{
    const int b = (wl.capacity + kStripWarps - 1) / kStripWarps;
    return b < kStripBlocks ? (b > 0 ? b : 1) : kStripBlocks;
}

template <typename R>
void launch_sweep(const Level<R>* lv, WorkList wl, Ctl* ctls, bool pseudo, int in_buf,
                  int out_buf, cudaStream_t s, bool delta, bool ring, double* partials, bool fas)
{
    const int g = pgrid_warps(wl), t = kStripWarps * 32;
    if (fas && pseudo && !delta) {
        k_sweep<R, true, false, false, true><<<g, t, 0, s>>>(lv, wl, ctls, in_buf, out_buf, nullptr);
        return;
    }
    if (partials && !pseudo && !delta) {
        k_sweep<R, false, false, true><<<g, t, 0, s>>>(lv, wl, ctls, in_buf, out_buf, partials);
        return;
    }
    if constexpr (std::is_same<R, float>::value) {
        if (delta && ring) {
            if (pseudo) k_sweep_ring32<true><<<g, t, 0, s>>>(lv, wl, ctls, in_buf, out_buf);
            else k_sweep_ring32<false><<<g, t, 0, s>>>(lv, wl, ctls, in_buf, out_buf);
            return;
        }
    }
    if (delta) {
        if (pseudo) k_sweep<R, true, true><<<g, t, 0, s>>>(lv, wl, ctls, in_buf, out_buf, nullptr);
        else k_sweep<R, false, true><<<g, t, 0, s>>>(lv, wl, ctls, in_buf, out_buf, nullptr);
        return;
    }
    if (pseudo) k_sweep<R, true><<<g, t, 0, s>>>(lv, wl, ctls, in_buf, out_buf, nullptr);
    else k_sweep<R, false><<<g, t, 0, s>>>(lv, wl, ctls, in_buf, out_buf, nullptr);
}

template <typename R>
void launch_apply(const Level<R>* lv, WorkList wl, Ctl* ctls, int mode, int state_buf,
                  double* partials, int write_r, cudaStream_t s, bool delta)
{
    const int g = pgrid_warps(wl), kThreads = kStripWarps * 32;
    if (delta && std::is_same<R, float>::value) {
        if (mode == APPLY_RESID)
            k_apply<R, APPLY_RESID, true><<<g, kThreads, 0, s>>>(lv, wl, ctls, state_buf, partials, write_r);
        else if (mode == APPLY_FAS)
            k_apply<R, APPLY_FAS, true><<<g, kThreads, 0, s>>>(lv, wl, ctls, state_buf, partials, write_r);
        else
            k_apply<R, APPLY_A, true><<<g, kThreads, 0, s>>>(lv, wl, ctls, state_buf, partials, write_r);
        return;
    }
    if (mode == APPLY_RESID)
        k_apply<R, APPLY_RESID><<<g, kThreads, 0, s>>>(lv, wl, ctls, state_buf, partials, write_r);
    else if (mode == APPLY_FAS)
        k_apply<R, APPLY_FAS><<<g, kThreads, 0, s>>>(lv, wl, ctls, state_buf, partials, write_r);
    else
        k_apply<R, APPLY_A><<<g, kThreads, 0, s>>>(lv, wl, ctls, state_buf, partials, write_r);
}

void launch_fas_aw32(const Level<float>* lv, WorkList wl, Ctl* ctls, cudaStream_t s)
{
    k_fas_aw32<<<pgrid_warps(wl), kStripWarps * 32, 0, s>>>(lv, wl, ctls);
}

template <typename R>
void launch_norm_state(const Level<R>* lv, WorkList wl, const Ctl* ctls, double* partials,
                       cudaStream_t s)
{
    k_norm_state<R><<<pgrid_warps(wl), kStripWarps * 32, 0, s>>>(lv, wl, ctls, partials);
}

template <typename R>
void launch_restrict(const Level<R>* lvf, const Level<R>* lvc, WorkList wl, Ctl* ctls,
                     int fine_buf, cudaStream_t s, bool delta)
{
    if (delta && std::is_same<R, float>::value)
        k_restrict<R, true><<<pgrid(wl), kThreads, 0, s>>>(lvf, lvc, wl, ctls, fine_buf);
    else
        k_restrict<R><<<pgrid(wl), kThreads, 0, s>>>(lvf, lvc, wl, ctls, fine_buf);
}

template <typename R>
void launch_restrict_sig(const Level<R>* lvf, const Level<R>* lvc, WorkList wl, cudaStream_t s)
{
    k_restrict_sig<R><<<pgrid(wl), kThreads, 0, s>>>(lvf, lvc, wl);
}

template <typename R>
void launch_prolong(const Level<R>* lvc, const Level<R>* lvf, WorkList wl, Ctl* ctls,
                    int coarse_buf, int fine_buf, cudaStream_t s, bool delta)
{
    if (delta && std::is_same<R, float>::value)
        k_prolong<R, true><<<pgrid(wl), kThreads, 0, s>>>(lvc, lvf, wl, ctls, coarse_buf, fine_buf);
    else
        k_prolong<R><<<pgrid(wl), kThreads, 0, s>>>(lvc, lvf, wl, ctls, coarse_buf, fine_buf);
}

template <typename R>
void launch_make_rhs(const Level<R>* lv, WorkList wl, const Ctl* ctls, int buf, cudaStream_t s)
{
    k_make_rhs<R><<<pgrid(wl), kThreads, 0, s>>>(lv, wl, ctls, buf);
}

template <typename R>
void launch_finalize(Ctl* ctls, const Level<R>* lv0, int nslots, const double* part,
                     const double* partb, int mode, int cur, BatchCtl* bctl, cudaStream_t s,
                     const int* slot_ids)
{
    if (nslots > 0)
        k_finalize<R><<<nslots, kThreads, 0, s>>>(ctls, lv0, part, partb, mode, cur, bctl, slot_ids);
}

template <typename R>
void launch_pack_state(const double* E, const double* Fx, const double* Fy, const double* T,
                       double tscale, Cell4<R>* out, int n, cudaStream_t s)
{
    k_pack_state<R><<<cdiv(n, kThreads), kThreads, 0, s>>>(E, Fx, Fy, T, tscale, out, n);
}

template <typename R>
void launch_unpack_state(const Cell4<R>* in, double* E, double* Fx, double* Fy, double* T, int n,
                         cudaStream_t s)
{
    k_unpack_state<R><<<cdiv(n, kThreads), kThreads, 0, s>>>(in, E, Fx, Fy, T, n);
}

template <typename R>
void launch_pack_sig(const double* sa, const double* ss, Sig2<R>* out, int n, cudaStream_t s)
{
    k_pack_sig<R><<<cdiv(n, kThreads), kThreads, 0, s>>>(sa, ss, out, n);
}

template <typename R>
void launch_check_state(const Cell4<R>* st, const Sig2<R>* sig, int n, double c, unsigned int* bad,
                        cudaStream_t s)
{
    k_check_state<R><<<cdiv(n, kThreads), kThreads, 0, s>>>(st, sig, n, (R)c, bad);
}

void launch_defect(const Level<double>* lv64, const Level<float>* lv32, WorkList wl, Ctl* ctls,
                   double* partials, cudaStream_t s, bool first_sweep)
{
    k_defect<<<pgrid_warps(wl), kStripWarps * 32, 0, s>>>(lv64, lv32, wl, ctls, partials,
                                                          first_sweep ? 1 : 0);
}

void launch_defect_dw(const Level<double>* lv64, const Level<float>* lv32, const DwLevel* dwd,
                      WorkList wl, Ctl* ctls, double* partials, cudaStream_t s, bool first_sweep)
{
    k_defect_dw<<<pgrid_warps(wl), kStripWarps * 32, 0, s>>>(lv64, lv32, dwd, wl, ctls, partials,
                                                             first_sweep ? 1 : 0);
}

void launch_dw_split(const Level<double>* lv, const DwLevel* dwd, WorkList wl, cudaStream_t s)
{
    k_dw_split<<<pgrid(wl), kThreads, 0, s>>>(lv, dwd, wl);
}

void launch_residual_dw(const Level<double>* lv, const Cell4<double>* u, DW4* scratch, int n,
                        WorkList wl, double* partials, cudaStream_t s)
{
    k_split_state_dw<<<cdiv(n, kThreads), kThreads, 0, s>>>(u, scratch, n);
    k_residual_dw<<<pgrid_warps(wl), kStripWarps * 32, 0, s>>>(lv, wl, scratch, partials);
}

void launch_accumulate(const Level<double>* lv64, const Level<float>* lv32, WorkList wl,
                       Ctl* ctls, int buf, cudaStream_t s, const DwLevel* dwd)
{
    k_accumulate<<<pgrid(wl), kThreads, 0, s>>>(lv64, lv32, dwd, wl, ctls, buf);
}

#define M1_INSTANTIATE(R)                                                                          \
    template void launch_sweep<R>(const Level<R>*, WorkList, Ctl*, bool, int, int, cudaStream_t,  \
                                  bool, bool, double*, bool);                                      \
    template void launch_apply<R>(const Level<R>*, WorkList, Ctl*, int, int, double*, int,        \
                                  cudaStream_t, bool);                                             \
    template void launch_norm_state<R>(const Level<R>*, WorkList, const Ctl*, double*,            \
                                       cudaStream_t);                                              \
    template void launch_restrict<R>(const Level<R>*, const Level<R>*, WorkList, Ctl*, int,       \
                                     cudaStream_t, bool);                                          \
    template void launch_restrict_sig<R>(const Level<R>*, const Level<R>*, WorkList,              \
                                         cudaStream_t);                                            \
    template void launch_prolong<R>(const Level<R>*, const Level<R>*, WorkList, Ctl*, int, int,   \
                                    cudaStream_t, bool);                                           \
    template void launch_make_rhs<R>(const Level<R>*, WorkList, const Ctl*, int, cudaStream_t);   \
    template void launch_finalize<R>(Ctl*, const Level<R>*, int, const double*, const double*,    \
                                     int, int, BatchCtl*, cudaStream_t, const int*);               \
    template void launch_pack_state<R>(const double*, const double*, const double*, const double*,\
                                       double, Cell4<R>*, int, cudaStream_t);                      \
    template void launch_unpack_state<R>(const Cell4<R>*, double*, double*, double*, double*, int,\
                                         cudaStream_t);                                            \
    template void launch_pack_sig<R>(const double*, const double*, Sig2<R>*, int, cudaStream_t);  \
    template void launch_check_state<R>(const Cell4<R>*, const Sig2<R>*, int, double,             \
                                        unsigned int*, cudaStream_t);

M1_INSTANTIATE(double)
M1_INSTANTIATE(float)

}  // namespace m1
