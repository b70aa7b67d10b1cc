/*
 * m1_oracle3d.c -- plain, slow, FP64 CPU oracle for one implicit time step of the
 * M1 moment model in three dimensions, solved by the nonlinear FAS multigrid of
 * Bloch, Tremblin, Gonzalez & Audit, "Towards a multigrid method for the M1 model
 * for radiative transfer" (arXiv:2208.14703).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call, link or load
 * this file: only the tests use it.  It shares no code, header, table or constant
 * generator with the CUDA implementation, nor with the 1D/2D oracle beside it.
 *
 * The paper's experiments are 1D and 2D; its restriction and prolongation are
 * written for d in {1, 2, 3} (Section 4.2, R = 2^-d P^T) and Section 6.3 expects a
 * larger gain in 3D.  This file extends the 2D reading axis by axis: the Rusanov
 * face flux of Eq. (6) on all three axes, the 3x3 pressure tensor of Eq. (5), the
 * tensor-product transfers of Eqs. (14)/(21) on three axes.  Walls are periodic,
 * reflecting (mirror, wall-normal flux negated), Neumann (copy) or inflow (the
 * prescribed E, F of the wall's face profile, T copied; differences see zero
 * there), as in 2D; coarse face profiles are the 1D full-weighting rule of the
 * 2D oracle applied along both tangential axes.  Every other reading (sources,
 * local solve, pseudo-time smoother, damping, norm, dtau control, levels) is the
 * one of the 2D oracle, marked [READING] or [EXT] where it applies.
 *
 * Data layout: a state is 5 planes [E | Fx | Fy | Fz | T], each nz*ny*nx doubles,
 * index (k*ny + j)*nx + i.  Inflow profiles: [6 walls][E, Fx, Fy, Fz][F] with
 * F = the largest face (max of ny*nz, nx*nz, nx*ny); the face of a wall on axis d
 * is indexed q_b * n_a + q_a over its two other axes a < b.
 *
 * Threads: as in the 2D oracle, the outer cell loops carry OpenMP pragmas that
 * the plain build ignores; the all-core build (-fopenmp) gives bit-for-bit the
 * same results (integer reductions only, the norm summed serially).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* Host threads the cell loops run on: 1 in the plain build. */
int ora3_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

enum { BC_PERIODIC = 0, BC_REFLECT = 1, BC_NEUMANN = 2, BC_INFLOW = 3 };
enum { KIND_STATE = 0, KIND_DIFF = 1 };
/* walls: 0 W (x low), 1 E (x high), 2 S (y low), 3 N (y high), 4 B (z low), 5 T (z high) */

#define NF 5                       /* fields per cell */
#define ADM_SLACK 1e-12            /* as in the 2D oracle's damping decision [READING] */

typedef struct {
    int n[3];                      /* nx, ny, nz */
    double h[3];                   /* hx, hy, hz */
    double c, a_r, c_v;
    int bc[6];
    const double* in[6];           /* inflow face profile of each wall (4 fields), or NULL */
    size_t fstride;                /* doubles per field of a profile: the largest face */
} grid3_t;

typedef struct { double E, F[3], T; } cell5_t;

static double sq(double x) { return x * x; }
static double dmin(double a, double b) { return a < b ? a : b; }

static size_t ncell(const grid3_t* g) { return (size_t)g->n[0] * g->n[1] * g->n[2]; }

static size_t idx(const grid3_t* g, int i, int j, int k)
{
    return ((size_t)k * g->n[1] + j) * g->n[0] + i;
}

static size_t face_max(const int n[3])
{
    size_t a = (size_t)n[1] * n[2], b = (size_t)n[0] * n[2], c = (size_t)n[0] * n[1];
    size_t m = a > b ? a : b;
    return m > c ? m : c;
}

static void set_inflow(grid3_t* g, const double* inflow)
{
    g->fstride = face_max(g->n);
    for (int w = 0; w < 6; ++w)
        g->in[w] = (inflow && g->bc[w] == BC_INFLOW) ? inflow + (size_t)w * 4 * g->fstride : NULL;
}

static void grid_from_desc(grid3_t* g, const int* idesc, const double* ddesc, const double* inflow)
{
    /* idesc = { nx, ny, nz, bc[6] }; ddesc = { hx, hy, hz, c, a_r, c_v } */
    for (int a = 0; a < 3; ++a) { g->n[a] = idesc[a]; g->h[a] = ddesc[a]; }
    for (int w = 0; w < 6; ++w) g->bc[w] = idesc[3 + w];
    g->c = ddesc[3]; g->a_r = ddesc[4]; g->c_v = ddesc[5];
    set_inflow(g, inflow);
}

/* The two axes tangential to a wall on axis d, in increasing order. */
static void tangential(int d, int* a, int* b)
{
    *a = d == 0 ? 1 : 0;
    *b = d == 2 ? 1 : 2;
}

static cell5_t load(const grid3_t* g, const double* v, int i, int j, int k)
{
    size_t n = ncell(g), q = idx(g, i, j, k);
    cell5_t s = { v[q], { v[n + q], v[2 * n + q], v[3 * n + q] }, v[4 * n + q] };
    return s;
}

static void store(const grid3_t* g, double* v, int i, int j, int k, cell5_t s)
{
    size_t n = ncell(g), q = idx(g, i, j, k);
    v[q] = s.E; v[n + q] = s.F[0]; v[2 * n + q] = s.F[1]; v[3 * n + q] = s.F[2]; v[4 * n + q] = s.T;
}

/* ------------------------------------------------------------------------ */
/* Section 2.1, Eq. (5) in 3D: chi = (3 + 4 f^2) / (5 + 2 sqrt(4 - 3 f^2)),
 * n = F/|F|, P = ((1 - chi)/2 I + (3 chi - 1)/2 n (x) n) E.  P is returned as
 * P[a][b], a, b in {x, y, z}.  f is clamped to 1. */
void ora3_closure(double E, const double* F, double c, double* P)
{
    double normF = sqrt(F[0] * F[0] + F[1] * F[1] + F[2] * F[2]);
    double f = normF / (c * E);
    if (f > 1.0) f = 1.0;
    double chi = (3.0 + 4.0 * f * f) / (5.0 + 2.0 * sqrt(4.0 - 3.0 * f * f));
    double nv[3] = { 0.0, 0.0, 0.0 };
    if (normF > 0.0)
        for (int a = 0; a < 3; ++a) nv[a] = F[a] / normF;
    double iso = 0.5 * (1.0 - chi), dir = 0.5 * (3.0 * chi - 1.0);
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) P[3 * a + b] = ((a == b ? iso : 0.0) + dir * nv[a] * nv[b]) * E;
}

/* ------------------------------------------------------------------------ */
/* Ghost cells, one layer per wall [READING]: periodic wrap, reflecting = mirror
 * cell with the wall-normal flux component negated, Neumann = copy, inflow = the
 * prescribed E, F of the face profile at the (clamped) tangential position with
 * T copied from the mirror cell; differences (kind DIFF) see zero at an inflow
 * wall.  Corners and edges resolve one axis after the other. */
static cell5_t get_cell(const grid3_t* g, const double* v, int p[3], int kind)
{
    for (int a = 0; a < 3; ++a) {
        if (p[a] >= 0 && p[a] < g->n[a]) continue;
        int wall = 2 * a + (p[a] < 0 ? 0 : 1);
        int q[3] = { p[0], p[1], p[2] };
        if (g->bc[wall] == BC_PERIODIC) {
            q[a] = p[a] < 0 ? p[a] + g->n[a] : p[a] - g->n[a];
            return get_cell(g, v, q, kind);
        }
        q[a] = p[a] < 0 ? -1 - p[a] : 2 * g->n[a] - 1 - p[a];
        cell5_t m = get_cell(g, v, q, kind);
        if (g->bc[wall] == BC_REFLECT) { m.F[a] = -m.F[a]; return m; }
        if (g->bc[wall] == BC_NEUMANN) return m;
        if (kind == KIND_DIFF) {
            m.E = m.F[0] = m.F[1] = m.F[2] = m.T = 0.0;
            return m;
        }
        int ta, tb;
        tangential(a, &ta, &tb);
        int ia = p[ta] < 0 ? 0 : (p[ta] >= g->n[ta] ? g->n[ta] - 1 : p[ta]);
        int ib = p[tb] < 0 ? 0 : (p[tb] >= g->n[tb] ? g->n[tb] - 1 : p[tb]);
        size_t f = (size_t)ib * g->n[ta] + ia;
        const double* prof = g->in[wall];
        m.E = prof[f];
        for (int c = 0; c < 3; ++c) m.F[c] = prof[(size_t)(1 + c) * g->fstride + f];
        return m;
    }
    return load(g, v, p[0], p[1], p[2]);
}

static double get_scalar(const grid3_t* g, const double* s, int p[3])
{
    int q[3] = { p[0], p[1], p[2] };
    for (int a = 0; a < 3; ++a) {
        if (q[a] >= 0 && q[a] < g->n[a]) continue;
        int wall = 2 * a + (q[a] < 0 ? 0 : 1);
        if (g->bc[wall] == BC_PERIODIC) q[a] = q[a] < 0 ? q[a] + g->n[a] : q[a] - g->n[a];
        else q[a] = q[a] < 0 ? -1 - q[a] : 2 * g->n[a] - 1 - q[a];
    }
    return s[idx(g, q[0], q[1], q[2])];
}

/* ------------------------------------------------------------------------ */
/* Section 3.1, Eq. (9) on axis d: the neighbour operator of the implicit Rusanov
 * scheme evaluated on one neighbour state; sign = +1 for the low-side neighbour
 * (L), -1 for the high-side one (R).  beta = dt / (2 h_d). */
static void neighbour_term(const grid3_t* g, double dt, int d, double sign, cell5_t nb,
                           double out[4])
{
    double beta = dt / (2.0 * g->h[d]), c = g->c, P[9];
    ora3_closure(nb.E, nb.F, c, P);
    out[0] = beta * (c * nb.E + sign * nb.F[d]);
    for (int a = 0; a < 3; ++a) out[1 + a] = c * beta * (nb.F[a] + sign * c * P[3 * d + a]);
}

/* Sum of the L and R terms of the six neighbours of cell (i, j, k), Eq. (10). */
static void neighbour_sum(const grid3_t* g, double dt, const double* v, int i, int j, int k,
                          double s[4])
{
    s[0] = s[1] = s[2] = s[3] = 0.0;
    for (int d = 0; d < 3; ++d)
        for (int side = -1; side <= 1; side += 2) {
            int p[3] = { i, j, k };
            p[d] += side;
            double t[4];
            neighbour_term(g, dt, d, side < 0 ? +1.0 : -1.0, get_cell(g, v, p, KIND_STATE), t);
            for (int q = 0; q < 4; ++q) s[q] += t[q];
        }
}

/* Transport diagonal 1 + c dt (1/hx + 1/hy + 1/hz), Eq. (9) on three axes. */
static double transport_diag(const grid3_t* g, double dt)
{
    return 1.0 + g->c * dt / g->h[0] + g->c * dt / g->h[1] + g->c * dt / g->h[2];
}

/* Eq. (12): A(v)_i = D(v_i) - sum of the neighbour terms, with the [EXT]
 * backward-Euler sources of the 2D oracle (k_a = c dt sigma_a, k_t = c dt
 * (sigma_a + sigma_s), gas row C_v T - k_a (E - a_r T^4)). */
static cell5_t apply_A_cell(const grid3_t* g, double dt, const double* sa, const double* ss,
                            const double* v, int i, int j, int k)
{
    size_t q = idx(g, i, j, k);
    cell5_t u = load(g, v, i, j, k), out;
    double diag = transport_diag(g, dt);
    double ka = g->c * dt * sa[q], kt = g->c * dt * (sa[q] + ss[q]);
    double src = ka * (u.E - g->a_r * sq(sq(u.T)));
    double s[4];
    neighbour_sum(g, dt, v, i, j, k, s);
    out.E = diag * u.E + src - s[0];
    for (int a = 0; a < 3; ++a) out.F[a] = (diag + kt) * u.F[a] - s[1 + a];
    out.T = g->c_v * u.T - src;
    return out;
}

void ora3_apply_A(const int* idesc, const double* ddesc, const double* inflow, double dt,
                  const double* sa, const double* ss, const double* v, double* out)
{
    grid3_t g; grid_from_desc(&g, idesc, ddesc, inflow);
    #pragma omp parallel for collapse(3) schedule(static)
    for (int k = 0; k < g.n[2]; ++k)
        for (int j = 0; j < g.n[1]; ++j)
            for (int i = 0; i < g.n[0]; ++i)
                store(&g, out, i, j, k, apply_A_cell(&g, dt, sa, ss, v, i, j, k));
}

static void residual(const grid3_t* g, double dt, const double* sa, const double* ss,
                     const double* b, const double* v, double* r)
{
    size_t n = ncell(g);
    #pragma omp parallel for collapse(3) schedule(static)
    for (int k = 0; k < g->n[2]; ++k)
        for (int j = 0; j < g->n[1]; ++j)
            for (int i = 0; i < g->n[0]; ++i) {
                size_t q = idx(g, i, j, k);
                cell5_t a = apply_A_cell(g, dt, sa, ss, v, i, j, k);
                r[q] = b[q] - a.E;
                for (int c = 0; c < 3; ++c) r[(1 + c) * n + q] = b[(1 + c) * n + q] - a.F[c];
                r[4 * n + q] = b[4 * n + q] - a.T;
            }
}

/* Eq. (13): r = b - A(v). */
void ora3_residual(const int* idesc, const double* ddesc, const double* inflow, double dt,
                   const double* sa, const double* ss, const double* b, const double* v, double* r)
{
    grid3_t g; grid_from_desc(&g, idesc, ddesc, inflow);
    residual(&g, dt, sa, ss, b, v, r);
}

/* [READING] ||r||^2 = sum over cells of h^3 (rE^2 + |rF|^2 / c^2 + rT^2). */
static double norm(const grid3_t* g, const double* r)
{
    size_t n = ncell(g);
    double vol = g->h[0] * g->h[1] * g->h[2], s = 0.0;
    for (size_t q = 0; q < n; ++q)
        s += vol * (sq(r[q]) + (sq(r[n + q]) + sq(r[2 * n + q]) + sq(r[3 * n + q])) / sq(g->c) +
                    sq(r[4 * n + q]));
    return sqrt(s);
}

double ora3_norm(const int* idesc, const double* ddesc, const double* r)
{
    grid3_t g; grid_from_desc(&g, idesc, ddesc, NULL);
    return norm(&g, r);
}

/* ------------------------------------------------------------------------ */
/* [EXT] D^{-1} of one cell, as in the 2D oracle with three flux components:
 *   (w0 + w1 diag) E + w1 k_a (E - a_r T^4) = bE,  (w0 + w1 (diag + k_t)) F = bF,
 *   (w0 + w1 C_v) T - w1 k_a (E - a_r T^4) = bT;
 * E eliminated, g(T) = C T + K T^4 - R solved by Newton from
 * T0 = min(R/C, (R/K)^(1/4)).  Returns the iteration count, -1 if it failed. */
static int local_solve(double w0, double w1, double diag, double ka, double kt, double c_v,
                       double a_r, const double beta[5], double out[5])
{
    double A = w0 + w1 * diag, k = w1 * ka;
    double Fden = w0 + w1 * (diag + kt);
    for (int a = 0; a < 3; ++a) out[1 + a] = beta[1 + a] / Fden;
    double C = w0 + w1 * c_v;
    double K = k * A * a_r / (A + k);
    double R = beta[4] + k * beta[0] / (A + k);
    double T;
    int it = 0, ok = 1;
    if (K == 0.0) {
        T = R / C;
    } else {
        T = dmin(R / C, pow(R / K, 0.25));
        ok = 0;
        for (it = 1; it <= 60; ++it) {
            double gT = C * T + K * sq(sq(T)) - R;
            double dg = C + 4.0 * K * T * T * T;
            double dT = gT / dg;
            T -= dT;
            if (fabs(dT) <= 1e-15 * T) { ok = 1; break; }
        }
    }
    out[4] = T;
    out[0] = (beta[0] + k * a_r * sq(sq(T))) / (A + k);
    return ok ? it : -1;
}

/* Algorithm 1, one pure Jacobi sweep of Eq. (10) with weights (w0, w1). */
static int jacobi_sweep(const grid3_t* g, double dt, const double* sa, const double* ss,
                        const double* rhs, const double* vin, double* vout, double w0, double w1)
{
    double diag = transport_diag(g, dt);
    int fail = 0, maxit = 0;
    #pragma omp parallel for collapse(3) schedule(static) reduction(|:fail) reduction(max:maxit)
    for (int k = 0; k < g->n[2]; ++k)
        for (int j = 0; j < g->n[1]; ++j)
            for (int i = 0; i < g->n[0]; ++i) {
                size_t q = idx(g, i, j, k);
                double s[4], beta[5], out[5];
                cell5_t b = load(g, rhs, i, j, k);
                neighbour_sum(g, dt, vin, i, j, k, s);
                beta[0] = b.E + w1 * s[0];
                for (int a = 0; a < 3; ++a) beta[1 + a] = b.F[a] + w1 * s[1 + a];
                beta[4] = b.T;
                int it = local_solve(w0, w1, diag, g->c * dt * sa[q], g->c * dt * (sa[q] + ss[q]),
                                     g->c_v, g->a_r, beta, out);
                if (it < 0) fail = 1; else if (it > maxit) maxit = it;
                cell5_t o = { out[0], { out[1], out[2], out[3] }, out[4] };
                store(g, vout, i, j, k, o);
            }
    return fail ? -1 : maxit;
}

int ora3_jacobi_sweep(const int* idesc, const double* ddesc, const double* inflow, double dt,
                      const double* sa, const double* ss, const double* rhs, const double* vin,
                      double* vout, double w0, double w1)
{
    grid3_t g; grid_from_desc(&g, idesc, ddesc, inflow);
    return jacobi_sweep(&g, dt, sa, ss, rhs, vin, vout, w0, w1);
}

/* ------------------------------------------------------------------------ */
/* Admissible set, Eq. (7) (+ [EXT] T > 0): the largest tau >= 0 with u + tau d
 * admissible: E, T bounds and the first positive root of
 * |F + tau dF|^2 = c^2 (E + tau dE)^2 [READING, as in 2D]. */
static double max_admissible_step(cell5_t u, cell5_t d, double c)
{
    double tau = INFINITY;
    if (d.E < 0.0) tau = dmin(tau, -u.E / d.E);
    if (d.T < 0.0) tau = dmin(tau, -u.T / d.T);
    double a = -c * c * d.E * d.E, b = -c * c * u.E * d.E, c0 = -c * c * u.E * u.E;
    for (int q = 0; q < 3; ++q) {
        a += d.F[q] * d.F[q];
        b += u.F[q] * d.F[q];
        c0 += u.F[q] * u.F[q];
    }
    if (c0 > 0.0) c0 = 0.0;
    double disc = b * b - a * c0, t = INFINITY;
    if (a > 0.0) {
        t = b <= 0.0 ? (-b + sqrt(disc)) / a : -c0 / (b + sqrt(disc));
    } else if (a < 0.0) {
        if (b > 0.0 && disc >= 0.0) t = -c0 / (b + sqrt(disc));
    } else {
        if (b > 0.0) t = -c0 / (2.0 * b);
    }
    return dmin(tau, t);
}

static int admissible(cell5_t s, double c)
{
    return s.E > 0.0 && s.T > 0.0 &&
           sq(s.F[0]) + sq(s.F[1]) + sq(s.F[2]) <= c * c * s.E * s.E * (1.0 + ADM_SLACK);
}

/* Algorithm 3: m pseudo-time steps, each the explicit half of Eq. (30) with the
 * limited step tau_i = min(dtau, theta tau*_i) [READING] and nu Jacobi sweeps of
 * u + dtau A(u) = u~ from u^m. */
static int pseudo_time_smooth(const grid3_t* g, double dt, const double* sa, const double* ss,
                              const double* f, double* u, double dtau, int m, int nu, double theta)
{
    size_t n = ncell(g);
    double* ut = malloc(NF * n * sizeof(double));
    double* w = malloc(NF * n * sizeof(double));
    double* w2 = malloc(NF * n * sizeof(double));
    int worst = 0;
    for (int it = 0; it < m; ++it) {
        #pragma omp parallel for collapse(3) schedule(static)
        for (int k = 0; k < g->n[2]; ++k)
            for (int j = 0; j < g->n[1]; ++j)
                for (int i = 0; i < g->n[0]; ++i) {
                    cell5_t s = load(g, u, i, j, k), d = load(g, f, i, j, k), o;
                    double tau = dmin(dtau, theta * max_admissible_step(s, d, g->c));
                    o.E = s.E + tau * d.E;
                    for (int a = 0; a < 3; ++a) o.F[a] = s.F[a] + tau * d.F[a];
                    o.T = s.T + tau * d.T;
                    store(g, ut, i, j, k, o);
                }
        memcpy(w, u, NF * n * sizeof(double));
        for (int s = 0; s < nu; ++s) {
            if (jacobi_sweep(g, dt, sa, ss, ut, w, w2, 1.0, dtau) < 0) worst = -1;
            memcpy(w, w2, NF * n * sizeof(double));
        }
        memcpy(u, w, NF * n * sizeof(double));
    }
    free(ut); free(w); free(w2);
    return worst;
}

int ora3_pseudo_time_smooth(const int* idesc, const double* ddesc, const double* inflow, double dt,
                            const double* sa, const double* ss, const double* f, double* u,
                            double dtau, int m, int nu, double theta)
{
    grid3_t g; grid_from_desc(&g, idesc, ddesc, inflow);
    return pseudo_time_smooth(&g, dt, sa, ss, f, u, dtau, m, nu, theta);
}

/* ------------------------------------------------------------------------ */
/* Section 4.2, Eq. (21) on three axes: R = 2^-3 P^T, weights 1/4, 1/2, 1/4 per
 * axis (27 fine cells, tensor product); fine ghosts by the wall rules. */
static void coarse_desc(const grid3_t* gf, grid3_t* gc)
{
    *gc = *gf;
    for (int a = 0; a < 3; ++a) { gc->n[a] = gf->n[a] / 2; gc->h[a] = 2.0 * gf->h[a]; }
    set_inflow(gc, NULL);          /* a coarse grid's profiles come from restrict_faces */
}

/* The 2D oracle's 1D profile rule, 1/4, 1/2, 1/4 with the ends copied, along one
 * tangential axis of a face. */
static double profile_weighted(const double* f, int nf, int i, int stride)
{
    int a = 2 * i - 1 < 0 ? 0 : 2 * i - 1, b = 2 * i, c = 2 * i + 1 >= nf ? nf - 1 : 2 * i + 1;
    return 0.25 * f[(size_t)a * stride] + 0.5 * f[(size_t)b * stride] + 0.25 * f[(size_t)c * stride];
}

/* Coarse face profiles of every inflow wall: the 1D rule along each tangential
 * axis (a tensor product).  out: [6][4][face_max(gc)]. */
static void restrict_faces(const grid3_t* gf, const grid3_t* gc, double* out)
{
    for (int w = 0; w < 6; ++w) {
        if (gf->bc[w] != BC_INFLOW || !gf->in[w]) continue;
        int d = w / 2, ta, tb;
        tangential(d, &ta, &tb);
        int nfa = gf->n[ta], nfb = gf->n[tb], nca = gc->n[ta], ncb = gc->n[tb];
        double* tmp = malloc((size_t)nca * nfb * sizeof(double));
        for (int fld = 0; fld < 4; ++fld) {
            const double* f = gf->in[w] + (size_t)fld * gf->fstride;
            double* o = out + ((size_t)w * 4 + fld) * gc->fstride;
            for (int ib = 0; ib < nfb; ++ib)             /* along a */
                for (int ia = 0; ia < nca; ++ia)
                    tmp[(size_t)ib * nca + ia] = nca == nfa ? f[(size_t)ib * nfa + ia]
                                                            : profile_weighted(f + (size_t)ib * nfa, nfa, ia, 1);
            for (int ib = 0; ib < ncb; ++ib)             /* along b */
                for (int ia = 0; ia < nca; ++ia)
                    o[(size_t)ib * nca + ia] = ncb == nfb ? tmp[(size_t)ib * nca + ia]
                                                          : profile_weighted(tmp + ia, nfb, ib, nca);
        }
        free(tmp);
    }
}

static void restrict_state(const grid3_t* gf, const grid3_t* gc, const double* fine, double* coarse,
                           int kind)
{
    static const double w[3] = { 0.25, 0.5, 0.25 };
    #pragma omp parallel for collapse(3) schedule(static)
    for (int kc = 0; kc < gc->n[2]; ++kc)
        for (int jc = 0; jc < gc->n[1]; ++jc)
            for (int ic = 0; ic < gc->n[0]; ++ic) {
                cell5_t acc = { 0.0, { 0.0, 0.0, 0.0 }, 0.0 };
                for (int cz = -1; cz <= 1; ++cz)
                    for (int by = -1; by <= 1; ++by)
                        for (int ax = -1; ax <= 1; ++ax) {
                            double wt = w[ax + 1] * w[by + 1] * w[cz + 1];
                            int p[3] = { 2 * ic + ax, 2 * jc + by, 2 * kc + cz };
                            cell5_t s = get_cell(gf, fine, p, kind);
                            acc.E += wt * s.E;
                            for (int a = 0; a < 3; ++a) acc.F[a] += wt * s.F[a];
                            acc.T += wt * s.T;
                        }
                store(gc, coarse, ic, jc, kc, acc);
            }
}

static void restrict_scalar(const grid3_t* gf, const grid3_t* gc, const double* fine, double* coarse)
{
    static const double w[3] = { 0.25, 0.5, 0.25 };
    #pragma omp parallel for collapse(3) schedule(static)
    for (int kc = 0; kc < gc->n[2]; ++kc)
        for (int jc = 0; jc < gc->n[1]; ++jc)
            for (int ic = 0; ic < gc->n[0]; ++ic) {
                double acc = 0.0;
                for (int cz = -1; cz <= 1; ++cz)
                    for (int by = -1; by <= 1; ++by)
                        for (int ax = -1; ax <= 1; ++ax) {
                            int p[3] = { 2 * ic + ax, 2 * jc + by, 2 * kc + cz };
                            acc += w[ax + 1] * w[by + 1] * w[cz + 1] * get_scalar(gf, fine, p);
                        }
                coarse[idx(gc, ic, jc, kc)] = acc;
            }
}

void ora3_restrict_state(const int* idesc_f, const double* ddesc_f, const double* inflow_f,
                         int kind, const double* fine, double* coarse)
{
    grid3_t gf, gc; grid_from_desc(&gf, idesc_f, ddesc_f, inflow_f); coarse_desc(&gf, &gc);
    restrict_state(&gf, &gc, fine, coarse, kind);
}

/* Section 4.2, Fig. 1 / Eq. (14) on each axis: fine 2i takes coarse i, fine
 * 2i + 1 takes (coarse i + coarse i+1)/2; the tensor product on three axes
 * (weights 1, 1/2, 1/4, 1/8).  Coarse cells past the grid are its ghosts. */
static cell5_t prolong_cell(const grid3_t* gc, const double* coarse, int i, int j, int k, int kind)
{
    int base[3] = { i / 2, j / 2, k / 2 }, odd[3] = { i % 2, j % 2, k % 2 };
    cell5_t r = { 0.0, { 0.0, 0.0, 0.0 }, 0.0 };
    for (int cz = 0; cz <= odd[2]; ++cz)
        for (int by = 0; by <= odd[1]; ++by)
            for (int ax = 0; ax <= odd[0]; ++ax) {
                double wt = (odd[0] ? 0.5 : 1.0) * (odd[1] ? 0.5 : 1.0) * (odd[2] ? 0.5 : 1.0);
                int p[3] = { base[0] + ax, base[1] + by, base[2] + cz };
                cell5_t s = get_cell(gc, coarse, p, kind);
                r.E += wt * s.E;
                for (int a = 0; a < 3; ++a) r.F[a] += wt * s.F[a];
                r.T += wt * s.T;
            }
    return r;
}

/* Plain prolongation of a coarse state onto the fine grid (ghosts of kind
 * `kind`; inflow_c: the coarse grid's face profiles, or NULL). */
void ora3_prolong(const int* idesc_f, const double* ddesc_f, const double* inflow_c, int kind,
                  const double* coarse, double* fine)
{
    grid3_t gf, gc; grid_from_desc(&gf, idesc_f, ddesc_f, NULL); coarse_desc(&gf, &gc);
    set_inflow(&gc, inflow_c);
    #pragma omp parallel for collapse(3) schedule(static)
    for (int k = 0; k < gf.n[2]; ++k)
        for (int j = 0; j < gf.n[1]; ++j)
            for (int i = 0; i < gf.n[0]; ++i)
                store(&gf, fine, i, j, k, prolong_cell(&gc, coarse, i, j, k, kind));
}

/* Algorithm 4's prolongation with Eq. (34): u += P(u_c - v_c), damped by
 * theta min(1, theta*) in cells whose target is inadmissible [READING]. */
static int prolong_correct(const grid3_t* gc, const grid3_t* gf, const double* uc,
                           const double* vc, double* uf, double theta)
{
    size_t nc = ncell(gc);
    double* e = malloc(NF * nc * sizeof(double));
    for (size_t q = 0; q < NF * nc; ++q) e[q] = uc[q] - vc[q];
    int damped = 0;
    #pragma omp parallel for collapse(3) schedule(static) reduction(+:damped)
    for (int k = 0; k < gf->n[2]; ++k)
        for (int j = 0; j < gf->n[1]; ++j)
            for (int i = 0; i < gf->n[0]; ++i) {
                cell5_t u = load(gf, uf, i, j, k);
                cell5_t pe = prolong_cell(gc, e, i, j, k, KIND_DIFF);
                double th = 1.0;
                cell5_t t;
                t.E = u.E + pe.E;
                for (int a = 0; a < 3; ++a) t.F[a] = u.F[a] + pe.F[a];
                t.T = u.T + pe.T;
                if (!admissible(t, gf->c)) {
                    th = theta * dmin(1.0, max_admissible_step(u, pe, gf->c));
                    t.E = u.E + th * pe.E;
                    for (int a = 0; a < 3; ++a) t.F[a] = u.F[a] + th * pe.F[a];
                    t.T = u.T + th * pe.T;
                    ++damped;
                }
                store(gf, uf, i, j, k, t);
            }
    free(e);
    return damped;
}

/* ------------------------------------------------------------------------ */
/* Levels 0 .. L_max - 1, each axis halved per level [READING, as in 2D];
 * opacities restricted by full weighting. */
typedef struct {
    grid3_t g;
    double *sa, *ss, *v, *u, *f, *r, *inflow;
} level3_t;

static void build_levels(level3_t* lv, int L, const grid3_t* g0, const double* sa, const double* ss)
{
    for (int l = 0; l < L; ++l) {
        level3_t* q = &lv[l];
        q->inflow = NULL;
        if (l == 0) {
            q->g = *g0;
        } else {
            coarse_desc(&lv[l - 1].g, &q->g);
            q->inflow = calloc((size_t)6 * 4 * q->g.fstride, sizeof(double));
            restrict_faces(&lv[l - 1].g, &q->g, q->inflow);
            set_inflow(&q->g, q->inflow);
        }
        size_t n = ncell(&q->g);
        q->sa = malloc(n * sizeof(double)); q->ss = malloc(n * sizeof(double));
        q->v = calloc(NF * n, sizeof(double)); q->u = calloc(NF * n, sizeof(double));
        q->f = calloc(NF * n, sizeof(double)); q->r = calloc(NF * n, sizeof(double));
        if (l == 0) {
            memcpy(q->sa, sa, n * sizeof(double)); memcpy(q->ss, ss, n * sizeof(double));
        } else {
            restrict_scalar(&lv[l - 1].g, &q->g, lv[l - 1].sa, q->sa);
            restrict_scalar(&lv[l - 1].g, &q->g, lv[l - 1].ss, q->ss);
        }
    }
}

static void free_levels(level3_t* lv, int L)
{
    for (int l = 0; l < L; ++l) {
        free(lv[l].sa); free(lv[l].ss); free(lv[l].v); free(lv[l].u); free(lv[l].f); free(lv[l].r);
        free(lv[l].inflow);
    }
}

/* Eq. (24): the FAS right-hand side f = A(v) + r of a coarse level. */
static void fas_rhs(level3_t* q, double dt)
{
    size_t n = ncell(&q->g);
    double* a = malloc(NF * n * sizeof(double));
    #pragma omp parallel for collapse(3) schedule(static)
    for (int k = 0; k < q->g.n[2]; ++k)
        for (int j = 0; j < q->g.n[1]; ++j)
            for (int i = 0; i < q->g.n[0]; ++i)
                store(&q->g, a, i, j, k, apply_A_cell(&q->g, dt, q->sa, q->ss, q->v, i, j, k));
    for (size_t s = 0; s < NF * n; ++s) q->f[s] = a[s] + q->r[s];
    free(a);
}

static int fine_jacobi(level3_t* q, double dt, const double* b, double* u, int nu)
{
    size_t n = ncell(&q->g);
    double* tmp = malloc(NF * n * sizeof(double));
    int worst = 0;
    for (int s = 0; s < nu; ++s) {
        if (jacobi_sweep(&q->g, dt, q->sa, q->ss, b, u, tmp, 0.0, 1.0) < 0) worst = -1;
        memcpy(u, tmp, NF * n * sizeof(double));
    }
    free(tmp);
    return worst;
}

/* Cycle shapes as in the 2D oracle (Section 4.2 recursion; Section 6.3 names W
 * and F): the coarse-grid corrections of level l are one visit of level l + 1
 * (V), a fresh and a repeated one (W), or a fresh F- and a repeated V-visit
 * (F); the coarsest level is visited once per correction. */
typedef struct {
    double dt, dtau, th_ex, th_c;
    int m, mc, nul, L, newton_fail, damped;
} ctx3_t;

static void coarse_visit(level3_t* lv, int l, int fresh, int shape, ctx3_t* c);

static void corrections(level3_t* lv, int l, int shape, ctx3_t* c)
{
    if (l + 1 == c->L - 1 || shape == 0) {
        coarse_visit(lv, l + 1, 1, shape, c);
    } else if (shape == 1) {
        coarse_visit(lv, l + 1, 1, 1, c);
        coarse_visit(lv, l + 1, 0, 1, c);
    } else {
        coarse_visit(lv, l + 1, 1, 2, c);
        coarse_visit(lv, l + 1, 0, 0, c);
    }
}

static void coarse_visit(level3_t* lv, int l, int fresh, int shape, ctx3_t* c)
{
    level3_t* q = &lv[l];
    size_t n = ncell(&q->g);
    if (fresh) {
        fas_rhs(q, c->dt);
        memcpy(q->u, q->v, NF * n * sizeof(double));
    }
    int mm = l == c->L - 1 ? c->mc : c->m;
    if (pseudo_time_smooth(&q->g, c->dt, q->sa, q->ss, q->f, q->u, c->dtau, mm, c->nul, c->th_ex) < 0)
        ++c->newton_fail;
    if (l == c->L - 1) return;
    level3_t* p = &lv[l + 1];
    residual(&q->g, c->dt, q->sa, q->ss, q->f, q->u, q->r);
    restrict_state(&q->g, &p->g, q->u, p->v, KIND_STATE);
    restrict_state(&q->g, &p->g, q->r, p->r, KIND_DIFF);
    corrections(lv, l, shape, c);
    c->damped += prolong_correct(&p->g, &q->g, p->u, p->v, q->u, c->th_c);
    if (pseudo_time_smooth(&q->g, c->dt, q->sa, q->ss, q->f, q->u, c->dtau, c->m, c->nul, c->th_ex) < 0)
        ++c->newton_fail;
}

/* Appendix A, Algorithm 4 in 3D: one implicit step v^n -> v^{n+1}.
 *   ip = { L_max, nu0, nu_l, m, m_coarse, max_cycles, dtau_rule, cycle shape }
 *   dp = { dtau0, grow, shrink, eps_i, eps_d, tol, dtau_min, dtau_max, theta_ex, theta_c }
 * The cycle loop, the stop tests and the dtau control are those of the 2D
 * oracle (printed |change| rule, or the worded signed rule when dtau_rule = 1).
 * stats = { cycles, res0, res, dtau, fine_sweeps, status, newton_fail, damped };
 * res_hist[kappa] for kappa = 0 .. cycles.  status: 0 converged, -4 not
 * converged, -2 inadmissible input, -1 invalid parameters. */
int ora3_implicit_step(const int* idesc, const double* ddesc, const double* inflow, double dt,
                       const double* sa, const double* ss, const int* ip, const double* dp,
                       double* v, double* stats, double* res_hist)
{
    grid3_t g0; grid_from_desc(&g0, idesc, ddesc, inflow);
    int L = ip[0], nu0 = ip[1], nul = ip[2], m = ip[3], mc = ip[4], maxc = ip[5];
    int signed_rule = ip[6], shape = ip[7];
    double dtau = dp[0], grow = dp[1], shrink = dp[2], eps_i = dp[3], eps_d = dp[4], tol = dp[5];
    double dtau_min = dp[6], dtau_max = dp[7], th_ex = dp[8], th_c = dp[9];
    for (int s = 0; s < 8; ++s) stats[s] = 0.0;
    if (L < 1 || shape < 0 || shape > 2) { stats[5] = -1; return -1; }
    size_t n0 = ncell(&g0);
    for (int k = 0; k < g0.n[2]; ++k)
        for (int j = 0; j < g0.n[1]; ++j)
            for (int i = 0; i < g0.n[0]; ++i)
                if (!admissible(load(&g0, v, i, j, k), g0.c)) { stats[5] = -2; return -2; }
    level3_t* lv = calloc((size_t)L, sizeof(level3_t));
    build_levels(lv, L, &g0, sa, ss);
    level3_t* q0 = &lv[0];
    double* b = malloc(NF * n0 * sizeof(double));
    memcpy(b, v, NF * n0 * sizeof(double));
    for (size_t q = 0; q < n0; ++q) b[4 * n0 + q] = g0.c_v * v[4 * n0 + q];
    memcpy(q0->v, v, NF * n0 * sizeof(double));
    residual(&g0, dt, sa, ss, b, q0->v, q0->r);
    double bnorm = norm(&g0, b);
    double res0 = norm(&g0, q0->r), res_prev = res0, res = res0;
    res_hist[0] = res0;
    int kappa = 0, status = 0, newton_fail = 0, damped = 0;
    long long fine_sweeps = 0;
    if (res0 > 1e-14 * transport_diag(&g0, dt) * bnorm) {
        status = -4;
        while (kappa < maxc) {
            memcpy(q0->u, q0->v, NF * n0 * sizeof(double));
            if (fine_jacobi(q0, dt, b, q0->u, nu0) < 0) ++newton_fail;
            fine_sweeps += nu0;
            if (L > 1) {
                level3_t* p = &lv[1];
                ctx3_t c = { dt, dtau, th_ex, th_c, m, mc, nul, L, 0, 0 };
                residual(&g0, dt, sa, ss, b, q0->u, q0->r);
                restrict_state(&g0, &p->g, q0->u, p->v, KIND_STATE);
                restrict_state(&g0, &p->g, q0->r, p->r, KIND_DIFF);
                corrections(lv, 0, shape, &c);
                c.damped += prolong_correct(&p->g, &g0, p->u, p->v, q0->u, th_c);
                if (fine_jacobi(q0, dt, b, q0->u, nu0) < 0) ++c.newton_fail;
                fine_sweeps += nu0;
                newton_fail += c.newton_fail;
                damped += c.damped;
            }
            memcpy(q0->v, q0->u, NF * n0 * sizeof(double));
            residual(&g0, dt, sa, ss, b, q0->v, q0->r);
            ++kappa;
            res = norm(&g0, q0->r);
            res_hist[kappa] = res;
            if (res <= tol * res0) { status = 0; break; }
            double delta = (signed_rule ? res_prev - res : fabs(res - res_prev)) / res0;
            if (delta > eps_i) dtau *= grow;
            if (delta < eps_d) dtau *= shrink;
            if (dtau < dtau_min) dtau = dtau_min;
            if (dtau > dtau_max) dtau = dtau_max;
            res_prev = res;
        }
    }
    memcpy(v, q0->v, NF * n0 * sizeof(double));
    stats[0] = kappa; stats[1] = res0; stats[2] = res; stats[3] = dtau;
    stats[4] = (double)fine_sweeps; stats[5] = status; stats[6] = newton_fail; stats[7] = damped;
    free(b);
    free_levels(lv, L);
    free(lv);
    return status;
}
