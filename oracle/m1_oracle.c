/*
 * m1_oracle.c -- plain, slow, FP64 CPU oracle for one implicit time step of the
 * M1 moment model solved by the nonlinear FAS multigrid of Bloch, Tremblin,
 * Gonzalez & Audit, "Towards a multigrid method for the M1 model for radiative
 * transfer" (arXiv:2208.14703).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call, link or load
 * this file: only the tests, the smoke check and the CPU-baseline leg of the
 * benchmark use it.  It shares no code, header, table or constant generator with
 * the CUDA implementation.
 *
 * Every function follows one passage of the paper, cited in its comment, and is
 * written for a reader checking it against that passage by eye: one cell at a
 * time, no blocking, no fusion, no reordering.  Passages the paper leaves open
 * (source terms, 2D operator, boundary ghosts, loop bounds of Algorithm 4, the
 * explicit pseudo-time sub-step, the prolongation damping factor, the residual
 * norm, the pseudo-time step thresholds) follow one stated reading, marked
 * [READING] here and listed in the design notes.  The source terms (absorption,
 * scattering, gas temperature) are not in the paper's solver at all: the paper
 * sets every opacity to zero (Section 2.1).  They are an extension derived from
 * the continuous system, Eq. (3), and are marked [EXT].
 *
 * Data layout: a state is 4 planes [E | Fx | Fy | T], each ny*nx doubles,
 * row-major (index j*nx+i).  In 1D, ny = 1 and the Fy plane stays zero.
 *
 * Threads.  The outer cell loops carry OpenMP pragmas.  The plain build ignores
 * them (one core); the all-core build (-fopenmp) runs the same loops on every
 * host core.  Every cell's arithmetic is the same in both, the loop reductions
 * are over integers and the norm is summed serially, so both builds give
 * bit-for-bit the same results.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

enum { BC_PERIODIC = 0, BC_REFLECT = 1, BC_NEUMANN = 2, BC_INFLOW = 3 };
enum { KIND_STATE = 0, KIND_DIFF = 1 };
enum { WALL_W = 0, WALL_E = 1, WALL_S = 2, WALL_N = 3 };

/* Tolerance of the admissibility test that decides whether a prolongated cell
 * is damped (Algorithm 4, prolongation step).  A relative slack of 1e-12 on
 * |F|^2 <= c^2 E^2 keeps cells that sit on the f = 1 boundary up to rounding
 * (a free-streaming beam) from being damped by rounding noise. [READING] */
#define ADM_SLACK 1e-12

typedef struct {
    int dim, nx, ny;
    double hx, hy, c, a_r, c_v;
    int bc[4];
    /* inflow ghost states per wall, length ny (W/E) or nx (S/N); NULL if unused */
    const double *in_E[4], *in_Fx[4], *in_Fy[4];
} grid_t;

typedef struct { double E, Fx, Fy, T; } cell_t;

static double sq(double x) { return x * x; }
static double dmin(double a, double b) { return a < b ? a : b; }

static void grid_from_desc(grid_t* g, const int* idesc, const double* ddesc, const double* inflow)
{
    g->dim = idesc[0]; g->nx = idesc[1]; g->ny = idesc[2];
    for (int w = 0; w < 4; ++w) g->bc[w] = idesc[3 + w];
    g->hx = ddesc[0]; g->hy = ddesc[1]; g->c = ddesc[2]; g->a_r = ddesc[3]; g->c_v = ddesc[4];
    /* inflow layout: [wall][field E,Fx,Fy][Lmax], Lmax = max(nx, ny) */
    int L = g->nx > g->ny ? g->nx : g->ny;
    for (int w = 0; w < 4; ++w) {
        if (inflow && g->bc[w] == BC_INFLOW) {
            g->in_E[w] = inflow + (size_t)(w * 3 + 0) * L;
            g->in_Fx[w] = inflow + (size_t)(w * 3 + 1) * L;
            g->in_Fy[w] = inflow + (size_t)(w * 3 + 2) * L;
        } else {
            g->in_E[w] = g->in_Fx[w] = g->in_Fy[w] = NULL;
        }
    }
}

/* Host threads the cell loops run on: 1 in the plain build. */
int ora_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------------ */
/* Section 2.1, Eq. (5): M1 closure.  chi = (3 + 4 f^2) / (5 + 2 sqrt(4 - 3 f^2)),
 * n = F/|F|, P = ((1 - chi)/2 I + (3 chi - 1)/2 n (x) n) E.  The flux lies in the
 * x-y plane; the components Pxx, Pxy, Pyy are returned.  f is clamped to 1 so
 * that rounding on the f = 1 boundary cannot leave the domain of the root. */
void ora_closure(double E, double Fx, double Fy, double c, double* P)
{
    double normF = sqrt(Fx * Fx + Fy * Fy);
    double f = normF / (c * E);
    if (f > 1.0) f = 1.0;
    double chi = (3.0 + 4.0 * f * f) / (5.0 + 2.0 * sqrt(4.0 - 3.0 * f * f));
    double nx = 0.0, ny = 0.0;
    if (normF > 0.0) { nx = Fx / normF; ny = Fy / normF; }
    double iso = 0.5 * (1.0 - chi), dir = 0.5 * (3.0 * chi - 1.0);
    P[0] = (iso + dir * nx * nx) * E;
    P[1] = (dir * nx * ny) * E;
    P[2] = (iso + dir * ny * ny) * E;
}

double ora_eddington_factor(double f)
{
    return (3.0 + 4.0 * f * f) / (5.0 + 2.0 * sqrt(4.0 - 3.0 * f * f));
}

/* ------------------------------------------------------------------------ */
/* Ghost cells.  The paper only asks for "appropriate boundary conditions"
 * (Section 4.2).  [READING] one ghost layer per wall:
 *   periodic: wrap;  reflecting: mirror cell with the wall-normal flux negated;
 *   Neumann: copy;   inflow: the prescribed (E, Fx, Fy), T copied.
 * Differences (errors, residuals) use the same rules except that an inflow
 * ghost holds zero, since the prescribed state has no error. */
static cell_t load(const grid_t* g, const double* v, int i, int j)
{
    size_t n = (size_t)g->nx * g->ny, k = (size_t)j * g->nx + i;
    cell_t s = { v[k], v[n + k], v[2 * n + k], v[3 * n + k] };
    return s;
}

static cell_t get_cell(const grid_t* g, const double* v, int i, int j, int kind)
{
    if (i < 0 || i >= g->nx) {
        int wall = i < 0 ? WALL_W : WALL_E;
        int bc = g->bc[wall];
        if (bc == BC_PERIODIC) return get_cell(g, v, i < 0 ? i + g->nx : i - g->nx, j, kind);
        int im = i < 0 ? -1 - i : 2 * g->nx - 1 - i;
        cell_t m = get_cell(g, v, im, j, kind);
        if (bc == BC_REFLECT) { m.Fx = -m.Fx; return m; }
        if (bc == BC_NEUMANN) return m;
        /* inflow */
        if (kind == KIND_DIFF) { m.E = m.Fx = m.Fy = m.T = 0.0; return m; }
        int jj = j < 0 ? 0 : (j >= g->ny ? g->ny - 1 : j);
        m.E = g->in_E[wall][jj]; m.Fx = g->in_Fx[wall][jj]; m.Fy = g->in_Fy[wall][jj];
        return m;
    }
    if (j < 0 || j >= g->ny) {
        int wall = j < 0 ? WALL_S : WALL_N;
        int bc = g->bc[wall];
        if (bc == BC_PERIODIC) return get_cell(g, v, i, j < 0 ? j + g->ny : j - g->ny, kind);
        int jm = j < 0 ? -1 - j : 2 * g->ny - 1 - j;
        cell_t m = get_cell(g, v, i, jm, kind);
        if (bc == BC_REFLECT) { m.Fy = -m.Fy; return m; }
        if (bc == BC_NEUMANN) return m;
        if (kind == KIND_DIFF) { m.E = m.Fx = m.Fy = m.T = 0.0; return m; }
        m.E = g->in_E[wall][i]; m.Fx = g->in_Fx[wall][i]; m.Fy = g->in_Fy[wall][i];
        return m;
    }
    return load(g, v, i, j);
}

static double get_scalar(const grid_t* g, const double* s, int i, int j)
{
    if (i < 0 || i >= g->nx) {
        if (g->bc[i < 0 ? WALL_W : WALL_E] == BC_PERIODIC) i = i < 0 ? i + g->nx : i - g->nx;
        else i = i < 0 ? -1 - i : 2 * g->nx - 1 - i;
    }
    if (j < 0 || j >= g->ny) {
        if (g->bc[j < 0 ? WALL_S : WALL_N] == BC_PERIODIC) j = j < 0 ? j + g->ny : j - g->ny;
        else j = j < 0 ? -1 - j : 2 * g->ny - 1 - j;
    }
    return s[(size_t)j * g->nx + i];
}

static void store(const grid_t* g, double* v, int i, int j, cell_t s)
{
    size_t n = (size_t)g->nx * g->ny, k = (size_t)j * g->nx + i;
    v[k] = s.E; v[n + k] = s.Fx; v[2 * n + k] = s.Fy; v[3 * n + k] = s.T;
}

/* ------------------------------------------------------------------------ */
/* Section 3.1, Eq. (9): the neighbour operators L (left/south neighbour) and
 * R (right/north neighbour) of the implicit Rusanov scheme, Eq. (6), evaluated
 * on one neighbour state.  axis 0 = x (uses Fx, Pxx, Pxy), axis 1 = y (uses Fy,
 * Pxy, Pyy); the 2D extension follows the same face flux on each axis.
 * sign = +1 for L (the neighbour on the low side), -1 for R. */
static void neighbour_term(const grid_t* g, double dt, double h, int axis, double sign,
                           cell_t nb, double out[3])
{
    double beta = dt / (2.0 * h), c = g->c, P[3];
    ora_closure(nb.E, nb.Fx, nb.Fy, c, P);
    double Fn = axis == 0 ? nb.Fx : nb.Fy;           /* flux normal to the face */
    double Pnx = axis == 0 ? P[0] : P[1];            /* P(normal, x) */
    double Pny = axis == 0 ? P[1] : P[2];            /* P(normal, y) */
    out[0] = beta * (c * nb.E + sign * Fn);
    out[1] = c * beta * (nb.Fx + sign * c * Pnx);
    out[2] = c * beta * (nb.Fy + sign * c * Pny);
}

/* Sum of the L and R terms of all neighbours of cell (i,j), Eq. (10). */
static void neighbour_sum(const grid_t* g, double dt, const double* v, int i, int j, double s[3])
{
    double t[3];
    s[0] = s[1] = s[2] = 0.0;
    neighbour_term(g, dt, g->hx, 0, +1.0, get_cell(g, v, i - 1, j, KIND_STATE), t);
    s[0] += t[0]; s[1] += t[1]; s[2] += t[2];
    neighbour_term(g, dt, g->hx, 0, -1.0, get_cell(g, v, i + 1, j, KIND_STATE), t);
    s[0] += t[0]; s[1] += t[1]; s[2] += t[2];
    if (g->dim == 2) {
        neighbour_term(g, dt, g->hy, 1, +1.0, get_cell(g, v, i, j - 1, KIND_STATE), t);
        s[0] += t[0]; s[1] += t[1]; s[2] += t[2];
        neighbour_term(g, dt, g->hy, 1, -1.0, get_cell(g, v, i, j + 1, KIND_STATE), t);
        s[0] += t[0]; s[1] += t[1]; s[2] += t[2];
    }
}

/* Transport diagonal 1 + c dt/hx (+ c dt/hy in 2D), Eq. (9). */
static double transport_diag(const grid_t* g, double dt)
{
    double d = 1.0 + g->c * dt / g->hx;
    if (g->dim == 2) d += g->c * dt / g->hy;
    return d;
}

/* ------------------------------------------------------------------------ */
/* Eq. (12): row i of the nonlinear operator A, A(v)_i = D(v_i) - L(v_{i-1}) -
 * R(v_{i+1}) (2D: plus the south/north pair), with the [EXT] backward-Euler
 * source terms of Eq. (3):  sigma_E = sigma_P = sigma_F = sigma_a, the (1-g)
 * sigma_R term read as sigma_s with g = 0; k_a = c dt sigma_a, k_t = c dt
 * (sigma_a + sigma_s); gas row C_v T - k_a (E - a_r T^4), right-hand side
 * C_v T^n. */
static cell_t apply_A_cell(const grid_t* g, double dt, const double* sa, const double* ss,
                           const double* v, int i, int j)
{
    size_t k = (size_t)j * g->nx + i;
    cell_t u = load(g, v, i, j), out;
    double diag = transport_diag(g, dt);
    double ka = g->c * dt * sa[k], kt = g->c * dt * (sa[k] + ss[k]);
    double src = ka * (u.E - g->a_r * sq(sq(u.T)));
    double s[3];
    neighbour_sum(g, dt, v, i, j, s);
    out.E = diag * u.E + src - s[0];
    out.Fx = (diag + kt) * u.Fx - s[1];
    out.Fy = (diag + kt) * u.Fy - s[2];
    out.T = g->c_v * u.T - src;
    return out;
}

void ora_apply_A(const int* idesc, const double* ddesc, const double* inflow, double dt,
                 const double* sa, const double* ss, const double* v, double* out)
{
    grid_t g; grid_from_desc(&g, idesc, ddesc, inflow);
    #pragma omp parallel for collapse(2) schedule(static)
    for (int j = 0; j < g.ny; ++j)
        for (int i = 0; i < g.nx; ++i) store(&g, out, i, j, apply_A_cell(&g, dt, sa, ss, v, i, j));
}

/* Eq. (13): residual r = b - A(v). */
void ora_residual(const int* idesc, const double* ddesc, const double* inflow, double dt,
                  const double* sa, const double* ss, const double* b, const double* v, double* r)
{
    grid_t g; grid_from_desc(&g, idesc, ddesc, inflow);
    size_t n = (size_t)g.nx * g.ny;
    #pragma omp parallel for collapse(2) schedule(static)
    for (int j = 0; j < g.ny; ++j)
        for (int i = 0; i < g.nx; ++i) {
            size_t k = (size_t)j * g.nx + i;
            cell_t a = apply_A_cell(&g, dt, sa, ss, v, i, j);
            r[k] = b[k] - a.E; r[n + k] = b[n + k] - a.Fx;
            r[2 * n + k] = b[2 * n + k] - a.Fy; r[3 * n + k] = b[3 * n + k] - a.T;
        }
}

/* [READING] The paper writes ||r|| without defining it.  Here
 * ||r||^2 = sum over cells of h^d (rE^2 + (rFx^2 + rFy^2)/c^2 + rT^2). */
double ora_norm(const int* idesc, const double* ddesc, const double* r)
{
    grid_t g; grid_from_desc(&g, idesc, ddesc, NULL);
    size_t n = (size_t)g.nx * g.ny;
    double vol = g.dim == 2 ? g.hx * g.hy : g.hx, s = 0.0;
    for (size_t k = 0; k < n; ++k)
        s += vol * (sq(r[k]) + (sq(r[n + k]) + sq(r[2 * n + k])) / sq(g.c) + sq(r[3 * n + k]));
    return sqrt(s);
}

/* ------------------------------------------------------------------------ */
/* [EXT] Inverse of the local operator D, Section 3.1: solves for one cell
 *   (w0 + w1 diag) E + w1 k_a (E - a_r T^4)      = bE
 *   (w0 + w1 (diag + k_t)) F                      = bF
 *   (w0 + w1 C_v) T - w1 k_a (E - a_r T^4)        = bT
 * with (w0, w1) = (0, 1) for the fine-level Jacobi update, Eq. (10), and
 * (1, dtau) for the implicit pseudo-time step of Eq. (30).  With k_a = 0 and
 * (w0, w1) = (0, 1) it is the paper's D^{-1} = (1 + c dt/h)^{-1} I (proof of
 * Proposition 1).  Eliminating E leaves g(T) = C T + K T^4 - R = 0 with
 * A = w0 + w1 diag, k = w1 k_a, C = w0 + w1 C_v, K = k A a_r / (A + k),
 * R = bT + k bE / (A + k); g is increasing and convex for T > 0, so Newton from
 * T0 = min(R/C, (R/K)^(1/4)) (both at or right of the root) decreases
 * monotonically to it.  Stops when |dT| <= 1e-15 T or after 60 iterations.
 * Returns the iteration count, -1 if it did not converge. */
int ora_local_solve(double w0, double w1, double diag, double ka, double kt, double c_v,
                    double a_r, const double* beta, double* out)
{
    double A = w0 + w1 * diag, k = w1 * ka;
    double Fden = w0 + w1 * (diag + kt);
    out[1] = beta[1] / Fden;
    out[2] = beta[2] / Fden;
    double C = w0 + w1 * c_v;
    double K = k * A * a_r / (A + k);
    double R = beta[3] + k * beta[0] / (A + k);
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
    out[3] = T;
    out[0] = (beta[0] + k * a_r * sq(sq(T))) / (A + k);
    return ok ? it : -1;
}

/* Algorithm 1, one sweep of Eq. (10):  v_out_i = D^{-1}(rhs_i + w1 (L(v_{i-1}) +
 * R(v_{i+1}) + ...)), every neighbour taken from the old iterate v_in (pure
 * Jacobi).  (w0, w1) as in ora_local_solve.  Returns the largest Newton
 * iteration count, or -1 if some local solve failed. */
static int jacobi_sweep(const grid_t* g, double dt, const double* sa, const double* ss,
                        const double* rhs, const double* vin, double* vout, double w0, double w1)
{
    double diag = transport_diag(g, dt);
    int fail = 0, maxit = 0;
    #pragma omp parallel for collapse(2) schedule(static) reduction(|:fail) reduction(max:maxit)
    for (int j = 0; j < g->ny; ++j)
        for (int i = 0; i < g->nx; ++i) {
            size_t k = (size_t)j * g->nx + i;
            double s[3], beta[4], out[4];
            cell_t b = load(g, rhs, i, j);
            neighbour_sum(g, dt, vin, i, j, s);
            beta[0] = b.E + w1 * s[0];
            beta[1] = b.Fx + w1 * s[1];
            beta[2] = b.Fy + w1 * s[2];
            beta[3] = b.T;
            int it = ora_local_solve(w0, w1, diag, g->c * dt * sa[k], g->c * dt * (sa[k] + ss[k]),
                                     g->c_v, g->a_r, beta, out);
            if (it < 0) fail = 1; else if (it > maxit) maxit = it;
            cell_t o = { out[0], out[1], out[2], out[3] };
            store(g, vout, i, j, o);
        }
    return fail ? -1 : maxit;
}

int ora_jacobi_sweep(const int* idesc, const double* ddesc, const double* inflow, double dt,
                     const double* sa, const double* ss, const double* rhs, const double* vin,
                     double* vout, double w0, double w1)
{
    grid_t g; grid_from_desc(&g, idesc, ddesc, inflow);
    return jacobi_sweep(&g, dt, sa, ss, rhs, vin, vout, w0, w1);
}

/* ------------------------------------------------------------------------ */
/* Admissible set S, Eq. (7) (with the [EXT] gas condition T > 0): the largest
 * step tau >= 0 such that u + tau d stays in S.  [READING] E + tau dE > 0,
 * T + tau dT > 0 and the first positive root of |F + tau dF|^2 = c^2 (E + tau dE)^2
 * (a quadratic a tau^2 + 2 b tau + c0).  Returns +inf when no bound applies. */
double ora_max_admissible_step(double E, double Fx, double Fy, double T, double dE,
                               double dFx, double dFy, double dT, double c)
{
    double tau = INFINITY;
    if (dE < 0.0) tau = dmin(tau, -E / dE);
    if (dT < 0.0) tau = dmin(tau, -T / dT);
    double a = dFx * dFx + dFy * dFy - c * c * dE * dE;
    double b = Fx * dFx + Fy * dFy - c * c * E * dE;
    double c0 = Fx * Fx + Fy * Fy - c * c * E * E;
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

static int admissible(cell_t s, double c)
{
    return s.E > 0.0 && s.T > 0.0 && s.Fx * s.Fx + s.Fy * s.Fy <= c * c * s.E * s.E * (1.0 + ADM_SLACK);
}

int ora_admissible(double E, double Fx, double Fy, double T, double c)
{
    cell_t s = { E, Fx, Fy, T };
    return admissible(s, c);
}

/* ------------------------------------------------------------------------ */
/* Algorithm 3 (pseudo-time smoother at a coarse level), m pseudo-time steps.
 * Each step: the explicit half of Eq. (30) per cell, u~ = u^m + tau_i f, with
 * the source f = A(v) + r constant over the sub-cycle; since f is constant the
 * sub-cycle of Algorithm 3 is a single step of total length tau_i.  [READING]
 * tau_i = min(dtau_im, theta * tau*_i), tau*_i the largest admissible step
 * along f (theta = 1/2).  Then the implicit half of Eq. (30),
 * u^{m+1} + dtau_im A(u^{m+1}) = u~, by nu Jacobi sweeps (Algorithm 1 with
 * (w0, w1) = (1, dtau_im)) starting from u^m.  u is updated in place. */
static int pseudo_time_smooth(const grid_t* g, double dt, const double* sa, const double* ss,
                              const double* f, double* u, double dtau, int m, int nu,
                              double theta)
{
    size_t n = (size_t)g->nx * g->ny;
    double* ut = malloc(4 * n * sizeof(double));
    double* w = malloc(4 * n * sizeof(double));
    double* w2 = malloc(4 * n * sizeof(double));
    int worst = 0;
    for (int it = 0; it < m; ++it) {
        #pragma omp parallel for collapse(2) schedule(static)
        for (int j = 0; j < g->ny; ++j)
            for (int i = 0; i < g->nx; ++i) {
                cell_t s = load(g, u, i, j), d = load(g, f, i, j), o;
                double tstar = ora_max_admissible_step(s.E, s.Fx, s.Fy, s.T, d.E, d.Fx, d.Fy, d.T, g->c);
                double tau = dmin(dtau, theta * tstar);
                o.E = s.E + tau * d.E; o.Fx = s.Fx + tau * d.Fx;
                o.Fy = s.Fy + tau * d.Fy; o.T = s.T + tau * d.T;
                store(g, ut, i, j, o);
            }
        memcpy(w, u, 4 * n * sizeof(double));
        for (int s = 0; s < nu; ++s) {
            int r = jacobi_sweep(g, dt, sa, ss, ut, w, w2, 1.0, dtau);
            if (r < 0) worst = -1;
            memcpy(w, w2, 4 * n * sizeof(double));
        }
        memcpy(u, w, 4 * n * sizeof(double));
    }
    free(ut); free(w); free(w2);
    return worst;
}

int ora_pseudo_time_smooth(const int* idesc, const double* ddesc, const double* inflow, double dt,
                           const double* sa, const double* ss, const double* f, double* u,
                           double dtau, int m, int nu, double theta)
{
    grid_t g; grid_from_desc(&g, idesc, ddesc, inflow);
    return pseudo_time_smooth(&g, dt, sa, ss, f, u, dtau, m, nu, theta);
}

/* ------------------------------------------------------------------------ */
/* Section 4.2, Eq. (21)/(22): full-weighting restriction R = 2^-d P^T,
 * weights 1/4, 1/2, 1/4 per axis (tensor product in 2D: 1/16, 1/8, 1/4).
 * Coarse cell ic gathers fine cells 2ic-1, 2ic, 2ic+1; the ghost rules above
 * supply fine cell -1.  In 1D the y axis is not coarsened. */
static void restrict_state(const grid_t* gf, const grid_t* gc, const double* fine, double* coarse,
                           int kind)
{
    static const double w[3] = { 0.25, 0.5, 0.25 };
    #pragma omp parallel for collapse(2) schedule(static)
    for (int jc = 0; jc < gc->ny; ++jc)
        for (int ic = 0; ic < gc->nx; ++ic) {
            cell_t acc = { 0, 0, 0, 0 };
            for (int b = -1; b <= 1; ++b) {
                double wy = gf->dim == 2 ? w[b + 1] : (b == 0 ? 1.0 : 0.0);
                if (wy == 0.0) continue;
                for (int a = -1; a <= 1; ++a) {
                    double wt = wy * w[a + 1];
                    int jf = gf->dim == 2 ? 2 * jc + b : 0;
                    cell_t s = get_cell(gf, fine, 2 * ic + a, jf, kind);
                    acc.E += wt * s.E; acc.Fx += wt * s.Fx; acc.Fy += wt * s.Fy; acc.T += wt * s.T;
                }
            }
            store(gc, coarse, ic, jc, acc);
        }
}

static void restrict_scalar(const grid_t* gf, const grid_t* gc, const double* fine, double* coarse)
{
    static const double w[3] = { 0.25, 0.5, 0.25 };
    #pragma omp parallel for collapse(2) schedule(static)
    for (int jc = 0; jc < gc->ny; ++jc)
        for (int ic = 0; ic < gc->nx; ++ic) {
            double acc = 0.0;
            for (int b = -1; b <= 1; ++b) {
                double wy = gf->dim == 2 ? w[b + 1] : (b == 0 ? 1.0 : 0.0);
                if (wy == 0.0) continue;
                for (int a = -1; a <= 1; ++a) {
                    int jf = gf->dim == 2 ? 2 * jc + b : 0;
                    acc += wy * w[a + 1] * get_scalar(gf, fine, 2 * ic + a, jf);
                }
            }
            coarse[(size_t)jc * gc->nx + ic] = acc;
        }
}

/* Section 4.2, Fig. 1 and Eq. (14) (1D), Eq. (18) (2D): fine cell 2i takes coarse
 * cell i, fine cell 2i+1 takes (coarse i + coarse i+1)/2; in 2D the tensor
 * product (weights 1, 1/2, 1/2, 1/4).  Coarse cell nc (past the last) is the
 * ghost of the coarse grid. */
static cell_t prolong_cell(const grid_t* gc, const double* coarse, int i, int j, int dim, int kind)
{
    int ic = i / 2, jc = dim == 2 ? j / 2 : 0;
    int ox = i % 2, oy = dim == 2 ? j % 2 : 0;
    cell_t r = { 0, 0, 0, 0 };
    for (int b = 0; b <= oy; ++b)
        for (int a = 0; a <= ox; ++a) {
            double wt = (ox ? 0.5 : 1.0) * (oy ? 0.5 : 1.0);
            cell_t s = get_cell(gc, coarse, ic + a, jc + b, kind);
            r.E += wt * s.E; r.Fx += wt * s.Fx; r.Fy += wt * s.Fy; r.T += wt * s.T;
        }
    return r;
}

/* Algorithm 4, prolongation step with Eq. (34): u_bar = u + P(u_c - v_c) per
 * fine cell; a cell whose target is not admissible is replaced by
 * u + theta_c P(e), theta_c = dtau_bar/(1 + dtau_bar).  [READING] theta_c =
 * theta * min(1, theta*), theta* the largest admissible fraction of P(e),
 * theta = 1/2.  Returns the number of damped cells. */
static int prolong_correct(const grid_t* gc, const grid_t* gf, const double* uc, const double* vc,
                           double* uf, double theta)
{
    size_t nc = (size_t)gc->nx * gc->ny;
    double* e = malloc(4 * nc * sizeof(double));
    for (size_t k = 0; k < 4 * nc; ++k) e[k] = uc[k] - vc[k];
    int damped = 0;
    #pragma omp parallel for collapse(2) schedule(static) reduction(+:damped)
    for (int j = 0; j < gf->ny; ++j)
        for (int i = 0; i < gf->nx; ++i) {
            cell_t u = load(gf, uf, i, j);
            cell_t pe = prolong_cell(gc, e, i, j, gf->dim, KIND_DIFF);
            cell_t t = { u.E + pe.E, u.Fx + pe.Fx, u.Fy + pe.Fy, u.T + pe.T };
            if (!admissible(t, gf->c)) {
                double ts = ora_max_admissible_step(u.E, u.Fx, u.Fy, u.T, pe.E, pe.Fx, pe.Fy, pe.T, gf->c);
                double th = theta * dmin(1.0, ts);
                t.E = u.E + th * pe.E; t.Fx = u.Fx + th * pe.Fx;
                t.Fy = u.Fy + th * pe.Fy; t.T = u.T + th * pe.T;
                ++damped;
            }
            store(gf, uf, i, j, t);
        }
    free(e);
    return damped;
}

/* Exported transfer entry points for the tests. */
static void coarse_desc(const grid_t* gf, grid_t* gc)
{
    *gc = *gf;
    gc->nx = gf->nx / 2;
    gc->ny = gf->dim == 2 ? gf->ny / 2 : 1;
    gc->hx = 2.0 * gf->hx;
    gc->hy = gf->dim == 2 ? 2.0 * gf->hy : gf->hy;
}

void ora_restrict_state(const int* idesc_f, const double* ddesc_f, const double* inflow_f,
                        int kind, const double* fine, double* coarse)
{
    grid_t gf, gc; grid_from_desc(&gf, idesc_f, ddesc_f, inflow_f); coarse_desc(&gf, &gc);
    restrict_state(&gf, &gc, fine, coarse, kind);
}

void ora_restrict_scalar(const int* idesc_f, const double* ddesc_f, const double* fine, double* coarse)
{
    grid_t gf, gc; grid_from_desc(&gf, idesc_f, ddesc_f, NULL); coarse_desc(&gf, &gc);
    restrict_scalar(&gf, &gc, fine, coarse);
}

/* Plain prolongation of a coarse state (ghosts of kind `kind`) onto the fine grid
 * described by idesc_f. */
void ora_prolong(const int* idesc_f, const double* ddesc_f, const double* inflow_c, int kind,
                 const double* coarse, double* fine)
{
    grid_t gf, gc; grid_from_desc(&gf, idesc_f, ddesc_f, NULL); coarse_desc(&gf, &gc);
    for (int w = 0; w < 4; ++w) gc.in_E[w] = gc.in_Fx[w] = gc.in_Fy[w] = NULL;
    if (inflow_c) {
        int L = gc.nx > gc.ny ? gc.nx : gc.ny;
        for (int w = 0; w < 4; ++w)
            if (gc.bc[w] == BC_INFLOW) {
                gc.in_E[w] = inflow_c + (size_t)(w * 3 + 0) * L;
                gc.in_Fx[w] = inflow_c + (size_t)(w * 3 + 1) * L;
                gc.in_Fy[w] = inflow_c + (size_t)(w * 3 + 2) * L;
            }
    }
    #pragma omp parallel for collapse(2) schedule(static)
    for (int j = 0; j < gf.ny; ++j)
        for (int i = 0; i < gf.nx; ++i) store(&gf, fine, i, j, prolong_cell(&gc, coarse, i, j, gf.dim, kind));
}

int ora_prolong_correct(const int* idesc_f, const double* ddesc_f, const double* uc,
                        const double* vc, double* uf, double theta)
{
    grid_t gf, gc; grid_from_desc(&gf, idesc_f, ddesc_f, NULL); coarse_desc(&gf, &gc);
    return prolong_correct(&gc, &gf, uc, vc, uf, theta);
}

/* ------------------------------------------------------------------------ */
/* The grid hierarchy, Section 4.2: level l has nx/2^l (x ny/2^l in 2D) cells of
 * size 2^l h.  [READING] L_max counts the grids including the fine one (Table 4:
 * 257^2 with L_max = 4 adds a 33^2 grid to L_max = 3; Section 5.1: L_max = 1 is
 * plain Jacobi), so levels are 0 .. L_max-1.  Opacities of level l+1 are the
 * full-weighting restriction of those of level l; inflow ghost profiles are
 * restricted along the wall with weights 1/4, 1/2, 1/4 (ends copied). */
typedef struct {
    grid_t g;
    double *sa, *ss, *inflow;
    double *v, *u, *f, *r, *tmp, *tmp2;
} level_t;

static void restrict_profile(const double* fine, int nf, double* coarse, int nc)
{
    for (int i = 0; i < nc; ++i) {
        int a = 2 * i - 1 < 0 ? 0 : 2 * i - 1, b = 2 * i, c = 2 * i + 1 >= nf ? nf - 1 : 2 * i + 1;
        coarse[i] = nc == nf ? fine[i] : 0.25 * fine[a] + 0.5 * fine[b] + 0.25 * fine[c];
    }
}

static void build_levels(level_t* lv, int L, const grid_t* g0, const double* sa, const double* ss)
{
    for (int l = 0; l < L; ++l) {
        level_t* q = &lv[l];
        if (l == 0) q->g = *g0; else coarse_desc(&lv[l - 1].g, &q->g);
        size_t n = (size_t)q->g.nx * q->g.ny;
        q->sa = malloc(n * sizeof(double)); q->ss = malloc(n * sizeof(double));
        q->v = calloc(4 * n, sizeof(double)); q->u = calloc(4 * n, sizeof(double));
        q->f = calloc(4 * n, sizeof(double)); q->r = calloc(4 * n, sizeof(double));
        q->tmp = calloc(4 * n, sizeof(double)); q->tmp2 = calloc(4 * n, sizeof(double));
        int Lp = q->g.nx > q->g.ny ? q->g.nx : q->g.ny;
        q->inflow = calloc((size_t)12 * Lp, sizeof(double));
        if (l == 0) {
            memcpy(q->sa, sa, n * sizeof(double)); memcpy(q->ss, ss, n * sizeof(double));
            for (int w = 0; w < 4; ++w)
                if (g0->bc[w] == BC_INFLOW) {
                    int len = w < 2 ? g0->ny : g0->nx;
                    memcpy(q->inflow + (size_t)(w * 3 + 0) * Lp, g0->in_E[w], len * sizeof(double));
                    memcpy(q->inflow + (size_t)(w * 3 + 1) * Lp, g0->in_Fx[w], len * sizeof(double));
                    memcpy(q->inflow + (size_t)(w * 3 + 2) * Lp, g0->in_Fy[w], len * sizeof(double));
                }
        } else {
            level_t* p = &lv[l - 1];
            restrict_scalar(&p->g, &q->g, p->sa, q->sa);
            restrict_scalar(&p->g, &q->g, p->ss, q->ss);
            int Lf = p->g.nx > p->g.ny ? p->g.nx : p->g.ny;
            for (int w = 0; w < 4; ++w)
                if (g0->bc[w] == BC_INFLOW) {
                    int nf = w < 2 ? p->g.ny : p->g.nx, nc = w < 2 ? q->g.ny : q->g.nx;
                    for (int fld = 0; fld < 3; ++fld)
                        restrict_profile(p->inflow + (size_t)(w * 3 + fld) * Lf, nf,
                                         q->inflow + (size_t)(w * 3 + fld) * Lp, nc);
                }
        }
        for (int w = 0; w < 4; ++w) {
            if (q->g.bc[w] == BC_INFLOW) {
                q->g.in_E[w] = q->inflow + (size_t)(w * 3 + 0) * Lp;
                q->g.in_Fx[w] = q->inflow + (size_t)(w * 3 + 1) * Lp;
                q->g.in_Fy[w] = q->inflow + (size_t)(w * 3 + 2) * Lp;
            }
        }
    }
}

static void free_levels(level_t* lv, int L)
{
    for (int l = 0; l < L; ++l) {
        free(lv[l].sa); free(lv[l].ss); free(lv[l].inflow);
        free(lv[l].v); free(lv[l].u); free(lv[l].f); free(lv[l].r); free(lv[l].tmp); free(lv[l].tmp2);
    }
}

/* Sizes of levels 0..L-1; returns -1 if a level above the coarsest is odd. */
int ora_level_sizes(const int* idesc, int L, int* nx_out, int* ny_out)
{
    int nx = idesc[1], ny = idesc[2];
    for (int l = 0; l < L; ++l) {
        nx_out[l] = nx; ny_out[l] = ny;
        if (nx % 2 || (idesc[0] == 2 && ny % 2)) return l + 1 < L ? -1 : 0;
        nx /= 2; if (idesc[0] == 2) ny /= 2;
    }
    return 0;
}

/* Level-l residual r = rhs - A_l(u). */
static void level_residual(level_t* q, double dt, const double* rhs, const double* u, double* r)
{
    size_t n = (size_t)q->g.nx * q->g.ny;
    #pragma omp parallel for collapse(2) schedule(static)
    for (int j = 0; j < q->g.ny; ++j)
        for (int i = 0; i < q->g.nx; ++i) {
            size_t k = (size_t)j * q->g.nx + i;
            cell_t a = apply_A_cell(&q->g, dt, q->sa, q->ss, u, i, j);
            r[k] = rhs[k] - a.E; r[n + k] = rhs[n + k] - a.Fx;
            r[2 * n + k] = rhs[2 * n + k] - a.Fy; r[3 * n + k] = rhs[3 * n + k] - a.T;
        }
}

/* FAS right-hand side of a coarse level, Eq. (24)/(28): f_l = A_l(v_l) + r_l. */
static void fas_rhs(level_t* q, double dt)
{
    size_t n = (size_t)q->g.nx * q->g.ny;
    #pragma omp parallel for collapse(2) schedule(static)
    for (int j = 0; j < q->g.ny; ++j)
        for (int i = 0; i < q->g.nx; ++i) {
            size_t k = (size_t)j * q->g.nx + i;
            cell_t a = apply_A_cell(&q->g, dt, q->sa, q->ss, q->v, i, j);
            q->f[k] = a.E + q->r[k];
            q->f[n + k] = a.Fx + q->r[n + k];
            q->f[2 * n + k] = a.Fy + q->r[2 * n + k];
            q->f[3 * n + k] = a.T + q->r[3 * n + k];
        }
}

/* nu fine-level Jacobi sweeps on A(u) = b (Algorithm 1), u updated in place. */
static int fine_jacobi(level_t* q, double dt, const double* b, double* u, int nu)
{
    size_t n = (size_t)q->g.nx * q->g.ny;
    int worst = 0;
    for (int s = 0; s < nu; ++s) {
        int r = jacobi_sweep(&q->g, dt, q->sa, q->ss, b, u, q->tmp, 0.0, 1.0);
        if (r < 0) worst = -1;
        memcpy(u, q->tmp, 4 * n * sizeof(double));
    }
    return worst;
}

/* ------------------------------------------------------------------------ */
/* Cycle shapes.  Section 4.2 builds the V-cycle by applying the two-grid FAS
 * correction recursively down to the coarsest grid; Section 6.3 names the W-
 * and F-cycles as the unexplored alternatives.  A visit of coarse level l takes
 * its FAS problem A_l(u_l) = f_l from the restriction made by level l - 1 when
 * it is fresh (f_l = A_l(v_l) + r_l, u_l = v_l, Eq. (24)), or keeps f_l and the
 * current u_l when it is a repeated visit; it pre-smooths, restricts to level
 * l + 1, applies the coarse-grid corrections of level l + 1, prolongates the
 * correction (Eq. (34)) and post-smooths.  The coarse-grid corrections of
 * level l are [READING]: V, one visit of level l + 1; W, two visits (the second
 * repeated: the standard gamma = 2 recursion); F, a fresh F-visit followed by a
 * repeated V-visit; the coarsest level, solved by pseudo-time stepping, is
 * visited once per correction whatever the shape.  With L_max <= 2 the three
 * shapes are the same cycle. */
enum { CYCLE_V = 0, CYCLE_W = 1, CYCLE_F = 2 };

typedef struct {
    double dt, dtau, th_ex, th_c;
    int m, mc, nul, literal, L;
    int newton_fail, damped;
    double* visits;               /* visits of each level, summed over the step */
} cycle_ctx_t;

static void coarse_visit(level_t* lv, int l, int fresh, int shape, cycle_ctx_t* c);

static void coarse_corrections(level_t* lv, int l, int shape, cycle_ctx_t* c)
{
    if (l + 1 == c->L - 1 || shape == CYCLE_V) {
        coarse_visit(lv, l + 1, 1, shape, c);
    } else if (shape == CYCLE_W) {
        coarse_visit(lv, l + 1, 1, CYCLE_W, c);
        coarse_visit(lv, l + 1, 0, CYCLE_W, c);
    } else {
        coarse_visit(lv, l + 1, 1, CYCLE_F, c);
        coarse_visit(lv, l + 1, 0, CYCLE_V, c);
    }
}

static void coarse_visit(level_t* lv, int l, int fresh, int shape, cycle_ctx_t* c)
{
    level_t* q = &lv[l];
    size_t n = (size_t)q->g.nx * q->g.ny;
    c->visits[l] += 1.0;
    if (fresh) {
        fas_rhs(q, c->dt);
        memcpy(q->u, q->v, 4 * n * sizeof(double));
    }
    if (l == c->L - 1) {
        if (pseudo_time_smooth(&q->g, c->dt, q->sa, q->ss, q->f, q->u, c->dtau, c->mc, c->nul, c->th_ex) < 0)
            ++c->newton_fail;
        return;
    }
    level_t* p = &lv[l + 1];
    if (pseudo_time_smooth(&q->g, c->dt, q->sa, q->ss, q->f, q->u, c->dtau, c->m, c->nul, c->th_ex) < 0)
        ++c->newton_fail;
    level_residual(q, c->dt, q->f, q->u, q->r);                /* r_bar = f - A(u) */
    restrict_state(&q->g, &p->g, c->literal ? q->v : q->u, p->v, KIND_STATE);
    restrict_state(&q->g, &p->g, q->r, p->r, KIND_DIFF);
    coarse_corrections(lv, l, shape, c);
    if (c->literal) memcpy(q->u, q->v, 4 * n * sizeof(double));
    c->damped += prolong_correct(&p->g, &q->g, p->u, p->v, q->u, c->th_c);
    if (pseudo_time_smooth(&q->g, c->dt, q->sa, q->ss, q->f, q->u, c->dtau, c->m, c->nul, c->th_ex) < 0)
        ++c->newton_fail;
}

/* ------------------------------------------------------------------------ */
/* Appendix A, Algorithm 4: one implicit time step, v^n -> v^{n+1}.
 *
 * Parameters (ip / dp arrays, Section 5 defaults in parentheses):
 *   ip = { L_max, nu0 (3), nu_l (1), m (3), m_coarse (3), max_cycles, literal_fas,
 *          dtau_rule, cycle shape (0 V, 1 W, 2 F; see coarse_corrections) }
 *   dp = { dtau0 (1e-3), grow (1.1), shrink (0.5), eps_i, eps_d, tol,
 *          dtau_min, dtau_max, theta_ex (1/2), theta_c (1/2) }
 * The state v (4 planes) holds v^n on entry, v^{n+1} on return; b = (E^n, F^n,
 * C_v T^n).  Cycle loop [READINGS]:
 *  - r_0 = b - A(v^n); stop at once if ||r_0|| <= 1e-14 diag ||b||, with
 *    diag = 1 + c dt/hx (+ c dt/hy) the transport diagonal (rounding floor);
 *  - cycle kappa = 1, 2, ...: down leg l = 0 .. L-2 (pre-smooth, residual,
 *    restriction of the smoothed iterate u_l and of the residual: standard FAS,
 *    Algorithm 2), coarsest level L-1 (pseudo-time solve; plain Jacobi sweeps
 *    when L = 1), up leg l = L-2 .. 0 (prolongation + damping of the correction
 *    applied to u_l, Eq. (34), then post-smoothing);
 *  - after the cycle r_kappa = b - A(v); stop when ||r_kappa|| <= tol ||r_0||;
 *    delta = | ||r_kappa|| - ||r_{kappa-1}|| | / ||r_0||; dtau *= grow if
 *    delta > eps_i, dtau *= shrink if delta < eps_d; clamp to [dtau_min, dtau_max].
 *    dtau_rule = 1 takes the signed decrease delta = (||r_{kappa-1}|| - ||r_kappa||)
 *    / ||r_0|| instead, the reading of the prose of Section 4 (increase when the
 *    residual decreases fast enough, decrease when it decreases slowly), so that
 *    a growing residual shrinks dtau; Algorithm 4 prints the absolute change.
 *  - literal_fas = 1 restricts and corrects the unsmoothed v_l instead (the
 *    letter of Algorithm 4), kept only for comparison (V-cycles only).
 * Outputs: stats = { cycles, res0, res, dtau, fine_sweeps, status, newton_fail,
 *   damped_cells, visits of level 0 .. L_max - 1 summed over the step }, res_hist[kappa] = ||r_kappa|| (kappa = 0..cycles, length
 *   max_cycles+1), dtau_hist[kappa-1] = dtau used in cycle kappa.
 * status: 0 converged, -4 not converged after max_cycles, -2 inadmissible input,
 * -1 invalid parameters (an unknown cycle shape, or literal_fas with W or F). */
int ora_implicit_step(const int* idesc, const double* ddesc, const double* inflow, double dt,
                      const double* sa, const double* ss, const int* ip, const double* dp,
                      double* v, double* stats, double* res_hist, double* dtau_hist)
{
    grid_t g0; grid_from_desc(&g0, idesc, ddesc, inflow);
    int L = ip[0], nu0 = ip[1], nul = ip[2], m = ip[3], mc = ip[4], maxc = ip[5], literal = ip[6];
    int signed_rule = ip[7], shape = ip[8];
    double dtau = dp[0], grow = dp[1], shrink = dp[2], eps_i = dp[3], eps_d = dp[4], tol = dp[5];
    double dtau_min = dp[6], dtau_max = dp[7], th_ex = dp[8], th_c = dp[9];
    if (shape < CYCLE_V || shape > CYCLE_F || (literal && shape != CYCLE_V)) {
        stats[5] = -1; return -1;
    }
    size_t n0 = (size_t)g0.nx * g0.ny;
    for (size_t k = 0; k < n0; ++k) {
        cell_t s = load(&g0, v, (int)(k % g0.nx), (int)(k / g0.nx));
        if (!(s.E > 0.0 && s.T > 0.0 && s.Fx * s.Fx + s.Fy * s.Fy <= s.E * s.E * g0.c * g0.c * (1.0 + ADM_SLACK))) {
            stats[5] = -2; return -2;
        }
    }
    level_t* lv = calloc((size_t)L, sizeof(level_t));
    build_levels(lv, L, &g0, sa, ss);
    level_t* q0 = &lv[0];
    double* visits = stats + 8;
    for (int l = 0; l < L; ++l) visits[l] = 0.0;
    /* Algorithm 4: b^h = v^n (E, F; [EXT] C_v T^n for the gas row), v_(0) = v^n. */
    double* b = malloc(4 * n0 * sizeof(double));
    memcpy(b, v, 4 * n0 * sizeof(double));
    for (size_t k = 0; k < n0; ++k) b[3 * n0 + k] = g0.c_v * v[3 * n0 + k];
    memcpy(q0->v, v, 4 * n0 * sizeof(double));

    double bnorm = ora_norm(idesc, ddesc, b);
    level_residual(q0, dt, b, q0->v, q0->r);
    double res0 = ora_norm(idesc, ddesc, q0->r), res_prev = res0, res = res0;
    res_hist[0] = res0;
    int kappa = 0, status = 0, newton_fail = 0, damped = 0;
    long long fine_sweeps = 0;

    /* [READING] a right-hand side already solved to rounding: ||r_0|| below
     * 1e-14 (1 + c dt/hx + c dt/hy) ||b||, the rounding floor of evaluating A */
    if (res0 > 1e-14 * transport_diag(&g0, dt) * bnorm) {
        status = -4;
        while (kappa < maxc) {
            /* ---- fine level (Algorithm 1 sweeps), then the coarse-grid
             * corrections of the cycle's shape ---- */
            memcpy(q0->u, q0->v, 4 * n0 * sizeof(double));
            visits[0] += 1.0;
            if (fine_jacobi(q0, dt, b, q0->u, nu0) < 0) ++newton_fail;
            fine_sweeps += nu0;
            if (L > 1) {
                level_t* p = &lv[1];
                cycle_ctx_t c = { dt, dtau, th_ex, th_c, m, mc, nul, literal, L, 0, 0, visits };
                level_residual(q0, dt, b, q0->u, q0->r);
                restrict_state(&q0->g, &p->g, literal ? q0->v : q0->u, p->v, KIND_STATE);
                restrict_state(&q0->g, &p->g, q0->r, p->r, KIND_DIFF);
                coarse_corrections(lv, 0, shape, &c);
                if (literal) memcpy(q0->u, q0->v, 4 * n0 * sizeof(double));
                c.damped += prolong_correct(&p->g, &q0->g, p->u, p->v, q0->u, th_c);
                if (fine_jacobi(q0, dt, b, q0->u, nu0) < 0) ++c.newton_fail;
                fine_sweeps += nu0;
                newton_fail += c.newton_fail;
                damped += c.damped;
            }
            /* ---- end of cycle: v <- u, residual, pseudo-time step control ---- */
            memcpy(q0->v, q0->u, 4 * n0 * sizeof(double));
            level_residual(q0, dt, b, q0->v, q0->r);
            ++kappa;
            res = ora_norm(idesc, ddesc, q0->r);
            res_hist[kappa] = res;
            dtau_hist[kappa - 1] = dtau;
            if (res <= tol * res0) { status = 0; break; }
            double delta = (signed_rule ? res_prev - res : fabs(res - res_prev)) / res0;
            if (delta > eps_i) dtau *= grow;
            if (delta < eps_d) dtau *= shrink;
            if (dtau < dtau_min) dtau = dtau_min;
            if (dtau > dtau_max) dtau = dtau_max;
            res_prev = res;
        }
    }
    memcpy(v, q0->v, 4 * n0 * sizeof(double));
    stats[0] = kappa; stats[1] = res0; stats[2] = res; stats[3] = dtau;
    stats[4] = (double)fine_sweeps; stats[5] = status; stats[6] = newton_fail; stats[7] = damped;
    free(b);
    free_levels(lv, L);
    free(lv);
    return status;
}
