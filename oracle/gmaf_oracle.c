/*
 * GMAF oracle: a plain, slow, FP64 CPU restatement of the piston-gap hot path
 * of "A GPU-boosted high-performance multi-working condition joint analysis
 * framework for predicting dynamics of textured axial piston pump"
 * (arXiv 2511.06824).
 *
 * THIS FILE IS TEST INFRASTRUCTURE.  Only the test-suite, the smoke check and
 * the benchmark's CPU-baseline leg may load it.  The CUDA library never links,
 * includes or calls it, and it shares no code, header, table or constant
 * generator with the CUDA library.
 *
 * Every function below follows the paper's steps in the paper's order.  Where
 * the paper is silent the reading adopted is stated at the function (the same
 * readings are listed in the design notes of the repository).
 *
 * Pins: every function is checked by the CPU test-suite against something other
 * than itself - closed forms, dense library solves and factorisations, brute
 * force, invariants and convergence orders.  None is checked against a worked
 * numeric example of the paper, which prints none: the whole path is parity
 * unpinned against the paper's own numbers.
 *
 * Build: gcc -O2 -std=c11 -ffp-contract=off -fopenmp -fPIC -shared -o liboracle.so gmaf_oracle.c -lm
 * (-ffp-contract=off: no fused multiply-add, so x86-64 and aarch64 give the
 * same bits.  -fopenmp is optional: without it every loop runs on one thread.)
 *
 * Threads: one by default.  oracle_set_threads(n) lets the loops whose
 * iterations are independent (assembly per cell, sparse products per row,
 * element-wise vector updates, the preconditioner's passes) run on n threads.
 * Each output element is computed by the same arithmetic whichever thread runs
 * it, and every reduction (dot products, norms, load integrals) stays a plain
 * sequential loop, so the results are bitwise the same for any thread count.
 *
 * Parameter arrays (plain doubles, so the oracle has no struct in common with
 * the CUDA library):
 *   phys[7]  = { R_k, L, c, mu, v_slide, p_chamber, p_case }
 *              R_k piston radius [m], L gap (coupling) length [m], c radial
 *              clearance [m] (R_c = R_k + c), mu viscosity [Pa s], v_slide
 *              axial speed of the piston relative to the bore (+z = chamber
 *              to case) [m/s], Dirichlet pressures at z = 0 and z = L [Pa].
 *   tex[6]   = { kind, radius, depth, area_density, offset_theta, offset_z }
 *              kind 0 smooth, 1 hexagonal lattice of flat-bottom circular
 *              dimples; offsets in metres on the unwrapped surface.
 *   state[8] = { e1, e2, e3, e4, edot1, edot2, edot3, edot4 }
 *              e1, e2 at z = 0, e3, e4 at z = L (Eq. 2.3) [m], rates [m/s].
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_PI 3.14159265358979323846

enum { OR_OK = 0, OR_INVALID = -1, OR_CONTACT = -2, OR_NOT_CONVERGED = -3,
       OR_NONFINITE = -4, OR_NOMEM = -5 };

/* Threads of the independent-iteration loops (see the header). */
static int g_threads = 1;
#define OR_PAR_MIN 8192   /* loops shorter than this stay on one thread */

/* Set the thread count (n < 1: all processors); returns the count in effect. */
int oracle_set_threads(int n)
{
#ifdef _OPENMP
    g_threads = n >= 1 ? n : omp_get_num_procs();
#else
    (void)n;
    g_threads = 1;
#endif
    return g_threads;
}

/* Processors available to the loops (1 when built without OpenMP). */
int oracle_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_num_procs();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------------ */
/* Texture (Eq. 2.3 h_Text; Fig. 10 is missing from the text, so the layout  */
/* is the hexagonal dimple lattice read in the design notes).                */
/* ------------------------------------------------------------------------ */

typedef struct {
    int on;
    double r, depth, oth, oz;
    double ath, az;          /* lattice pitch along x (circumference) and z */
} lattice;

static lattice make_lattice(const double *tex, double Rk)
{
    lattice lt;
    memset(&lt, 0, sizeof lt);
    if (tex == NULL || tex[0] == 0.0 || tex[2] == 0.0) return lt;
    lt.on = 1;
    lt.r = tex[1];
    lt.depth = tex[2];
    lt.oth = tex[4];
    lt.oz = tex[5];
    double rho = tex[3];
    double circ = 2.0 * OR_PI * Rk;
    /* ideal hexagonal spacing for area density rho: pi r^2 / (a0 * a0*sqrt(3)/2) = rho */
    double a0 = lt.r * sqrt(2.0 * OR_PI / (sqrt(3.0) * rho));
    double ncol = round(circ / a0);
    if (ncol < 1.0) ncol = 1.0;
    lt.ath = circ / ncol;                        /* whole number of columns */
    lt.az = OR_PI * lt.r * lt.r / (rho * lt.ath); /* exact density rho     */
    return lt;
}

/* Depth of the texture at unwrapped position (x, z).  A point is inside a
 * dimple when its distance to the nearest lattice centre is strictly below the
 * radius.  Row k has centres at z = oz + k az and x = oth + (k odd) ath/2 + m ath.
 * Rows k0-1 .. k0+2 around the point are examined. */
static double texture_depth(const lattice *lt, double x, double z)
{
    if (!lt->on) return 0.0;
    double k0 = floor((z - lt->oz) / lt->az);
    for (int dk = -1; dk <= 2; ++dk) {
        double k = k0 + (double)dk;
        double zc = lt->oz + k * lt->az;
        double dz = z - zc;
        long long ki = (long long)k;
        double shift = (ki & 1LL) ? 0.5 * lt->ath : 0.0;
        double u = x - lt->oth - shift;
        double m = floor(u / lt->ath);
        double dxa = u - m * lt->ath;
        double dxb = u - (m + 1.0) * lt->ath;
        double r2 = lt->r * lt->r;
        if (dxa * dxa + dz * dz < r2) return lt->depth;
        if (dxb * dxb + dz * dz < r2) return lt->depth;
    }
    return 0.0;
}

/* ------------------------------------------------------------------------ */
/* Film thickness, Eq. 2.3, and its rate dh/dt = sum_i dh/de_i edot_i.        */
/* z = 0 is the chamber end and carries e1, e2; z = L carries e3, e4.        */
/* ------------------------------------------------------------------------ */

static double film(const double *phys, const lattice *lt, const double *e,
                   double theta, double z)
{
    double Rk = phys[0], L = phys[1], c = phys[2];
    double Rc = Rk + c;
    double t = z / L;
    double ex = e[0] + (e[2] - e[0]) * t;
    double ey = e[1] + (e[3] - e[1]) * t;
    double X = Rc * cos(theta) - ex;
    double Y = Rc * sin(theta) - ey;
    double h = sqrt(X * X + Y * Y) - Rk;
    return h + texture_depth(lt, Rk * theta, z);
}

static double film_rate(const double *phys, const double *e, const double *ed,
                        double theta, double z)
{
    double Rk = phys[0], L = phys[1], c = phys[2];
    double Rc = Rk + c;
    double t = z / L;
    double ex = e[0] + (e[2] - e[0]) * t;
    double ey = e[1] + (e[3] - e[1]) * t;
    double X = Rc * cos(theta) - ex;
    double Y = Rc * sin(theta) - ey;
    double rho = sqrt(X * X + Y * Y);
    /* dh/dex = -X/rho, dh/dey = -Y/rho; dex/de1 = 1-t, dex/de3 = t, likewise y */
    double exd = ed[0] * (1.0 - t) + ed[2] * t;
    double eyd = ed[1] * (1.0 - t) + ed[3] * t;
    return -(X / rho) * exd - (Y / rho) * eyd;
}

double oracle_film(const double *phys, const double *tex, const double *e,
                   double theta, double z)
{
    lattice lt = make_lattice(tex, phys[0]);
    return film(phys, &lt, e, theta, z);
}

double oracle_film_rate(const double *phys, const double *e, const double *ed,
                        double theta, double z)
{
    return film_rate(phys, e, ed, theta, z);
}

double oracle_texture_depth(const double *phys, const double *tex, double x, double z)
{
    lattice lt = make_lattice(tex, phys[0]);
    return texture_depth(&lt, x, z);
}

void oracle_lattice(const double *phys, const double *tex, double out[2])
{
    lattice lt = make_lattice(tex, phys[0]);
    out[0] = lt.ath;
    out[1] = lt.az;
}

/* ------------------------------------------------------------------------ */
/* FVM assembly (Eq. 2.1, 2.4; compressed diagonals Eq. 2.5-2.7).             */
/*                                                                          */
/* Reynolds equation in the piston frame (not printed in the paper; reading):*/
/*   div( h^3/(12 mu) grad p ) = (U_b/2) dh/dz + dh/dt,  U_b = -v_slide,     */
/* on the unwrapped gap x = R_k theta (periodic), z in [0, L] (Dirichlet).   */
/* Cell-centred finite volumes on nth x nz cells, theta fastest.  Face       */
/* conductances use h at the face midpoints.  Row P:                         */
/*   A_P p_P - a_E p_E - a_W p_W - a_N p_N - a_S p_S = S_P                    */
/* with a_E = g_e dz/dx, a_N = g_n dx/dz, g = h^3/(12 mu), A_P = sum a (+ the */
/* half-cell Dirichlet conductance 2 g dx/dz at z = 0 and z = L), and        */
/*   S_P = -(U_b/2)(h_n - h_s) dx - hdot_P dx dz + Dirichlet terms.          */
/* Storage: D = A_P, aE (coupling to i+1, wrap at nth-1), aN (coupling to    */
/* j+1, zero in the last row).  a_W(i) = aE(i-1), a_S(j) = aN(j-1).          */
/* Returns OR_CONTACT when any film thickness used is <= 0.                  */
/* ------------------------------------------------------------------------ */

int oracle_assemble(int nth, int nz, const double *phys, const double *tex,
                    const double *state, double *D, double *aE, double *aN,
                    double *S)
{
    if (nth < 3 || nz < 2 || !phys || !state || !D || !aE || !aN || !S)
        return OR_INVALID;
    double Rk = phys[0], L = phys[1], mu = phys[3], v = phys[4];
    double pch = phys[5], pcase = phys[6];
    double Ub = -v;
    lattice lt = make_lattice(tex, Rk);
    const double *e = state, *ed = state + 4;
    double dth = 2.0 * OR_PI / (double)nth;
    double dx = Rk * dth;
    double dz = L / (double)nz;
    int contact = 0;
    size_t n = (size_t)nth * (size_t)nz;
    double *aB = (double *)calloc(n, sizeof(double));
    if (!aB) return OR_NOMEM;

#pragma omp parallel for schedule(static) num_threads(g_threads) reduction(| : contact) if (n >= OR_PAR_MIN)
    for (int j = 0; j < nz; ++j) {
        for (int i = 0; i < nth; ++i) {
            size_t P = (size_t)i + (size_t)nth * (size_t)j;
            double thc = ((double)i + 0.5) * dth;
            double the = ((double)i + 1.0) * dth;
            double zc = ((double)j + 0.5) * dz;
            double zn = ((double)j + 1.0) * dz;
            double zs = (double)j * dz;
            double he = film(phys, &lt, e, the, zc);
            double hn = film(phys, &lt, e, thc, zn);
            double hs = film(phys, &lt, e, thc, zs);
            if (he <= 0.0 || hn <= 0.0 || hs <= 0.0) contact = 1;
            double ge = he * he * he / (12.0 * mu);
            double gn = hn * hn * hn / (12.0 * mu);
            double gs = hs * hs * hs / (12.0 * mu);
            aE[P] = ge * dz / dx;
            aN[P] = (j < nz - 1) ? gn * dx / dz : 0.0;
            double b = 0.0, sb = 0.0;
            if (j == 0) {               /* Dirichlet face z = 0 at distance dz/2 */
                double a = gs * dx / (0.5 * dz);
                b += a;
                sb += a * pch;
            }
            if (j == nz - 1) {          /* Dirichlet face z = L at distance dz/2 */
                double a = gn * dx / (0.5 * dz);
                b += a;
                sb += a * pcase;
            }
            aB[P] = b;
            double hdot = film_rate(phys, e, ed, thc, zc);
            S[P] = -(Ub / 2.0) * (hn - hs) * dx - hdot * dx * dz + sb;
        }
    }
#pragma omp parallel for schedule(static) num_threads(g_threads) if (n >= OR_PAR_MIN)
    for (int j = 0; j < nz; ++j) {
        for (int i = 0; i < nth; ++i) {
            size_t P = (size_t)i + (size_t)nth * (size_t)j;
            size_t W = (size_t)((i + nth - 1) % nth) + (size_t)nth * (size_t)j;
            double aW = aE[W];
            double aS = (j > 0) ? aN[P - (size_t)nth] : 0.0;
            D[P] = aE[P] + aW + aN[P] + aS + aB[P];
        }
    }
    free(aB);
    return contact ? OR_CONTACT : OR_OK;
}

/* ------------------------------------------------------------------------ */
/* The matrix as a generic sparse matrix (CSR), built from the stencil.       */
/* The ASSOR factors use L = the strictly lower triangle of A in the global   */
/* index order idx = i + nth*j (Eq. 3.8, theta fastest), read off the CSR    */
/* by column < row, with no stencil-specific rule.                           */
/* ------------------------------------------------------------------------ */

typedef struct {
    size_t n;
    size_t *rowptr;
    size_t *col;
    double *val;
} csr;

static void csr_free(csr *m)
{
    free(m->rowptr);
    free(m->col);
    free(m->val);
    memset(m, 0, sizeof *m);
}

static int csr_build(int nth, int nz, const double *D, const double *aE,
                     const double *aN, csr *m)
{
    size_t n = (size_t)nth * (size_t)nz;
    m->n = n;
    m->rowptr = (size_t *)malloc((n + 1) * sizeof(size_t));
    m->col = (size_t *)malloc(5 * n * sizeof(size_t));
    m->val = (double *)malloc(5 * n * sizeof(double));
    if (!m->rowptr || !m->col || !m->val) { csr_free(m); return OR_NOMEM; }
    size_t k = 0;
    for (int j = 0; j < nz; ++j) {
        for (int i = 0; i < nth; ++i) {
            size_t P = (size_t)i + (size_t)nth * (size_t)j;
            size_t E = (size_t)((i + 1) % nth) + (size_t)nth * (size_t)j;
            size_t W = (size_t)((i + nth - 1) % nth) + (size_t)nth * (size_t)j;
            m->rowptr[P] = k;
            if (j > 0) { m->col[k] = P - (size_t)nth; m->val[k] = -aN[P - (size_t)nth]; ++k; }
            m->col[k] = W; m->val[k] = -aE[W]; ++k;
            m->col[k] = P; m->val[k] = D[P]; ++k;
            m->col[k] = E; m->val[k] = -aE[P]; ++k;
            if (j < nz - 1) { m->col[k] = P + (size_t)nth; m->val[k] = -aN[P]; ++k; }
        }
    }
    m->rowptr[n] = k;
    return OR_OK;
}

/* y = A x (part 0 = whole row, part -1 = strictly lower, part +1 = strictly upper) */
static void csr_apply(const csr *m, int part, const double *x, double *y)
{
#pragma omp parallel for schedule(static) num_threads(g_threads) if (m->n >= OR_PAR_MIN)
    for (size_t r = 0; r < m->n; ++r) {
        double s = 0.0;
        for (size_t k = m->rowptr[r]; k < m->rowptr[r + 1]; ++k) {
            size_t c = m->col[k];
            if (part < 0 && c >= r) continue;
            if (part > 0 && c <= r) continue;
            s += m->val[k] * x[c];
        }
        y[r] = s;
    }
}

/* Dense copy of one condition's matrix (row-major n x n), for small checks. */
int oracle_dense_matrix(int nth, int nz, const double *D, const double *aE,
                        const double *aN, double *out)
{
    csr m;
    int st = csr_build(nth, nz, D, aE, aN, &m);
    if (st) return st;
    memset(out, 0, m.n * m.n * sizeof(double));
    for (size_t r = 0; r < m.n; ++r)
        for (size_t k = m.rowptr[r]; k < m.rowptr[r + 1]; ++k)
            out[r * m.n + m.col[k]] += m.val[k];
    csr_free(&m);
    return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* Joint system A_G p_G = S_G (Eq. 3.7-3.8): ncond blocks, system-major      */
/* {p_G}[i + j n] = {p_j}[i].                                                 */
/* ------------------------------------------------------------------------ */

typedef struct {
    int nth, nz, ncond;
    size_t n;
    csr *blk;
    const double *D;
} joint;

static void joint_free(joint *J)
{
    if (J->blk) {
        for (int c = 0; c < J->ncond; ++c) csr_free(&J->blk[c]);
        free(J->blk);
    }
    J->blk = NULL;
}

static int joint_build(int nth, int nz, int ncond, const double *D,
                       const double *aE, const double *aN, joint *J)
{
    J->nth = nth; J->nz = nz; J->ncond = ncond;
    J->n = (size_t)nth * (size_t)nz;
    J->D = D;
    J->blk = (csr *)calloc((size_t)ncond, sizeof(csr));
    if (!J->blk) return OR_NOMEM;
    for (int c = 0; c < ncond; ++c) {
        size_t o = (size_t)c * J->n;
        int st = csr_build(nth, nz, D + o, aE + o, aN + o, &J->blk[c]);
        if (st) { joint_free(J); return st; }
    }
    return OR_OK;
}

static void joint_apply(const joint *J, int part, const double *x, double *y)
{
    for (int c = 0; c < J->ncond; ++c) {
        size_t o = (size_t)c * J->n;
        csr_apply(&J->blk[c], part, x + o, y + o);
    }
}

/* Preconditioner application z = M^-1 r.
 *  precond 0: Jacobi, M = D (Eq. 2.8).
 *  precond 1: ASSOR-II (Eq. 3.3-3.6), in the paper's two steps:
 *     v = (I - w D^-1 L) D^-1 r                      (Eq. 3.5)
 *     z = (2 - w) w (I - w D^-1 L^T) v               (Eq. 3.6)
 *  L^T is applied as the strictly upper triangle of A (A is symmetric).
 *  precond 2: ASSOR-I (Eq. 3.2), a diagonal preconditioner:
 *     {M^-1}_ii = w (2 - w) / {(D + w L) D^-1 (D + w L)^T}_ii,
 *  where, B = D + w L being lower triangular with diagonal D,
 *     {B D^-1 B^T}_ii = sum_k B_ik^2 / D_k = D_i + w^2 sum_{k < i} L_ik^2 / D_k. */
static void joint_precond(const joint *J, int precond, double omega,
                          const double *r, double *z, double *t1, double *t2)
{
    size_t N = J->n * (size_t)J->ncond;
    const double *D = J->D;
    if (precond == 0) {
#pragma omp parallel for schedule(static) num_threads(g_threads) if (N >= OR_PAR_MIN)
        for (size_t k = 0; k < N; ++k) z[k] = r[k] / D[k];
        return;
    }
    if (precond == 2) {
        for (int c = 0; c < J->ncond; ++c) {
            const csr *m = &J->blk[c];
            size_t o = (size_t)c * J->n;
#pragma omp parallel for schedule(static) num_threads(g_threads) if (m->n >= OR_PAR_MIN)
            for (size_t row = 0; row < m->n; ++row) {
                double s = 0.0;
                for (size_t k = m->rowptr[row]; k < m->rowptr[row + 1]; ++k) {
                    size_t col = m->col[k];
                    if (col >= row) continue;               /* strictly lower */
                    s += m->val[k] * m->val[k] / D[o + col];
                }
                double diag = D[o + row] + omega * omega * s;
                z[o + row] = omega * (2.0 - omega) * r[o + row] / diag;
            }
        }
        return;
    }
    /* t1 = D^-1 r */
#pragma omp parallel for schedule(static) num_threads(g_threads) if (N >= OR_PAR_MIN)
    for (size_t k = 0; k < N; ++k) t1[k] = r[k] / D[k];
    /* t2 = L t1 ; v = t1 - w D^-1 t2  (stored in t1's place via z) */
    joint_apply(J, -1, t1, t2);
#pragma omp parallel for schedule(static) num_threads(g_threads) if (N >= OR_PAR_MIN)
    for (size_t k = 0; k < N; ++k) z[k] = t1[k] - omega * (t2[k] / D[k]);
    /* t2 = L^T v ; z = (2-w) w (v - w D^-1 t2) */
    joint_apply(J, +1, z, t2);
    double c = (2.0 - omega) * omega;
#pragma omp parallel for schedule(static) num_threads(g_threads) if (N >= OR_PAR_MIN)
    for (size_t k = 0; k < N; ++k) z[k] = c * (z[k] - omega * (t2[k] / D[k]));
}

static double dot(size_t N, const double *a, const double *b)
{
    double s = 0.0;
    for (size_t k = 0; k < N; ++k) s += a[k] * b[k];
    return s;
}

int oracle_apply_matrix(int nth, int nz, int ncond, const double *D,
                        const double *aE, const double *aN, const double *x,
                        double *y)
{
    joint J;
    int st = joint_build(nth, nz, ncond, D, aE, aN, &J);
    if (st) return st;
    joint_apply(&J, 0, x, y);
    joint_free(&J);
    return OR_OK;
}

int oracle_apply_precond(int nth, int nz, int ncond, const double *D,
                         const double *aE, const double *aN, int precond,
                         double omega, const double *r, double *z)
{
    joint J;
    int st = joint_build(nth, nz, ncond, D, aE, aN, &J);
    if (st) return st;
    size_t N = J.n * (size_t)ncond;
    double *t1 = (double *)malloc(N * sizeof(double));
    double *t2 = (double *)malloc(N * sizeof(double));
    if (!t1 || !t2) { free(t1); free(t2); joint_free(&J); return OR_NOMEM; }
    joint_precond(&J, precond, omega, r, z, t1, t2);
    free(t1); free(t2);
    joint_free(&J);
    return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* Joint PCG, Table 1, on A_G with one set of scalars (alpha, beta, d are    */
/* sums over all blocks) and the synchronized criterion Eq. 3.9:             */
/*   ||r_G||_2 / ||S_G||_2 <= eps.                                           */
/* Readings: r0 = S - A p0 (Table 1 step 2 printed with the opposite sign,   */
/* which contradicts steps 4-5); the criterion is also tested on r0; the     */
/* in-loop test uses the recurrence residual; after exit the true residual   */
/* S - A p is formed and, if it exceeds 10 eps, the iteration restarts once  */
/* from the current p with the remaining iteration budget.  ||S|| = 0 gives  */
/* p = 0.                                                                    */
/* out[0] = recurrence relative residual at exit, out[1] = true relative     */
/* residual at exit.                                                         */
/* ------------------------------------------------------------------------ */

int oracle_solve_joint(int nth, int nz, int ncond, const double *D,
                       const double *aE, const double *aN, const double *S,
                       double *p, int precond, double omega, double eps,
                       int max_iter, int zero_init, int *iters_out,
                       double *out)
{
    if (nth < 3 || nz < 2 || ncond < 1 || !(eps > 0.0) || max_iter < 0 ||
        (precond != 0 && !(omega > 0.0 && omega < 2.0)) ||
        (precond != 0 && precond != 1 && precond != 2))
        return OR_INVALID;
    joint J;
    int st = joint_build(nth, nz, ncond, D, aE, aN, &J);
    if (st) return st;
    size_t N = J.n * (size_t)ncond;
    double *r = (double *)malloc(N * sizeof(double));
    double *z = (double *)malloc(N * sizeof(double));
    double *u = (double *)malloc(N * sizeof(double));
    double *v = (double *)malloc(N * sizeof(double));
    double *t1 = (double *)malloc(N * sizeof(double));
    double *t2 = (double *)malloc(N * sizeof(double));
    if (!r || !z || !u || !v || !t1 || !t2) { st = OR_NOMEM; goto done; }

    double normS = sqrt(dot(N, S, S));
    if (zero_init) memset(p, 0, N * sizeof(double));
    int iters = 0;
    double rel = 0.0, true_rel = 0.0;
    if (!isfinite(normS)) { st = OR_NONFINITE; goto done; }
    if (normS == 0.0) {
        memset(p, 0, N * sizeof(double));
        st = OR_OK;
        goto done;
    }
    int restarted = 0;
    for (;;) {
        /* step 1-2: r0 = S - A p0, z0 = M^-1 r0, u0 = z0, d0 = r0.z0 */
        joint_apply(&J, 0, p, v);
#pragma omp parallel for schedule(static) num_threads(g_threads) if (N >= OR_PAR_MIN)
        for (size_t k = 0; k < N; ++k) r[k] = S[k] - v[k];
        rel = sqrt(dot(N, r, r)) / normS;
        int converged = rel <= eps;
        if (!isfinite(rel)) { st = OR_NONFINITE; goto done; }
        if (!converged) {
            joint_precond(&J, precond, omega, r, z, t1, t2);
            memcpy(u, z, N * sizeof(double));
            double d = dot(N, r, z);
            while (iters < max_iter) {
                /* step 3: v = A u, alpha = d / u.v */
                joint_apply(&J, 0, u, v);
                double uv = dot(N, u, v);
                if (!isfinite(uv) || !isfinite(d) || !(uv > 0.0)) { st = OR_NONFINITE; goto done; }
                double alpha = d / uv;
                /* step 4-5 */
#pragma omp parallel for schedule(static) num_threads(g_threads) if (N >= OR_PAR_MIN)
                for (size_t k = 0; k < N; ++k) p[k] = p[k] + alpha * u[k];
#pragma omp parallel for schedule(static) num_threads(g_threads) if (N >= OR_PAR_MIN)
                for (size_t k = 0; k < N; ++k) r[k] = r[k] - alpha * v[k];
                ++iters;
                /* step 6: synchronized criterion, Eq. 3.9 */
                rel = sqrt(dot(N, r, r)) / normS;
                if (!isfinite(rel)) { st = OR_NONFINITE; goto done; }
                if (rel <= eps) { converged = 1; break; }
                /* step 7-9 */
                joint_precond(&J, precond, omega, r, z, t1, t2);
                double dn = dot(N, r, z);
                double beta = dn / d;
                d = dn;
#pragma omp parallel for schedule(static) num_threads(g_threads) if (N >= OR_PAR_MIN)
                for (size_t k = 0; k < N; ++k) u[k] = z[k] + beta * u[k];
            }
        }
        /* true residual */
        joint_apply(&J, 0, p, v);
#pragma omp parallel for schedule(static) num_threads(g_threads) if (N >= OR_PAR_MIN)
        for (size_t k = 0; k < N; ++k) t1[k] = S[k] - v[k];
        true_rel = sqrt(dot(N, t1, t1)) / normS;
        if (!isfinite(true_rel)) { st = OR_NONFINITE; goto done; }
        if (converged && true_rel <= 10.0 * eps) { st = OR_OK; break; }
        if (restarted || iters >= max_iter) { st = OR_NOT_CONVERGED; break; }
        restarted = 1;
    }
done:
    if (iters_out) *iters_out = iters;
    if (out) { out[0] = rel; out[1] = true_rel; }
    free(r); free(z); free(u); free(v); free(t1); free(t2);
    joint_free(&J);
    return st;
}

/* ------------------------------------------------------------------------ */
/* Loads, Sec. 2.4-III: force and moment from normal pressure and from       */
/* viscous shear, integrated on the surface elements bounded by the pressure */
/* nodes.  Nodes: the cell centres plus the two boundary lines z = 0 (p_ch)  */
/* and z = L (p_case), periodic in theta.  Elements: nth x (nz+1) rectangles */
/* between them (first and last have height dz/2).                           */
/*  - pressure: traction -p n, n = (cos t, sin t, 0); element value = mean   */
/*    of the integrand at its 4 corners times the element area R_k dth dz_e. */
/*  - shear: tau_z = -(h/2) dp/dz + mu U_b / h, tau_t = -(h/2) (1/R_k) dp/dt, */
/*    traction tau_t (-sin t, cos t, 0) + tau_z (0, 0, 1), with dp/dz, dp/dt */
/*    from differences of edge means and h (texture included) at the element */
/*    centre, times the element area.                                        */
/*  - moments: r x f about the bore axis at z = 0, r = (R_k cos t, R_k sin t, z). */
/* loads[0..5] = pressure (Fx,Fy,Fz,Mx,My,Mz), loads[6..11] = shear.          */
/* ------------------------------------------------------------------------ */

static void add_load(double *acc, double th, double Rk, double z, double fx,
                     double fy, double fz, double w)
{
    double rx = Rk * cos(th), ry = Rk * sin(th), rz = z;
    acc[0] += w * fx;
    acc[1] += w * fy;
    acc[2] += w * fz;
    acc[3] += w * (ry * fz - rz * fy);
    acc[4] += w * (rz * fx - rx * fz);
    acc[5] += w * (rx * fy - ry * fx);
}

int oracle_loads(int nth, int nz, const double *phys, const double *tex,
                 const double *state, const double *p, double *loads)
{
    if (nth < 3 || nz < 2 || !phys || !state || !p || !loads) return OR_INVALID;
    double Rk = phys[0], L = phys[1], mu = phys[3], v = phys[4];
    double pch = phys[5], pcase = phys[6];
    double Ub = -v;
    lattice lt = make_lattice(tex, Rk);
    double dth = 2.0 * OR_PI / (double)nth;
    double dz = L / (double)nz;
    double accp[6] = {0, 0, 0, 0, 0, 0}, accs[6] = {0, 0, 0, 0, 0, 0};
    int contact = 0;
    for (int er = 0; er <= nz; ++er) {
        double zlo = (er == 0) ? 0.0 : ((double)er - 0.5) * dz;
        double zhi = (er == nz) ? L : ((double)er + 0.5) * dz;
        double dze = (er == 0 || er == nz) ? 0.5 * dz : dz;
        for (int i = 0; i < nth; ++i) {
            int i2 = (i + 1) % nth;
            double pla = (er == 0) ? pch : p[(size_t)i + (size_t)nth * (size_t)(er - 1)];
            double plb = (er == 0) ? pch : p[(size_t)i2 + (size_t)nth * (size_t)(er - 1)];
            double pha = (er == nz) ? pcase : p[(size_t)i + (size_t)nth * (size_t)er];
            double phb = (er == nz) ? pcase : p[(size_t)i2 + (size_t)nth * (size_t)er];
            double tha = ((double)i + 0.5) * dth;
            double thb = ((double)i2 + 0.5) * dth;
            double A = Rk * dth * dze;
            /* pressure: 2-D trapezoid over the 4 corners */
            double w = 0.25 * A;
            add_load(accp, tha, Rk, zlo, -pla * cos(tha), -pla * sin(tha), 0.0, w);
            add_load(accp, thb, Rk, zlo, -plb * cos(thb), -plb * sin(thb), 0.0, w);
            add_load(accp, tha, Rk, zhi, -pha * cos(tha), -pha * sin(tha), 0.0, w);
            add_load(accp, thb, Rk, zhi, -phb * cos(thb), -phb * sin(thb), 0.0, w);
            /* shear at the element centre */
            double thc = ((double)i + 1.0) * dth;
            double zc = 0.5 * (zlo + zhi);
            double hc = film(phys, &lt, state, thc, zc);
            if (hc <= 0.0) contact = 1;
            double dpdz = ((pha + phb) - (pla + plb)) / (2.0 * dze);
            double dpdt = ((plb + phb) - (pla + pha)) / (2.0 * dth);
            double tz = -(hc / 2.0) * dpdz + mu * Ub / hc;
            double tt = -(hc / 2.0) * dpdt / Rk;
            add_load(accs, thc, Rk, zc, -tt * sin(thc), tt * cos(thc), tz, A);
        }
    }
    for (int k = 0; k < 6; ++k) { loads[k] = accp[k]; loads[6 + k] = accs[k]; }
    return contact ? OR_CONTACT : OR_OK;
}

/* ------------------------------------------------------------------------ */
/* One Picard iteration of the general (double-Jacobian) scheme,             */
/* Eq. 2.12-2.19, for the joint batch of 9 working conditions:               */
/*   0: (e, edot);  1..4: e_j + d_e;  5..8: edot_j + d_edot.                  */
/* Generalized force of the linear tilt (virtual work):                      */
/*   G = (Fx - My/L, Fy + Mx/L, My/L, -Mx/L) + F_ext                          */
/* with (F, M) = pressure + shear loads.  Jacobian J (6 x 8, row-major) by   */
/* forward differences (Eq. 2.13-2.14) of the 6 loads.  Update: with the     */
/* backward-difference closure e_new = e_prev + dt edot_new (Eq. 2.22),      */
/* Eq. 2.12 becomes (J_edot + dt J_e) delta = -G - J_e (e_prev + dt edot - e),*/
/* edot += delta, e = e_prev + dt edot.  The state is only updated when the  */
/* joint solve converged.                                                    */
/* ------------------------------------------------------------------------ */

static int solve4(double K[4][4], double b[4], double x[4])
{
    int piv[4] = {0, 1, 2, 3};
    double A[4][5];
    for (int r = 0; r < 4; ++r) {
        for (int c = 0; c < 4; ++c) A[r][c] = K[r][c];
        A[r][4] = b[r];
    }
    for (int k = 0; k < 4; ++k) {
        int best = k;
        for (int r = k + 1; r < 4; ++r)
            if (fabs(A[r][k]) > fabs(A[best][k])) best = r;
        if (A[best][k] == 0.0 || !isfinite(A[best][k])) return OR_NONFINITE;
        if (best != k) {
            for (int c = 0; c < 5; ++c) { double t = A[k][c]; A[k][c] = A[best][c]; A[best][c] = t; }
            int t = piv[k]; piv[k] = piv[best]; piv[best] = t;
        }
        for (int r = k + 1; r < 4; ++r) {
            double f = A[r][k] / A[k][k];
            for (int c = k; c < 5; ++c) A[r][c] -= f * A[k][c];
        }
    }
    for (int r = 3; r >= 0; --r) {
        double s = A[r][4];
        for (int c = r + 1; c < 4; ++c) s -= A[r][c] * x[c];
        x[r] = s / A[r][r];
    }
    return OR_OK;
}

int oracle_generalized_force(double L, const double *F6, double *G4)
{
    G4[0] = F6[0] - F6[4] / L;
    G4[1] = F6[1] + F6[3] / L;
    G4[2] = F6[4] / L;
    G4[3] = -F6[3] / L;
    return OR_OK;
}

int oracle_picard_step(int nth, int nz, const double *phys, const double *tex,
                       double *state, const double *e_prev, double dt,
                       const double *F_ext, double d_e, double d_edot,
                       int precond, double omega, double eps, int max_iter,
                       double *loads_out, double *J_out, double *G_out,
                       int *iters_out, double *loads_all, double *p_out)
{
    if (nth < 3 || nz < 2 || !phys || !state || !e_prev || !F_ext || !(d_e != 0.0) ||
        !(d_edot != 0.0))
        return OR_INVALID;
    const int K = 9;
    size_t n = (size_t)nth * (size_t)nz;
    size_t N = n * (size_t)K;
    double *D = (double *)malloc(N * sizeof(double));
    double *aE = (double *)malloc(N * sizeof(double));
    double *aN = (double *)malloc(N * sizeof(double));
    double *S = (double *)malloc(N * sizeof(double));
    double *p = (double *)calloc(N, sizeof(double));
    int st = OR_OK;
    if (!D || !aE || !aN || !S || !p) { st = OR_NOMEM; goto done; }

    double cond[9][8];
    for (int k = 0; k < K; ++k) memcpy(cond[k], state, 8 * sizeof(double));
    for (int j = 0; j < 4; ++j) {
        cond[1 + j][j] += d_e;
        cond[5 + j][4 + j] += d_edot;
    }
    for (int k = 0; k < K; ++k) {
        size_t o = (size_t)k * n;
        int s = oracle_assemble(nth, nz, phys, tex, cond[k], D + o, aE + o, aN + o, S + o);
        if (s) { st = s; goto done; }
    }
    int iters = 0;
    double res[2];
    int sst = oracle_solve_joint(nth, nz, K, D, aE, aN, S, p, precond, omega, eps,
                                 max_iter, 1, &iters, res);
    if (iters_out) *iters_out = iters;
    if (sst != OR_OK && sst != OR_NOT_CONVERGED) { st = sst; goto done; }
    if (p_out) memcpy(p_out, p, N * sizeof(double));

    double Lk[9][12];
    for (int k = 0; k < K; ++k) {
        int s = oracle_loads(nth, nz, phys, tex, cond[k], p + (size_t)k * n, Lk[k]);
        if (s) { st = s; goto done; }
        if (loads_all) memcpy(loads_all + 12 * k, Lk[k], 12 * sizeof(double));
    }
    double F[9][6];
    for (int k = 0; k < K; ++k)
        for (int c = 0; c < 6; ++c) F[k][c] = Lk[k][c] + Lk[k][6 + c];
    double J[6][8];
    for (int r = 0; r < 6; ++r)
        for (int c = 0; c < 8; ++c)
            J[r][c] = (F[1 + c][r] - F[0][r]) / (c < 4 ? d_e : d_edot);
    double L = phys[1];
    double G[4];
    oracle_generalized_force(L, F[0], G);
    for (int k = 0; k < 4; ++k) G[k] += F_ext[k];
    if (loads_out) memcpy(loads_out, Lk[0], 12 * sizeof(double));
    if (J_out) for (int r = 0; r < 6; ++r) for (int c = 0; c < 8; ++c) J_out[r * 8 + c] = J[r][c];
    if (G_out) memcpy(G_out, G, 4 * sizeof(double));
    if (sst == OR_NOT_CONVERGED) { st = sst; goto done; }

    /* generalized Jacobians: columns of J mapped through G(.) */
    double Je[4][4], Jd[4][4];
    for (int c = 0; c < 4; ++c) {
        double col[6], g[4];
        for (int r = 0; r < 6; ++r) col[r] = J[r][c];
        oracle_generalized_force(L, col, g);
        for (int r = 0; r < 4; ++r) Je[r][c] = g[r];
        for (int r = 0; r < 6; ++r) col[r] = J[r][4 + c];
        oracle_generalized_force(L, col, g);
        for (int r = 0; r < 4; ++r) Jd[r][c] = g[r];
    }
    double Km[4][4], rhs[4], gap[4], delta[4];
    for (int k = 0; k < 4; ++k) gap[k] = e_prev[k] + dt * state[4 + k] - state[k];
    for (int r = 0; r < 4; ++r) {
        double s = 0.0;
        for (int c = 0; c < 4; ++c) {
            Km[r][c] = Jd[r][c] + dt * Je[r][c];
            s += Je[r][c] * gap[c];
        }
        rhs[r] = -G[r] - s;
    }
    int s4 = solve4(Km, rhs, delta);
    if (s4) { st = s4; goto done; }
    for (int k = 0; k < 4; ++k) {
        state[4 + k] = state[4 + k] + delta[k];
        state[k] = e_prev[k] + dt * state[4 + k];
    }
done:
    free(D); free(aE); free(aN); free(S); free(p);
    return st;
}

/* ------------------------------------------------------------------------ */
/* One conventional (simplified) Picard iteration, Eq. 2.20-2.22: the       */
/* Jacobian F_,e is dropped, so only the base condition and the 4 rate      */
/* perturbations are solved (5 conditions, one joint system, Eq. 3.9).      */
/*   F_,edot by forward differences (Eq. 2.14) on the generalized force,    */
/*   edot_new = edot - [F_,edot]^-1 F            (Eq. 2.21)                 */
/*   e_new    = e - [F_,edot / dt]^-1 F = e + dt (edot_new - edot)  (2.22)  */
/* F is the generalized force G of the oil loads plus F_ext.  J_out is the  */
/* 6 x 8 load Jacobian with its 4 e-columns zero (not computed).            */
/* ------------------------------------------------------------------------ */
int oracle_picard_step_simplified(int nth, int nz, const double *phys, const double *tex,
                                  double *state, double dt, const double *F_ext,
                                  double d_edot, int precond, double omega, double eps,
                                  int max_iter, double *loads_out, double *J_out,
                                  double *G_out, int *iters_out)
{
    if (nth < 3 || nz < 2 || !phys || !state || !F_ext || !(d_edot != 0.0))
        return OR_INVALID;
    const int K = 5;
    size_t n = (size_t)nth * (size_t)nz;
    size_t N = n * (size_t)K;
    double *D = (double *)malloc(N * sizeof(double));
    double *aE = (double *)malloc(N * sizeof(double));
    double *aN = (double *)malloc(N * sizeof(double));
    double *S = (double *)malloc(N * sizeof(double));
    double *p = (double *)calloc(N, sizeof(double));
    int st = OR_OK;
    if (!D || !aE || !aN || !S || !p) { st = OR_NOMEM; goto done; }

    double cond[5][8];
    for (int k = 0; k < K; ++k) memcpy(cond[k], state, 8 * sizeof(double));
    for (int j = 0; j < 4; ++j) cond[1 + j][4 + j] += d_edot;
    for (int k = 0; k < K; ++k) {
        size_t o = (size_t)k * n;
        int s = oracle_assemble(nth, nz, phys, tex, cond[k], D + o, aE + o, aN + o, S + o);
        if (s) { st = s; goto done; }
    }
    int iters = 0;
    double res[2];
    int sst = oracle_solve_joint(nth, nz, K, D, aE, aN, S, p, precond, omega, eps,
                                 max_iter, 1, &iters, res);
    if (iters_out) *iters_out = iters;
    if (sst != OR_OK && sst != OR_NOT_CONVERGED) { st = sst; goto done; }

    double Lk[5][12];
    for (int k = 0; k < K; ++k) {
        int s = oracle_loads(nth, nz, phys, tex, cond[k], p + (size_t)k * n, Lk[k]);
        if (s) { st = s; goto done; }
    }
    double F[5][6];
    for (int k = 0; k < K; ++k)
        for (int c = 0; c < 6; ++c) F[k][c] = Lk[k][c] + Lk[k][6 + c];
    double J[6][4];
    for (int r = 0; r < 6; ++r)
        for (int c = 0; c < 4; ++c) J[r][c] = (F[1 + c][r] - F[0][r]) / d_edot;
    double L = phys[1];
    double G[4];
    oracle_generalized_force(L, F[0], G);
    for (int k = 0; k < 4; ++k) G[k] += F_ext[k];
    if (loads_out) memcpy(loads_out, Lk[0], 12 * sizeof(double));
    if (J_out)
        for (int r = 0; r < 6; ++r)
            for (int c = 0; c < 8; ++c) J_out[r * 8 + c] = c < 4 ? 0.0 : J[r][c - 4];
    if (G_out) memcpy(G_out, G, 4 * sizeof(double));
    if (sst == OR_NOT_CONVERGED) { st = sst; goto done; }

    double Jd[4][4], rhs[4], delta[4];
    for (int c = 0; c < 4; ++c) {
        double col[6], g[4];
        for (int r = 0; r < 6; ++r) col[r] = J[r][c];
        oracle_generalized_force(L, col, g);
        for (int r = 0; r < 4; ++r) Jd[r][c] = g[r];
    }
    for (int r = 0; r < 4; ++r) rhs[r] = -G[r];
    int s4 = solve4(Jd, rhs, delta);
    if (s4) { st = s4; goto done; }
    for (int k = 0; k < 4; ++k) {
        state[4 + k] = state[4 + k] + delta[k];     /* Eq. 2.21 */
        state[k] = state[k] + dt * delta[k];        /* Eq. 2.22 */
    }
done:
    free(D); free(aE); free(aN); free(S); free(p);
    return st;
}

