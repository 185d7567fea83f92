// Geometry, FVM assembly, load integration and the Picard update on the GPU.
//
//  - film thickness: Eq. 2.3 with h_Text from a hexagonal dimple lattice;
//  - assembly: Sec. 2.1 (Eq. 2.1, 2.4-2.7) and Sec. 2.4-I, one thread per cell
//    looping over the conditions, so the texture and the trigonometry of a cell
//    are evaluated once for the whole joint batch;
//  - loads: Sec. 2.4-III, pressure and viscous shear;
//  - Picard: Eq. 2.12-2.19 with the backward-difference closure of Eq. 2.22.
#include <cmath>

#include "gmaf_internal.cuh"

namespace gmaf {

// ------------------------------------------------------------------ host: geometry set-up

Lattice make_lattice(const gmaf_texture *tex, double Rk)
{
    Lattice lt{};
    if (tex == nullptr || tex->kind == 0 || tex->depth == 0.0) return lt;
    lt.on = 1;
    lt.r = tex->radius;
    lt.depth = tex->depth;
    lt.oth = tex->offset_theta;
    lt.oz = tex->offset_z;
    const double rho = tex->area_density;
    const double circ = 2.0 * kPi * Rk;
    // column count: nearest whole number to the ideal hexagonal pitch for density rho
    const double a0 = lt.r * std::sqrt(2.0 * kPi / (std::sqrt(3.0) * rho));
    double ncol = std::round(circ / a0);
    if (ncol < 1.0) ncol = 1.0;
    lt.ath = circ / ncol;
    lt.az = kPi * lt.r * lt.r / (rho * lt.ath);   // one dimple per ath x az cell
    return lt;
}

Geom make_geom(const gmaf_grid *g, const gmaf_physics *ph, const gmaf_texture *tex)
{
    Geom G{};
    G.nth = g->n_theta;
    G.nz = g->n_z;
    G.Rk = ph->R_k;
    G.L = ph->L;
    G.c = ph->c;
    G.mu = ph->mu;
    G.v = ph->v_slide;
    G.pch = ph->p_chamber;
    G.pcase = ph->p_case;
    G.dth = 2.0 * kPi / (double)G.nth;
    G.dx = G.Rk * G.dth;
    G.dz = G.L / (double)G.nz;
    G.invL = 1.0 / G.L;
    G.lt = make_lattice(tex, G.Rk);
    return G;
}

// ------------------------------------------------------------------ device: film thickness

// Texture depth at unwrapped (x, z).  The lattice decision is an integer one,
// so it is written with explicitly rounded operations (no contraction into
// fused multiply-adds) to take the same decision as a plain IEEE evaluation.
__device__ __forceinline__ double texture_depth(const Lattice &lt, double x, double z)
{
    if (!lt.on) return 0.0;
    const double k0 = floor(__ddiv_rn(__dsub_rn(z, lt.oz), lt.az));
    const double r2 = __dmul_rn(lt.r, lt.r);
#pragma unroll
    for (int dk = -1; dk <= 2; ++dk) {
        const double k = __dadd_rn(k0, (double)dk);
        const double zc = __dadd_rn(lt.oz, __dmul_rn(k, lt.az));
        const double dz = __dsub_rn(z, zc);
        const long long ki = (long long)k;
        const double shift = (ki & 1LL) ? __dmul_rn(0.5, lt.ath) : 0.0;
        const double u = __dsub_rn(__dsub_rn(x, lt.oth), shift);
        const double m = floor(__ddiv_rn(u, lt.ath));
        const double dxa = __dsub_rn(u, __dmul_rn(m, lt.ath));
        const double dxb = __dsub_rn(u, __dmul_rn(__dadd_rn(m, 1.0), lt.ath));
        const double dz2 = __dmul_rn(dz, dz);
        if (__dadd_rn(__dmul_rn(dxa, dxa), dz2) < r2) return lt.depth;
        if (__dadd_rn(__dmul_rn(dxb, dxb), dz2) < r2) return lt.depth;
    }
    return 0.0;
}

// Smooth part of Eq. 2.3 for a condition: sqrt((Rc cos - ex)^2 + (Rc sin - ey)^2) - Rk.
// t = z / L along the gap; e = state[0..3].
struct FilmPt {
    double X, Y, rho;
};

__device__ __forceinline__ FilmPt film_pt(const Geom &g, const double *e, double ct, double st,
                                          double t)
{
    const double Rc = g.Rk + g.c;
    const double ex = e[0] + (e[2] - e[0]) * t;
    const double ey = e[1] + (e[3] - e[1]) * t;
    FilmPt f;
    f.X = Rc * ct - ex;
    f.Y = Rc * st - ey;
    f.rho = sqrt(f.X * f.X + f.Y * f.Y);
    return f;
}

// ------------------------------------------------------------------ trig table

// trig = [cos(theta_c), sin(theta_c), cos(theta_e), sin(theta_e)] x nth with
// theta_c = (i + 1/2) dth (cell centres) and theta_e = (i + 1) dth (east faces).
__global__ void k_trig(int nth, double dth, double *trig)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nth) return;
    const double tc = ((double)i + 0.5) * dth;
    const double te = ((double)i + 1.0) * dth;
    double s, c;
    sincos(tc, &s, &c);
    trig[i] = c;
    trig[nth + i] = s;
    sincos(te, &s, &c);
    trig[2 * nth + i] = c;
    trig[3 * nth + i] = s;
}

int launch_trig(const Geom &g, double *trig, cudaStream_t s)
{
    k_trig<<<(g.nth + 127) / 128, 128, 0, s>>>(g.nth, g.dth, trig);
    return cuda_status(cudaGetLastError());
}

// ------------------------------------------------------------------ condition fan-out (Eq. 2.17-2.19)

// conds[k] = base for k = 0; e_{k-1} + d_e for k = 1..4; edot_{k-5} + d_edot for k = 5..8.
// cslot_write[k] = k for k <= 4 (own coefficients), -1 for k >= 5: the ė-perturbed
// conditions share the coefficients of condition 0 because A depends on e only.
// General scheme (Eq. 2.13-2.19): condition 0 = (e, edot), 1..4 = e_j + d_e,
// 5..8 = edot_j + d_edot; coefficient slots 0..4 (A does not depend on edot).
// Simplified scheme (Eq. 2.20): 0 = (e, edot), 1..4 = edot_j + d_edot, all in slot 0.
__global__ void k_fanout(const double base0, const double base1, const double base2,
                         const double base3, const double base4, const double base5,
                         const double base6, const double base7, double d_e, double d_edot,
                         double *conds, int *cslot_write, int simplified)
{
    const int k = threadIdx.x;
    if (k >= (simplified ? 5 : 9)) return;
    double s[8] = {base0, base1, base2, base3, base4, base5, base6, base7};
    if (simplified) {
        if (k >= 1) s[4 + (k - 1)] += d_edot;
        cslot_write[k] = (k == 0) ? 0 : -1;
    } else {
        if (k >= 1 && k <= 4) s[k - 1] += d_e;
        if (k >= 5) s[4 + (k - 5)] += d_edot;
        cslot_write[k] = (k <= 4) ? k : -1;
    }
    for (int q = 0; q < 8; ++q) conds[k * 8 + q] = s[q];
}

int launch_fanout(const double *b, double d_e, double d_edot, double *conds, int *cslot_write,
                  cudaStream_t s, int simplified)
{
    k_fanout<<<1, 32, 0, s>>>(b[0], b[1], b[2], b[3], b[4], b[5], b[6], b[7], d_e, d_edot, conds,
                              cslot_write, simplified);
    return cuda_status(cudaGetLastError());
}

// ------------------------------------------------------------------ assembly

// Pass 1, one thread per cell, all conditions: a_E, a_N, the Dirichlet
// conductance (parked in D) and the source S.  coef_slot[k] >= 0 selects where
// condition k's coefficients go; -1 writes only S.
__global__ void __launch_bounds__(256) k_assemble(Geom g, int ncond,
                                                  const double *__restrict__ conds,
                                                  const int *__restrict__ coef_slot,
                                                  double *__restrict__ D, double *__restrict__ aE,
                                                  double *__restrict__ aN, double *__restrict__ S,
                                                  const double *__restrict__ trig,
                                                  int *__restrict__ flags)
{
    const long long n = (long long)g.nth * g.nz;
    const double Ub = -g.v;
    const double inv12mu = 1.0 / (12.0 * g.mu);
    int contact = 0;
    for (long long P = (long long)blockIdx.x * blockDim.x + threadIdx.x; P < n;
         P += (long long)gridDim.x * blockDim.x) {
        const int j = (int)(P / g.nth);
        const int i = (int)(P - (long long)j * g.nth);
        const double cc = trig[i], sc = trig[g.nth + i];
        const double ce = trig[2 * g.nth + i], se = trig[3 * g.nth + i];
        const double thc = ((double)i + 0.5) * g.dth;
        const double the = ((double)i + 1.0) * g.dth;
        const double zc = ((double)j + 0.5) * g.dz;
        const double zn = ((double)j + 1.0) * g.dz;
        const double zs = (double)j * g.dz;
        // texture once per face for the whole joint batch
        const double hTe = texture_depth(g.lt, __dmul_rn(g.Rk, the), zc);
        const double hTn = texture_depth(g.lt, __dmul_rn(g.Rk, thc), zn);
        const double hTs = texture_depth(g.lt, __dmul_rn(g.Rk, thc), zs);
        const double tc = zc * g.invL, tn = zn * g.invL, ts = zs * g.invL;
        for (int k = 0; k < ncond; ++k) {
            const double *st = conds + 8 * k;
            const FilmPt fe = film_pt(g, st, ce, se, tc);
            const FilmPt fn = film_pt(g, st, cc, sc, tn);
            const FilmPt fs = film_pt(g, st, cc, sc, ts);
            const FilmPt fc = film_pt(g, st, cc, sc, tc);
            const double he = (fe.rho - g.Rk) + hTe;
            const double hn = (fn.rho - g.Rk) + hTn;
            const double hs = (fs.rho - g.Rk) + hTs;
            contact |= (he <= 0.0) | (hn <= 0.0) | (hs <= 0.0);
            // dh/dt = -(X/rho) dex/dt - (Y/rho) dey/dt at the cell centre
            const double exd = st[4] * (1.0 - tc) + st[6] * tc;
            const double eyd = st[5] * (1.0 - tc) + st[7] * tc;
            const double hdot = -(fc.X * exd + fc.Y * eyd) / fc.rho;
            const double gn = hn * hn * hn * inv12mu;
            const double gs = hs * hs * hs * inv12mu;
            double aB = 0.0, sB = 0.0;
            if (j == 0) {
                const double a = gs * g.dx / (0.5 * g.dz);
                aB += a;
                sB += a * g.pch;
            }
            if (j == g.nz - 1) {
                const double a = gn * g.dx / (0.5 * g.dz);
                aB += a;
                sB += a * g.pcase;
            }
            const size_t q = (size_t)k * (size_t)n + (size_t)P;
            S[q] = -(Ub / 2.0) * (hn - hs) * g.dx - hdot * g.dx * g.dz + sB;
            const int slot = coef_slot[k];
            if (slot >= 0) {
                const double ge = he * he * he * inv12mu;
                const size_t qc = (size_t)slot * (size_t)n + (size_t)P;
                aE[qc] = ge * g.dz / g.dx;
                aN[qc] = (j < g.nz - 1) ? gn * g.dx / g.dz : 0.0;
                D[qc] = aB;
            }
        }
    }
    if (contact) atomicOr(flags, 1);
}

// Pass 2: D = a_E + a_W + a_N + a_S + a_B, with a_W(i) = a_E(i-1) (periodic) and
// a_S(j) = a_N(j-1), so that the stored diagonals describe a symmetric matrix.
__global__ void __launch_bounds__(256) k_diag(int nth, int nz, int nslots, double *__restrict__ D,
                                              const double *__restrict__ aE,
                                              const double *__restrict__ aN)
{
    const long long n = (long long)nth * nz;
    const long long total = n * nslots;
    for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < total;
         q += (long long)gridDim.x * blockDim.x) {
        const long long s = q / n;
        const long long P = q - s * n;
        const int j = (int)(P / nth);
        const int i = (int)(P - (long long)j * nth);
        const long long base = s * n + (long long)j * nth;
        const double aW = aE[base + (i == 0 ? nth - 1 : i - 1)];
        const double aS = (j > 0) ? aN[q - nth] : 0.0;
        D[q] = aE[q] + aW + aN[q] + aS + D[q];
    }
}

int launch_assemble(const Geom &g, int ncond, const double *conds, const int *coef_slot,
                    double *D, double *aE, double *aN, double *S, const double *trig, int *flags,
                    int nslots, cudaStream_t s)
{
    const long long n = (long long)g.nth * g.nz;
    int blocks = (int)((n + 255) / 256);
    if (blocks > 152 * 16) blocks = 152 * 16;
    k_assemble<<<blocks, 256, 0, s>>>(g, ncond, conds, coef_slot, D, aE, aN, S, trig, flags);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_status(e);
    long long tot = n * nslots;
    int b2 = (int)((tot + 255) / 256);
    if (b2 > 152 * 16) b2 = 152 * 16;
    k_diag<<<b2, 256, 0, s>>>(g.nth, g.nz, nslots, D, aE, aN);
    return cuda_status(cudaGetLastError());
}

// ------------------------------------------------------------------ loads

__device__ __forceinline__ double warp_sum(double x)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
}

// Pressure: the element-wise 2-D trapezoid (mean of the 4 corners times the
// element area) summed over elements equals a sum over pressure nodes with
// weight R_k dth (dz_below + dz_above)/2, dz_e = dz/2 for the two boundary
// element rows.  Shear: per element at its centre, dp/dz and dp/dtheta from
// differences of edge means.  Node rows r = 0 .. nz+1 (0: z = 0 with p_ch,
// nz+1: z = L with p_case, else cell centres); element rows er = 0 .. nz.
// Grid: blockIdx.y = condition.  Each block writes 12 partial sums; the last
// block of a condition (by ticket) adds them in block order.
__global__ void __launch_bounds__(256) k_loads(Geom g, const double *__restrict__ conds,
                                               const double *__restrict__ p,
                                               const double *__restrict__ trig,
                                               double *__restrict__ partials,
                                               unsigned int *__restrict__ tickets,
                                               double *__restrict__ loads, int *flags)
{
    const int k = blockIdx.y;
    const int nth = g.nth, nz = g.nz;
    const long long n = (long long)nth * nz;
    const double *pk = p + (size_t)k * (size_t)n;
    const double *st = conds + 8 * k;
    const double Ub = -g.v;
    double acc[12];
#pragma unroll
    for (int q = 0; q < 12; ++q) acc[q] = 0.0;
    int contact = 0;
    const long long total = (long long)nth * (nz + 2);
    for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < total;
         q += (long long)gridDim.x * blockDim.x) {
        const int r = (int)(q / nth);
        const int i = (int)(q - (long long)r * nth);
        // node (i, r): pressure
        const double zr = (r == 0) ? 0.0 : ((r == nz + 1) ? g.L : ((double)r - 0.5) * g.dz);
        const double pr = (r == 0) ? g.pch : ((r == nz + 1) ? g.pcase : pk[(size_t)(r - 1) * nth + i]);
        const double dzb = (r == 0) ? 0.0 : ((r == 1 || r == nz + 1) ? 0.5 * g.dz : g.dz);
        const double dza = (r == nz + 1) ? 0.0 : ((r == 0 || r == nz) ? 0.5 * g.dz : g.dz);
        const double w = g.Rk * g.dth * (0.5 * (dzb + dza));
        {
            const double ct = trig[i], sn = trig[nth + i];
            const double fx = -pr * ct * w, fy = -pr * sn * w;
            const double rx = g.Rk * ct, ry = g.Rk * sn;
            acc[0] += fx;
            acc[1] += fy;
            acc[3] += -zr * fy;
            acc[4] += zr * fx;
            acc[5] += rx * fy - ry * fx;
        }
        if (r <= nz) {
            // element (i, er = r): corners (i, r), (i+1, r), (i, r+1), (i+1, r+1)
            const int i2 = (i + 1 == nth) ? 0 : i + 1;
            const int er = r;
            const double pla = pr;
            const double plb = (er == 0) ? g.pch : pk[(size_t)(er - 1) * nth + i2];
            const double pha = (er == nz) ? g.pcase : pk[(size_t)er * nth + i];
            const double phb = (er == nz) ? g.pcase : pk[(size_t)er * nth + i2];
            const double dze = (er == 0 || er == nz) ? 0.5 * g.dz : g.dz;
            const double zlo = zr;
            const double zhi = (er == nz) ? g.L : ((double)er + 0.5) * g.dz;
            const double zc = 0.5 * (zlo + zhi);
            const double thc = ((double)i + 1.0) * g.dth;
            const double ce = trig[2 * nth + i], se = trig[3 * nth + i];
            const double hT = texture_depth(g.lt, __dmul_rn(g.Rk, thc), zc);
            const FilmPt f = film_pt(g, st, ce, se, zc * g.invL);
            const double hc = (f.rho - g.Rk) + hT;
            contact |= (hc <= 0.0);
            const double A = g.Rk * g.dth * dze;
            const double dpdz = ((pha + phb) - (pla + plb)) / (2.0 * dze);
            const double dpdt = ((plb + phb) - (pla + pha)) / (2.0 * g.dth);
            const double tz = -(hc / 2.0) * dpdz + g.mu * Ub / hc;
            const double tt = -(hc / 2.0) * dpdt / g.Rk;
            const double fx = -tt * se * A, fy = tt * ce * A, fz = tz * A;
            const double rx = g.Rk * ce, ry = g.Rk * se;
            acc[6] += fx;
            acc[7] += fy;
            acc[8] += fz;
            acc[9] += ry * fz - zc * fy;
            acc[10] += zc * fx - rx * fz;
            acc[11] += rx * fy - ry * fx;
        }
    }
    if (contact) atomicOr(flags, 1);

    __shared__ double red[12][8];
    __shared__ int s_last;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int q = 0; q < 12; ++q) {
        const double s = warp_sum(acc[q]);
        if (lane == 0) red[q][wid] = s;
    }
    __syncthreads();
    double *part = partials + (size_t)k * gridDim.x * 12;
    if (threadIdx.x < 12) {
        double s = 0.0;
        for (int w2 = 0; w2 < nw; ++w2) s += red[threadIdx.x][w2];
        part[(size_t)blockIdx.x * 12 + threadIdx.x] = s;
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned t = atomicAdd(&tickets[k], 1u);
        s_last = (t == gridDim.x - 1);
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    if (threadIdx.x < 12) {
        double s = 0.0;
        for (unsigned b = 0; b < gridDim.x; ++b) s += __ldcg(&part[(size_t)b * 12 + threadIdx.x]);
        loads[(size_t)k * 12 + threadIdx.x] = s;
    }
    if (threadIdx.x == 0) tickets[k] = 0u;
}

static int loads_blocks(const Geom &g, int num_sms)
{
    const long long total = (long long)g.nth * (g.nz + 2);
    long long b = (total + 255) / 256;
    long long cap = (long long)num_sms * 2;
    if (b > cap) b = cap;
    if (b < 1) b = 1;
    return (int)b;
}

size_t loads_partials_bytes(int ncond, int num_sms)
{
    return (size_t)ncond * (size_t)num_sms * 2 * 12 * sizeof(double) + kMaxCond * sizeof(unsigned);
}

int launch_loads(const Geom &g, int ncond, const double *conds, const double *p,
                 const double *trig, double *partials, unsigned int *tickets, double *loads,
                 int *flags, int num_sms, cudaStream_t s)
{
    const int bx = loads_blocks(g, num_sms);
    dim3 grid(bx, ncond);
    k_loads<<<grid, 256, 0, s>>>(g, conds, p, trig, partials, tickets, loads, flags);
    return cuda_status(cudaGetLastError());
}

// ------------------------------------------------------------------ Picard update

// result layout (doubles): [0..11] loads of condition 0, [12..59] J (6 x 8),
// [60..63] G, [64..71] new state, [72] status (0 ok, -4 singular).
__global__ void k_picard(const double *__restrict__ loads, PicardIn in, double dt, double d_e,
                         double d_edot, double L, double *__restrict__ result)
{
    if (threadIdx.x != 0) return;
    const double *base = in.base, *e_prev = in.e_prev, *F_ext = in.F_ext;
    const bool simp = in.simplified != 0;
    const int K = simp ? 5 : 9;
    double F[9][6];
    for (int k = 0; k < K; ++k)
        for (int c = 0; c < 6; ++c) F[k][c] = loads[k * 12 + c] + loads[k * 12 + 6 + c];
    // load Jacobian by forward differences (Eq. 2.13-2.14); the simplified scheme
    // forms only the rate columns, from its conditions 1..4
    double J[6][8];
    for (int r = 0; r < 6; ++r)
        for (int c = 0; c < 8; ++c) {
            if (simp)
                J[r][c] = c < 4 ? 0.0 : (F[1 + (c - 4)][r] - F[0][r]) / d_edot;
            else
                J[r][c] = (F[1 + c][r] - F[0][r]) / (c < 4 ? d_e : d_edot);
        }
    // generalized force of the linear tilt: (Fx - My/L, Fy + Mx/L, My/L, -Mx/L)
    auto gen = [L](const double *f, double *gout) {
        gout[0] = f[0] - f[4] / L;
        gout[1] = f[1] + f[3] / L;
        gout[2] = f[4] / L;
        gout[3] = -f[3] / L;
    };
    double G[4];
    gen(F[0], G);
    for (int q = 0; q < 4; ++q) G[q] += F_ext[q];
    double Je[4][4], Jd[4][4];
    for (int c = 0; c < 4; ++c) {
        double col[6], gg[4];
        for (int r = 0; r < 6; ++r) col[r] = J[r][c];
        gen(col, gg);
        for (int r = 0; r < 4; ++r) Je[r][c] = gg[r];
        for (int r = 0; r < 6; ++r) col[r] = J[r][4 + c];
        gen(col, gg);
        for (int r = 0; r < 4; ++r) Jd[r][c] = gg[r];
    }
    // general: (J_edot + dt J_e) delta = -G - J_e (e_prev + dt edot - e);
    // simplified (Eq. 2.20-2.21): J_edot delta = -G
    double A[4][5];
    for (int r = 0; r < 4; ++r) {
        double s = 0.0;
        for (int c = 0; c < 4; ++c) {
            A[r][c] = simp ? Jd[r][c] : Jd[r][c] + dt * Je[r][c];
            if (!simp) s += Je[r][c] * (e_prev[c] + dt * base[4 + c] - base[c]);
        }
        A[r][4] = -G[r] - s;
    }
    int status = 0;
    // Gaussian elimination with partial pivoting
    for (int k = 0; k < 4 && status == 0; ++k) {
        int best = k;
        for (int r = k + 1; r < 4; ++r)
            if (fabs(A[r][k]) > fabs(A[best][k])) best = r;
        if (A[best][k] == 0.0 || !isfinite(A[best][k])) {
            status = -4;
            break;
        }
        if (best != k)
            for (int c = 0; c < 5; ++c) {
                const double t = A[k][c];
                A[k][c] = A[best][c];
                A[best][c] = t;
            }
        for (int r = k + 1; r < 4; ++r) {
            const double f = A[r][k] / A[k][k];
            for (int c = k; c < 5; ++c) A[r][c] -= f * A[k][c];
        }
    }
    double delta[4] = {0, 0, 0, 0};
    if (status == 0) {
        for (int r = 3; r >= 0; --r) {
            double s = A[r][4];
            for (int c = r + 1; c < 4; ++c) s -= A[r][c] * delta[c];
            delta[r] = s / A[r][r];
        }
    }
    for (int q = 0; q < 12; ++q) result[q] = loads[q];
    for (int r = 0; r < 6; ++r)
        for (int c = 0; c < 8; ++c) result[12 + r * 8 + c] = J[r][c];
    for (int q = 0; q < 4; ++q) result[60 + q] = G[q];
    for (int q = 0; q < 4; ++q) {
        const double ed = base[4 + q] + delta[q];
        result[64 + 4 + q] = ed;
        // general: e = e_prev + dt edot_new; simplified: e += dt delta (Eq. 2.22)
        result[64 + q] = simp ? base[q] + dt * delta[q] : e_prev[q] + dt * ed;
    }
    result[72] = (double)status;
}

int launch_picard_update(const double *loads, const PicardIn &in, double dt, double d_e,
                         double d_edot, double L, double *result, cudaStream_t s)
{
    k_picard<<<1, 32, 0, s>>>(loads, in, dt, d_e, d_edot, L, result);
    return cuda_status(cudaGetLastError());
}

}  // namespace gmaf
