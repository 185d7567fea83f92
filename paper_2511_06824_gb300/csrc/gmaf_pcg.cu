// Joint preconditioned conjugate gradient on the GPU.
//
// Table 1 (with r0 = S - A p0) on the block-diagonal joint system of Eq. 3.7-3.8,
// one set of scalars for the whole joint system and the synchronized criterion
// of Eq. 3.9.  The preconditioner is ASSOR-II (Eq. 3.3-3.6) or Jacobi (Eq. 2.8).
//
// One iteration is two persistent kernels:
//   phase A:  p += alpha' u';  u = z + beta u';  v = A u;  partial u.v
//   phase B:  r -= alpha v;  z = M^-1 r;  partial r.z, r.r
// Each block stages a tile of the fields with a halo in shared memory and
// recomputes the halo values it needs (u in A; r, D^-1 r and the first ASSOR
// pass in B), so a phase needs no grid-wide barrier inside it.  The dot products
// are reduced per block in a fixed order; the last block to finish (atomic
// ticket, no waiting) adds the block partials in block order and updates the
// scalars, so the result does not depend on scheduling.  The iteration loop is a
// CUDA graph WHILE node whose condition is written by phase B's last block.
//
// ASSOR-II uses L = the strictly lower triangle of A in the joint index order
// (theta fastest).  In the stencil: lower neighbours of cell (i, j) are S (j > 0),
// W (i > 0) and, through the periodic wrap, E when i = n_theta - 1; upper
// neighbours are N (j < n_z - 1), E (i < n_theta - 1) and W when i = 0.
//
// T = double (FP64 mode) or float (inner solve of the mixed-precision mode, whose
// dot products are accumulated exactly per thread in two-float form and reduced in
// FP64).
#include <cmath>
#include <cstring>
#include <mutex>

#include "gmaf_internal.cuh"

namespace gmaf {

// ------------------------------------------------------------------ accumulation

template <typename T>
struct Acc;

template <>
struct Acc<double> {
    double s = 0.0;
    __device__ __forceinline__ void add(double a, double b) { s = fma(a, b, s); }
    __device__ __forceinline__ double value() const { return s; }
};

// Two-float accumulation: exact products (TwoProduct with an FMA) and
// compensated sums (TwoSum), so a thread's partial is accurate to about 2^-44
// relative to the sum of magnitudes before it is handed to FP64.
template <>
struct Acc<float> {
    float hi = 0.0f, lo = 0.0f;
    __device__ __forceinline__ void add(float a, float b)
    {
        const float p = __fmul_rn(a, b);
        const float pe = __fmaf_rn(a, b, -p);
        const float s = __fadd_rn(hi, p);
        const float bb = __fsub_rn(s, hi);
        const float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(p, bb));
        hi = s;
        lo = __fadd_rn(lo, __fadd_rn(e, pe));
    }
    __device__ __forceinline__ double value() const { return (double)hi + (double)lo; }
};

__device__ __forceinline__ double warp_sum_d(double x)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
}

// Block-reduce NV values, publish the block partial, and let the last block
// (by ticket) form the totals in block order.  Returns true in the last block;
// tot[] is valid in thread 0 of that block.
template <int NV>
__device__ __forceinline__ bool reduce_last(const double (&val)[NV], double *partials,
                                            unsigned int *ticket, double (&tot)[NV])
{
    __shared__ double red[NV][32];
    __shared__ int s_last;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int q = 0; q < NV; ++q) {
        const double s = warp_sum_d(val[q]);
        if (lane == 0) red[q][wid] = s;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
#pragma unroll
        for (int q = 0; q < NV; ++q) {
            double s = 0.0;
            for (int w = 0; w < nw; ++w) s += red[q][w];
            partials[(size_t)q * gridDim.x + blockIdx.x] = s;
        }
        __threadfence();
        const unsigned t = atomicAdd(ticket, 1u);
        s_last = (t == gridDim.x - 1);
    }
    __syncthreads();
    if (!s_last) return false;
    __threadfence();
#pragma unroll
    for (int q = 0; q < NV; ++q) {
        double s = 0.0;
        for (unsigned b = threadIdx.x; b < gridDim.x; b += blockDim.x)
            s += __ldcg(&partials[(size_t)q * gridDim.x + b]);
        s = warp_sum_d(s);
        __syncthreads();
        if (lane == 0) red[q][wid] = s;
        __syncthreads();
        if (threadIdx.x == 0) {
            double t = 0.0;
            for (int w = 0; w < nw; ++w) t += red[q][w];
            tot[q] = t;
        }
    }
    if (threadIdx.x == 0) *ticket = 0u;
    return true;
}

__device__ __forceinline__ int wrapi(int i, int n)
{
    int r = i % n;
    return r < 0 ? r + n : r;
}

__device__ __forceinline__ bool finite_d(double x) { return isfinite(x); }

// ------------------------------------------------------------------ tile geometry

template <int TX, int TY>
struct TileOf {
    int cond, i0, j0;
};

template <int TX, int TY>
__device__ __forceinline__ TileOf<TX, TY> tile_of(long long t, int K, int tiles_x)
{
    TileOf<TX, TY> r;
    r.cond = (int)(t % K);          // conditions of one spatial tile are adjacent,
    const long long sp = t / K;     // so coefficient slots shared by several
    const int ty = (int)(sp / tiles_x);   // conditions are re-read from L2
    const int tx = (int)(sp - (long long)ty * tiles_x);
    r.i0 = tx * TX;
    r.j0 = ty * TY;
    return r;
}

// ------------------------------------------------------------------ phase A

template <typename T, int TX, int TY>
__global__ void __launch_bounds__(kThreads) k_phase_a(const PcgDesc<T> *__restrict__ dp)
{
    const PcgDesc<T> &d = *dp;
    Scalars *sc = d.sc;
    __shared__ T su[TY + 2][TX + 2];
    __shared__ int s_done, s_k, s_first;
    __shared__ double s_alpha, s_beta;
    if (threadIdx.x == 0) {
        s_done = sc->done;
        s_k = sc->iter;
        s_first = sc->first;
        s_alpha = sc->alpha;
        s_beta = sc->beta;
        if (blockIdx.x == 0) {
            // stop unless phase B's last block asks for another iteration
            if (d.use_cond) cudaGraphSetConditional(d.cond, 0u);
            sc->guard += 1;
        }
    }
    __syncthreads();
    if (s_done) return;
    const int k = s_k, first = s_first;
    const T alpha_prev = (T)s_alpha, beta = (T)s_beta;
    const int nth = d.nth, nz = d.nz;
    const long long n = d.n;
    const T *uo_base = d.u[(k + 1) & 1];
    T *un_base = d.u[k & 1];
    Acc<T> acc;
    for (long long t = blockIdx.x; t < d.ntiles; t += gridDim.x) {
        const TileOf<TX, TY> tl = tile_of<TX, TY>(t, d.K, d.tiles_x);
        const size_t off = (size_t)tl.cond * (size_t)n;
        const size_t coff = (size_t)d.cslot[tl.cond] * (size_t)n;
        const T *z = d.z + off;
        const T *uo = uo_base + off;
        for (int l = threadIdx.x; l < (TY + 2) * (TX + 2); l += kThreads) {
            const int rr = l / (TX + 2), cc = l - rr * (TX + 2);
            const int gj = tl.j0 - 1 + rr;
            const int gi = wrapi(tl.i0 - 1 + cc, nth);
            T val = T(0);
            if (gj >= 0 && gj < nz) {
                const size_t q = (size_t)gj * nth + gi;
                val = first ? z[q] : z[q] + beta * uo[q];
            }
            su[rr][cc] = val;
        }
        __syncthreads();
        for (int l = threadIdx.x; l < TY * TX; l += kThreads) {
            const int tj = l / TX, ti = l - tj * TX;
            const int gj = tl.j0 + tj, gi = tl.i0 + ti;
            if (gj < nz && gi < nth) {
                const size_t q = (size_t)gj * nth + gi;
                const size_t row = coff + (size_t)gj * nth;
                const T uc = su[tj + 1][ti + 1];
                const T dd = d.D[coff + q];
                const T ae = d.aE[coff + q];
                const T aw = d.aE[row + (gi == 0 ? nth - 1 : gi - 1)];
                const T an = d.aN[coff + q];
                const T as = gj > 0 ? d.aN[coff + q - nth] : T(0);
                const T vv = dd * uc - ae * su[tj + 1][ti + 2] - aw * su[tj + 1][ti] -
                             an * su[tj + 2][ti + 1] - as * su[tj][ti + 1];
                un_base[off + q] = uc;
                d.v[off + q] = vv;
                if (!first) d.p[off + q] += alpha_prev * uo[q];
                acc.add(uc, vv);
            }
        }
        __syncthreads();
    }
    double val[1] = {acc.value()};
    double tot[1];
    if (reduce_last<1>(val, d.partials, &sc->ticket[kTicketA], tot) && threadIdx.x == 0) {
        const double uv = tot[0];
        sc->pending = 0;
        if (!finite_d(uv) || !(uv > 0.0) || !finite_d(sc->d)) {
            sc->status = GMAF_NONFINITE;
            sc->done = 1;
        } else {
            sc->alpha = sc->d / uv;
        }
    }
}

// ------------------------------------------------------------------ phase B

template <typename T, int TX, int TY, bool INIT>
__global__ void __launch_bounds__(kThreads) k_phase_b(const PcgDesc<T> *__restrict__ dp)
{
    const PcgDesc<T> &d = *dp;
    Scalars *sc = d.sc;
    __shared__ T sy[TY + 2][TX + 4];   // D^-1 r on the tile, halo: 1 row each side,
    __shared__ T sw[TY + 2][TX + 4];   // 2 columns west, 2 east (column c <-> i0 - 2 + c)
    __shared__ T sr[TY][TX];
    __shared__ int s_done, s_k;
    __shared__ double s_alpha;
    if (threadIdx.x == 0) {
        s_done = sc->done;
        s_k = sc->iter;
        s_alpha = sc->alpha;
    }
    __syncthreads();
    if (s_done) return;
    const int k = s_k;
    const T alpha = (T)s_alpha;
    const int nth = d.nth, nz = d.nz;
    const long long n = d.n;
    const T omega = d.omega, c1 = d.c1;
    const T *ro_base = d.r[k & 1];
    T *rn_base = d.r[(k + 1) & 1];
    const bool assor = (d.precond == 1);
    Acc<T> arz, arr;
    for (long long t = blockIdx.x; t < d.ntiles; t += gridDim.x) {
        const TileOf<TX, TY> tl = tile_of<TX, TY>(t, d.K, d.tiles_x);
        const size_t off = (size_t)tl.cond * (size_t)n;
        const size_t coff = (size_t)d.cslot[tl.cond] * (size_t)n;
        const T *ro = ro_base + off;
        const T *vv = d.v + off;
        const T *invD = d.invD + coff;
        const T *aE = d.aE + coff;
        const T *aN = d.aN + coff;
        // r_new and y = D^-1 r_new on the tile and its halo
        for (int l = threadIdx.x; l < (TY + 2) * (TX + 4); l += kThreads) {
            const int rr = l / (TX + 4), cc = l - rr * (TX + 4);
            const int gj = tl.j0 - 1 + rr;
            const int gi = wrapi(tl.i0 - 2 + cc, nth);
            T y = T(0);
            if (gj >= 0 && gj < nz) {
                const size_t q = (size_t)gj * nth + gi;
                const T r = INIT ? ro[q] : ro[q] - alpha * vv[q];
                y = r * invD[q];
                const int tj = rr - 1, ti = cc - 2;
                if (tj >= 0 && tj < TY && ti >= 0 && ti < TX) sr[tj][ti] = r;
            }
            sy[rr][cc] = y;
        }
        __syncthreads();
        if (assor) {
            // first ASSOR pass (Eq. 3.5): w = y + omega D^-1 sum_{lower} a y on the tile
            // plus the north row and the east/west columns the second pass reads
            for (int l = threadIdx.x; l < (TY + 1) * (TX + 2); l += kThreads) {
                const int rr = 1 + l / (TX + 2), cc = 1 + (l - (l / (TX + 2)) * (TX + 2));
                const int gj = tl.j0 - 1 + rr;
                const int gi = wrapi(tl.i0 - 2 + cc, nth);
                T w = T(0);
                if (gj < nz) {
                    const size_t q = (size_t)gj * nth + gi;
                    const size_t row = (size_t)gj * nth;
                    T s = T(0);
                    if (gj > 0) s += aN[q - nth] * sy[rr - 1][cc];
                    if (gi > 0) s += aE[row + gi - 1] * sy[rr][cc - 1];
                    if (gi == nth - 1) s += aE[q] * sy[rr][cc + 1];
                    w = sy[rr][cc] + omega * invD[q] * s;
                }
                sw[rr][cc] = w;
            }
            __syncthreads();
        }
        // second pass (Eq. 3.6) and the dot products
        for (int l = threadIdx.x; l < TY * TX; l += kThreads) {
            const int tj = l / TX, ti = l - tj * TX;
            const int gj = tl.j0 + tj, gi = tl.i0 + ti;
            if (gj < nz && gi < nth) {
                const size_t q = (size_t)gj * nth + gi;
                const int rr = tj + 1, cc = ti + 2;
                T zz;
                if (assor) {
                    T s = T(0);
                    if (gj < nz - 1) s += aN[q] * sw[rr + 1][cc];
                    if (gi < nth - 1) s += aE[q] * sw[rr][cc + 1];
                    if (gi == 0) s += aE[(size_t)gj * nth + nth - 1] * sw[rr][cc - 1];
                    zz = c1 * (sw[rr][cc] + omega * invD[q] * s);
                } else {
                    zz = sy[rr][cc];
                }
                const T r = sr[tj][ti];
                d.z[off + q] = zz;
                if (!INIT) rn_base[off + q] = r;
                arz.add(r, zz);
                arr.add(r, r);
            }
        }
        __syncthreads();
    }
    double val[2] = {arz.value(), arr.value()};
    double tot[2];
    if (reduce_last<2>(val, d.partials, &sc->ticket[kTicketB], tot) && threadIdx.x == 0) {
        const double rz = tot[0], rr = tot[1];
        const double rel = sqrt(rr) / sc->normS;
        sc->rel = rel;
        int done = 0;
        if (INIT) {
            sc->d = rz;
            sc->first = 1;
            sc->pending = 0;
            if (sc->zero_rhs) {
                sc->converged = 1;
                done = 1;
            } else if (!finite_d(rz) || !finite_d(rr)) {
                sc->status = GMAF_NONFINITE;
                done = 1;
            } else if (rel <= d.eps) {
                sc->converged = 1;
                done = 1;
            } else if (sc->iter >= d.max_iter) {
                done = 1;
            }
        } else {
            const int it = k + 1;
            sc->iter = it;
            sc->first = 0;
            sc->pending = 1;
            if (!finite_d(rz) || !finite_d(rr)) {
                sc->status = GMAF_NONFINITE;
                done = 1;
            } else if (rel <= d.eps) {
                sc->converged = 1;
                done = 1;
            } else if (it >= d.max_iter) {
                done = 1;
            } else {
                sc->beta = rz / sc->d;
                sc->d = rz;
            }
            if (sc->guard > d.max_iter + 4) {   // loop guard: never more bodies than iterations
                sc->status = GMAF_TIMEOUT;
                done = 1;
            }
        }
        sc->done = done;
        if (d.use_cond) cudaGraphSetConditional(d.cond, done ? 0u : 1u);
    }
}

// ------------------------------------------------------------------ init, finalize

// r0 = b - A p0 (p0 = 0 when zero_init) into r[iter & 1]; ||b||^2.
template <typename T>
__global__ void __launch_bounds__(kThreads) k_init_r(const PcgDesc<T> *__restrict__ dp)
{
    const PcgDesc<T> &d = *dp;
    Scalars *sc = d.sc;
    const int nth = d.nth, nz = d.nz;
    const long long n = d.n, N = n * d.K;
    T *r = d.r[sc->iter & 1];
    Acc<T> abb;
    for (long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x; g < N;
         g += (long long)gridDim.x * blockDim.x) {
        const int cond = (int)(g / n);
        const long long P = g - (long long)cond * n;
        const T bb = d.b[g];
        T rv = bb;
        if (d.zero_init) {
            d.p[g] = T(0);
        } else {
            const int j = (int)(P / nth), i = (int)(P - (long long)j * nth);
            const size_t c = (size_t)d.cslot[cond] * (size_t)n + (size_t)P;
            const size_t row = (size_t)cond * (size_t)n + (size_t)j * nth;
            const T *p = d.p;
            T ap = d.D[c] * p[g] - d.aE[c] * p[row + (i == nth - 1 ? 0 : i + 1)] -
                   d.aE[c - P + (size_t)j * nth + (i == 0 ? nth - 1 : i - 1)] *
                       p[row + (i == 0 ? nth - 1 : i - 1)];
            if (j < nz - 1) ap -= d.aN[c] * p[g + nth];
            if (j > 0) ap -= d.aN[c - nth] * p[g - nth];
            rv = bb - ap;
        }
        r[g] = rv;
        abb.add(bb, bb);
    }
    double val[1] = {abb.value()};
    double tot[1];
    if (reduce_last<1>(val, d.partials, &sc->ticket[kTicketInit], tot) && threadIdx.x == 0) {
        sc->normS = sqrt(tot[0]);
        sc->zero_rhs = (tot[0] == 0.0);
        if (!finite_d(tot[0])) {
            sc->status = GMAF_NONFINITE;
            sc->done = 1;
        }
    }
}

// The update p += alpha u of the last iteration (deferred to phase A otherwise).
template <typename T>
__global__ void __launch_bounds__(kThreads) k_finalize(const PcgDesc<T> *__restrict__ dp)
{
    const PcgDesc<T> &d = *dp;
    Scalars *sc = d.sc;
    if (!sc->pending) return;
    const T alpha = (T)sc->alpha;
    const T *u = d.u[(sc->iter + 1) & 1];
    const long long N = d.n * d.K;
    for (long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x; g < N;
         g += (long long)gridDim.x * blockDim.x)
        d.p[g] += alpha * u[g];
}

__global__ void k_reset(Scalars *sc, int keep_iter)
{
    if (threadIdx.x != 0) return;
    if (!keep_iter) sc->iter = 0;
    sc->first = 1;
    sc->done = 0;
    sc->converged = 0;
    sc->status = 0;
    sc->pending = 0;
    sc->guard = 0;
    sc->zero_rhs = 0;
    sc->alpha = 0.0;
    sc->beta = 0.0;
    for (int q = 0; q < 6; ++q) sc->ticket[q] = 0u;
}

// ------------------------------------------------------------------ FP64 residual, conversions

// r = S - A p (FP64), partial ||r||^2 and ||S||^2; last block sets true_rel and rnorm.
__global__ void __launch_bounds__(kThreads) k_resid64(const ResidDesc *__restrict__ dp)
{
    const ResidDesc &d = *dp;
    const int nth = d.nth, nz = d.nz;
    const long long n = d.n, N = n * d.K;
    double arr = 0.0, ass = 0.0;
    for (long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x; g < N;
         g += (long long)gridDim.x * blockDim.x) {
        const int cond = (int)(g / n);
        const long long P = g - (long long)cond * n;
        const int j = (int)(P / nth), i = (int)(P - (long long)j * nth);
        const size_t crow = (size_t)d.cslot[cond] * (size_t)n + (size_t)j * nth;
        const size_t row = (size_t)cond * (size_t)n + (size_t)j * nth;
        const size_t c = crow + i;
        const double *p = d.p;
        const int ie = (i == nth - 1) ? 0 : i + 1, iw = (i == 0) ? nth - 1 : i - 1;
        double ap = d.D[c] * p[g] - d.aE[c] * p[row + ie] - d.aE[crow + iw] * p[row + iw];
        if (j < nz - 1) ap -= d.aN[c] * p[g + nth];
        if (j > 0) ap -= d.aN[c - nth] * p[g - nth];
        const double s = d.S[g];
        const double rv = s - ap;
        if (d.r) d.r[g] = rv;
        arr = fma(rv, rv, arr);
        ass = fma(s, s, ass);
    }
    double val[2] = {arr, ass};
    double tot[2];
    if (reduce_last<2>(val, d.partials, &d.sc->ticket[kTicketResid], tot) && threadIdx.x == 0) {
        const double nS = sqrt(tot[1]);
        d.sc->rnorm = sqrt(tot[0]);
        d.sc->true_rel = (nS > 0.0) ? sqrt(tot[0]) / nS : 0.0;
        d.sc->normS = nS;
        if (!finite_d(tot[0]) || !finite_d(tot[1])) d.sc->status = GMAF_NONFINITE;
    }
}

// 1/D for FP64 coefficient slots.
__global__ void k_invd64(const double *__restrict__ D, double *__restrict__ invD, long long m)
{
    for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < m;
         q += (long long)gridDim.x * blockDim.x)
        invD[q] = 1.0 / D[q];
}

// FP32 copies of the coefficient slots scaled by a power of two so that the
// FP32 entries are of order one: A32 = scale * A.
__global__ void k_to_f32(const double *__restrict__ D, const double *__restrict__ aE,
                         const double *__restrict__ aN, float *__restrict__ D32,
                         float *__restrict__ invD32, float *__restrict__ aE32,
                         float *__restrict__ aN32, long long m, Scalars *sc)
{
    const double scale = ldexp(1.0, -ilogb(D[0]));
    if (blockIdx.x == 0 && threadIdx.x == 0) sc->scale = scale;
    for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < m;
         q += (long long)gridDim.x * blockDim.x) {
        const double dd = D[q] * scale;
        D32[q] = (float)dd;
        invD32[q] = (float)(1.0 / dd);
        aE32[q] = (float)(aE[q] * scale);
        aN32[q] = (float)(aN[q] * scale);
    }
}

// b32 = r64 / ||r64|| (unit-norm right-hand side of the inner FP32 solve).
__global__ void k_make_b32(const double *__restrict__ r64, float *__restrict__ b32, long long N,
                           const Scalars *__restrict__ outer)
{
    const double inv = 1.0 / outer->rnorm;
    for (long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x; g < N;
         g += (long long)gridDim.x * blockDim.x)
        b32[g] = (float)(r64[g] * inv);
}

// p64 += scale * ||r64|| * x32  (delta = A^-1 r64 = scale ||r64|| (scale A)^-1 (r64/||r64||)).
__global__ void k_update_p64(double *__restrict__ p, const float *__restrict__ x, long long N,
                             const Scalars *__restrict__ outer)
{
    const double f = outer->scale * outer->rnorm;
    for (long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x; g < N;
         g += (long long)gridDim.x * blockDim.x)
        p[g] = fma(f, (double)x[g], p[g]);
}

// ------------------------------------------------------------------ host driver

template <typename T>
struct TileCfg;
template <>
struct TileCfg<double> {
    static constexpr int TX = 128, TY = 8;
};
template <>
struct TileCfg<float> {
    static constexpr int TX = 128, TY = 16;
};

static int grid_for(const void *kernel, long long work_items, int num_sms)
{
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kThreads, 0) != cudaSuccess ||
        per_sm < 1)
        per_sm = 1;
    long long g = (long long)per_sm * num_sms;
    if (g > work_items) g = work_items;
    if (g < 1) g = 1;
    return (int)g;
}

static int stream_grid(long long N, int num_sms)
{
    long long g = (N + kThreads - 1) / kThreads;
    const long long cap = (long long)num_sms * 8;
    if (g > cap) g = cap;
    if (g < 1) g = 1;
    return (int)g;
}

#define GMAF_TRY(x)                                  \
    do {                                             \
        int st__ = (x);                              \
        if (st__ != GMAF_OK) return st__;            \
    } while (0)

#define GMAF_CUDA(x) GMAF_TRY(cuda_status(x))

template <typename T>
struct PcgRun {
    PcgDesc<T> *d_desc;     // device copy of h
    PcgDesc<T> h;
    int grid_a, grid_b, grid_s;
};

template <typename T>
static void launch_phase(const PcgRun<T> &run, cudaStream_t s, int which)
{
    constexpr int TX = TileCfg<T>::TX, TY = TileCfg<T>::TY;
    const PcgDesc<T> *dd = run.d_desc;
    if (which == 0) {
        k_phase_b<T, TX, TY, true><<<run.grid_b, kThreads, 0, s>>>(dd);
    } else if (which == 1) {
        k_phase_a<T, TX, TY><<<run.grid_a, kThreads, 0, s>>>(dd);
        k_phase_b<T, TX, TY, false><<<run.grid_b, kThreads, 0, s>>>(dd);
    } else {
        k_finalize<T><<<run.grid_s, kThreads, 0, s>>>(dd);
    }
}

static bool graph_matches(const GraphCache &gc, int ga, int gb, int gs, const void *desc)
{
    return gc.exec && gc.grid_a == ga && gc.grid_b == gb && gc.grid_s == gs && gc.desc == desc;
}

// Build and instantiate  [init B] -> WHILE{A -> B} -> [finalize]  for a launch
// shape.  The kernels read everything through the device descriptor, so one
// instantiated graph serves every problem of that shape.
template <typename T>
static int build_graph(PcgRun<T> &run, GraphCache &gc, cudaStream_t s)
{
    if (gc.exec) {
        cudaGraphExecDestroy(gc.exec);
        gc.exec = nullptr;
    }
    cudaGraph_t g = nullptr;
    GMAF_CUDA(cudaGraphCreate(&g, 0));
    cudaGraphConditionalHandle h;
    cudaError_t e = cudaGraphConditionalHandleCreate(&h, g, 0u, cudaGraphCondAssignDefault);
    constexpr int TX = TileCfg<T>::TX, TY = TileCfg<T>::TY;
    const PcgDesc<T> *dd = run.d_desc;
    void *args[] = {(void *)&dd};
    cudaGraphNode_t n_init, n_while, n_fin, n_a, n_b;
    cudaKernelNodeParams kp{};
    kp.blockDim = dim3(kThreads);
    kp.kernelParams = args;
    if (e == cudaSuccess) {
        kp.func = (void *)k_phase_b<T, TX, TY, true>;
        kp.gridDim = dim3(run.grid_b);
        e = cudaGraphAddKernelNode(&n_init, g, nullptr, 0, &kp);
    }
    cudaGraphNodeParams cp{};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = h;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    if (e == cudaSuccess) e = cudaGraphAddNode(&n_while, g, &n_init, nullptr, 1, &cp);
    if (e == cudaSuccess) {
        cudaGraph_t body = cp.conditional.phGraph_out[0];
        kp.func = (void *)k_phase_a<T, TX, TY>;
        kp.gridDim = dim3(run.grid_a);
        e = cudaGraphAddKernelNode(&n_a, body, nullptr, 0, &kp);
        if (e == cudaSuccess) {
            kp.func = (void *)k_phase_b<T, TX, TY, false>;
            kp.gridDim = dim3(run.grid_b);
            e = cudaGraphAddKernelNode(&n_b, body, &n_a, 1, &kp);
        }
    }
    if (e == cudaSuccess) {
        kp.func = (void *)k_finalize<T>;
        kp.gridDim = dim3(run.grid_s);
        e = cudaGraphAddKernelNode(&n_fin, g, &n_while, 1, &kp);
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&gc.exec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        gc.exec = nullptr;
        return cuda_status(e);
    }
    gc.handle = h;
    gc.grid_a = run.grid_a;
    gc.grid_b = run.grid_b;
    gc.grid_s = run.grid_s;
    gc.desc = run.d_desc;
    (void)s;
    return GMAF_OK;
}

// Launch shape, partial-sum buffer and descriptor slot of a run.
template <typename T>
static int setup_run(gmaf_ctx *ctx, PcgRun<T> &run, PcgDesc<T> *desc_slot)
{
    constexpr int TX = TileCfg<T>::TX, TY = TileCfg<T>::TY;
    PcgDesc<T> &h = run.h;
    h.tiles_x = (h.nth + TX - 1) / TX;
    h.tiles_y = (h.nz + TY - 1) / TY;
    h.ntiles = (long long)h.tiles_x * h.tiles_y * h.K;
    run.grid_a = grid_for((const void *)k_phase_a<T, TX, TY>, h.ntiles, ctx->num_sms);
    run.grid_b = grid_for((const void *)k_phase_b<T, TX, TY, false>, h.ntiles, ctx->num_sms);
    run.grid_s = stream_grid(h.n * h.K, ctx->num_sms);
    int gm = run.grid_a > run.grid_b ? run.grid_a : run.grid_b;
    if (run.grid_s > gm) gm = run.grid_s;
    GMAF_TRY(ensure(ctx, B_PART, (size_t)2 * gm * sizeof(double)));
    h.partials = (double *)ctx->buf[B_PART];
    run.d_desc = desc_slot;
    return GMAF_OK;
}

// Upload the descriptor, building the loop graph first when needed.
// The loop runs as a graph WHILE node unless the host drives it in chunks
// (GMAF_NO_GRAPH, or per-phase event timing).  Only kernels launched by that
// graph may write its condition, so the descriptor enables the condition
// writes exactly when the graph is used.
static bool use_graph(const gmaf_ctx *ctx) { return !ctx->no_graph && !ctx->phase_timing; }

template <typename T>
static int prepare(gmaf_ctx *ctx, PcgRun<T> &run, GraphCache &gc)
{
    if (!use_graph(ctx)) {
        run.h.use_cond = 0;
    } else {
        if (!graph_matches(gc, run.grid_a, run.grid_b, run.grid_s, run.d_desc))
            GMAF_TRY(build_graph<T>(run, gc, ctx->stream));
        run.h.use_cond = 1;
        run.h.cond = gc.handle;
    }
    GMAF_CUDA(cudaMemcpyAsync(run.d_desc, &run.h, sizeof(PcgDesc<T>), cudaMemcpyHostToDevice,
                              ctx->stream));
    return GMAF_OK;
}

// Event pair around a launch when phase timing is on.
struct PhaseClock {
    gmaf_ctx *ctx;
    int used = 0;
    int kinds[33];
    bool on() const { return ctx->phase_timing && ctx->ev_ready; }
    void begin(cudaStream_t s)
    {
        if (on()) cudaEventRecord(ctx->ev[2 * used], s);
    }
    void end(cudaStream_t s, int kind)
    {
        if (!on()) return;
        cudaEventRecord(ctx->ev[2 * used + 1], s);
        kinds[used++] = kind;
    }
    // after the stream has been synchronised
    void collect()
    {
        for (int q = 0; q < used; ++q) {
            float ms = 0.0f;
            if (cudaEventElapsedTime(&ms, ctx->ev[2 * q], ctx->ev[2 * q + 1]) == cudaSuccess) {
                ctx->phase_ms[kinds[q]] += ms;
                ctx->phase_count[kinds[q]] += 1;
            }
        }
        used = 0;
    }
};

// [reset] [init_r] [init B] WHILE{A, B} [finalize], all on the stream.
template <typename T>
static int pcg_once(gmaf_ctx *ctx, PcgRun<T> &run, GraphCache &gc, bool keep_iter, bool do_init_r)
{
    cudaStream_t s = ctx->stream;
    k_reset<<<1, 32, 0, s>>>(run.h.sc, keep_iter ? 1 : 0);
    GMAF_CUDA(cudaGetLastError());
    if (do_init_r) {
        k_init_r<T><<<run.grid_s, kThreads, 0, s>>>(run.d_desc);
        GMAF_CUDA(cudaGetLastError());
    }
    if (use_graph(ctx)) {
        if (!run.h.use_cond) return GMAF_CUDA_ERROR;   // descriptor prepared for another mode
        return cuda_status(cudaGraphLaunch(gc.exec, s));
    }
    if (run.h.use_cond) return GMAF_CUDA_ERROR;
    // host-chunked loop control: phases return at once after `done` is set
    constexpr int TX = TileCfg<T>::TX, TY = TileCfg<T>::TY;
    const PcgDesc<T> *dd = run.d_desc;
    int *done_h = (int *)ctx->pinned;
    PhaseClock clk{ctx};
    clk.begin(s);
    k_phase_b<T, TX, TY, true><<<run.grid_b, kThreads, 0, s>>>(dd);
    clk.end(s, 2);
    GMAF_CUDA(cudaGetLastError());
    const int chunk = 16;
    for (int it = 0; it <= run.h.max_iter + chunk; it += chunk) {
        GMAF_CUDA(cudaMemcpyAsync(done_h, &run.h.sc->done, sizeof(int), cudaMemcpyDeviceToHost, s));
        GMAF_CUDA(cudaStreamSynchronize(s));
        clk.collect();
        if (*done_h) break;
        for (int q = 0; q < chunk; ++q) {
            clk.begin(s);
            k_phase_a<T, TX, TY><<<run.grid_a, kThreads, 0, s>>>(dd);
            clk.end(s, 0);
            clk.begin(s);
            k_phase_b<T, TX, TY, false><<<run.grid_b, kThreads, 0, s>>>(dd);
            clk.end(s, 1);
        }
        GMAF_CUDA(cudaGetLastError());
    }
    k_finalize<T><<<run.grid_s, kThreads, 0, s>>>(dd);
    return cuda_status(cudaGetLastError());
}

static int read_scalars(gmaf_ctx *ctx, const Scalars *d_sc, Scalars *h_sc)
{
    GMAF_CUDA(cudaMemcpyAsync(h_sc, d_sc, sizeof(Scalars), cudaMemcpyDeviceToHost, ctx->stream));
    GMAF_CUDA(cudaStreamSynchronize(ctx->stream));
    return GMAF_OK;
}

int solve_joint_device(gmaf_ctx *ctx, int nth, int nz, int K, int nslots, const int *cslot_host,
                       const double *D, const double *aE, const double *aN, const double *S,
                       double *p, const gmaf_solver_opts *opts, gmaf_solve_info *info)
{
    cudaStream_t s = ctx->stream;
    const long long n = (long long)nth * nz;
    const long long N = n * K;
    const long long m = n * nslots;
    gmaf_solve_info inf{};
    GMAF_TRY(ensure(ctx, B_SCAL, 2 * sizeof(Scalars)));
    Scalars *dsc = (Scalars *)ctx->buf[B_SCAL];        // PCG run (FP64, or FP32 inner)
    Scalars *dsc_outer = dsc + 1;                       // FP64 residual of the outer loop
    GMAF_TRY(ensure(ctx, B_CSLOT, kMaxCond * sizeof(int)));
    int *cs_pin = (int *)((char *)ctx->pinned + 6144);
    std::memcpy(cs_pin, cslot_host, (size_t)K * sizeof(int));
    GMAF_CUDA(cudaMemcpyAsync(ctx->buf[B_CSLOT], cs_pin, (size_t)K * sizeof(int),
                              cudaMemcpyHostToDevice, s));
    const int *cslot = (const int *)ctx->buf[B_CSLOT];
    Scalars *hsc = (Scalars *)((char *)ctx->pinned + 2048);
    Scalars *ho = (Scalars *)((char *)ctx->pinned + 4096);
    const int gs = stream_grid(N, ctx->num_sms);

    // descriptor buffer: [0, 1024) FP64 PCG, [1024, 2048) FP32 PCG, [3072, 4096) residual
    GMAF_TRY(ensure(ctx, B_DESC, 4096));
    char *dbase = (char *)ctx->buf[B_DESC];
    ResidDesc *d_rdesc = (ResidDesc *)(dbase + 3072);
    ResidDesc *rd_pin = (ResidDesc *)((char *)ctx->pinned + 8192);
    ResidDesc &rd = *rd_pin;
    rd = ResidDesc{};
    rd.nth = nth;
    rd.nz = nz;
    rd.K = K;
    rd.n = n;
    rd.D = D;
    rd.aE = aE;
    rd.aN = aN;
    rd.cslot = cslot;
    rd.S = S;
    rd.p = p;

    if (opts->precision == 0) {
        GMAF_TRY(ensure(ctx, B_INVD, (size_t)m * sizeof(double)));
        const int bufs[] = {B_R0, B_R1, B_U0, B_U1, B_Z, B_V};
        for (int b : bufs) GMAF_TRY(ensure(ctx, b, (size_t)N * sizeof(double)));
        k_invd64<<<stream_grid(m, ctx->num_sms), kThreads, 0, s>>>(D, (double *)ctx->buf[B_INVD], m);
        GMAF_CUDA(cudaGetLastError());
        PcgRun<double> run{};
        PcgDesc<double> &h = run.h;
        h.nth = nth;
        h.nz = nz;
        h.K = K;
        h.n = n;
        h.precond = opts->precond;
        h.zero_init = opts->zero_init;
        h.D = D;
        h.invD = (const double *)ctx->buf[B_INVD];
        h.aE = aE;
        h.aN = aN;
        h.cslot = cslot;
        h.b = S;
        h.p = p;
        h.z = (double *)ctx->buf[B_Z];
        h.v = (double *)ctx->buf[B_V];
        h.u[0] = (double *)ctx->buf[B_U0];
        h.u[1] = (double *)ctx->buf[B_U1];
        h.r[0] = (double *)ctx->buf[B_R0];
        h.r[1] = (double *)ctx->buf[B_R1];
        h.omega = opts->omega;
        h.c1 = opts->omega * (2.0 - opts->omega);
        h.eps = opts->eps;
        h.max_iter = opts->max_iter;
        h.sc = dsc;
        GMAF_TRY(setup_run<double>(ctx, run, (PcgDesc<double> *)dbase));
        GMAF_TRY(prepare<double>(ctx, run, ctx->graph64));
        rd.partials = h.partials;
        rd.sc = dsc_outer;
        int restarted = 0;
        bool keep = false, init_r = true;
        for (;;) {
            GMAF_TRY(pcg_once<double>(ctx, run, ctx->graph64, keep, init_r));
            // true residual S - A p into r[iter & 1], where a restart reads it
            GMAF_TRY(read_scalars(ctx, dsc, hsc));
            rd.r = h.r[hsc->iter & 1];
            GMAF_CUDA(cudaMemcpyAsync(d_rdesc, &rd, sizeof(ResidDesc), cudaMemcpyHostToDevice, s));
            {
                PhaseClock clk{ctx};
                clk.begin(s);
                k_resid64<<<gs, kThreads, 0, s>>>(d_rdesc);
                clk.end(s, 3);
                GMAF_CUDA(cudaGetLastError());
                GMAF_TRY(read_scalars(ctx, dsc_outer, ho));
                clk.collect();
            }
            double true_rel = ho->true_rel;
            if (hsc->zero_rhs) {
                GMAF_CUDA(cudaMemsetAsync(p, 0, (size_t)N * sizeof(double), s));
                GMAF_CUDA(cudaStreamSynchronize(s));
                true_rel = 0.0;
            }
            inf.iterations = hsc->iter;
            inf.rel_residual = hsc->rel;
            inf.true_rel_residual = true_rel;
            inf.restarts = restarted;
            inf.outer_iterations = 1;
            if (hsc->status != 0 || ho->status != 0) {
                inf.status = hsc->status != 0 ? hsc->status : ho->status;
                break;
            }
            if ((hsc->converged || hsc->zero_rhs) && true_rel <= 10.0 * opts->eps) {
                inf.status = GMAF_OK;
                break;
            }
            if (restarted || hsc->iter >= opts->max_iter) {
                inf.status = GMAF_NOT_CONVERGED;
                break;
            }
            restarted = 1;
            keep = true;
            init_r = false;     // r[iter & 1] already holds S - A p
        }
        *info = inf;
        return inf.status;
    }

    // ---------------- mixed precision: FP64 iterative refinement around an FP32 PCG
    GMAF_TRY(ensure(ctx, B_D32, (size_t)m * sizeof(float)));
    GMAF_TRY(ensure(ctx, B_INVD32, (size_t)m * sizeof(float)));
    GMAF_TRY(ensure(ctx, B_AE32, (size_t)m * sizeof(float)));
    GMAF_TRY(ensure(ctx, B_AN32, (size_t)m * sizeof(float)));
    const int fbufs[] = {B_B32, B_X32, B_R032, B_R132, B_U032, B_U132, B_Z32, B_V32};
    for (int b : fbufs) GMAF_TRY(ensure(ctx, b, (size_t)N * sizeof(float)));
    GMAF_TRY(ensure(ctx, B_R64, (size_t)N * sizeof(double)));
    k_to_f32<<<stream_grid(m, ctx->num_sms), kThreads, 0, s>>>(
        D, aE, aN, (float *)ctx->buf[B_D32], (float *)ctx->buf[B_INVD32], (float *)ctx->buf[B_AE32],
        (float *)ctx->buf[B_AN32], m, dsc_outer);
    GMAF_CUDA(cudaGetLastError());
    if (opts->zero_init) GMAF_CUDA(cudaMemsetAsync(p, 0, (size_t)N * sizeof(double), s));

    PcgRun<float> run{};
    PcgDesc<float> &h = run.h;
    h.nth = nth;
    h.nz = nz;
    h.K = K;
    h.n = n;
    h.precond = opts->precond;
    h.zero_init = 1;
    h.D = (const float *)ctx->buf[B_D32];
    h.invD = (const float *)ctx->buf[B_INVD32];
    h.aE = (const float *)ctx->buf[B_AE32];
    h.aN = (const float *)ctx->buf[B_AN32];
    h.cslot = cslot;
    h.b = (const float *)ctx->buf[B_B32];
    h.p = (float *)ctx->buf[B_X32];
    h.z = (float *)ctx->buf[B_Z32];
    h.v = (float *)ctx->buf[B_V32];
    h.u[0] = (float *)ctx->buf[B_U032];
    h.u[1] = (float *)ctx->buf[B_U132];
    h.r[0] = (float *)ctx->buf[B_R032];
    h.r[1] = (float *)ctx->buf[B_R132];
    h.omega = (float)opts->omega;
    h.c1 = (float)(opts->omega * (2.0 - opts->omega));
    h.sc = dsc;
    GMAF_TRY(setup_run<float>(ctx, run, (PcgDesc<float> *)(dbase + 1024)));
    rd.partials = h.partials;
    rd.sc = dsc_outer;
    rd.r = (double *)ctx->buf[B_R64];
    GMAF_CUDA(cudaMemcpyAsync(d_rdesc, &rd, sizeof(ResidDesc), cudaMemcpyHostToDevice, s));

    const double inner_floor = 1e-5;
    const int max_outer = 12;
    int total_inner = 0, outer = 0;
    inf.status = GMAF_NOT_CONVERGED;
    for (;;) {
        {
            PhaseClock clk{ctx};
            clk.begin(s);
            k_resid64<<<gs, kThreads, 0, s>>>(d_rdesc);
            clk.end(s, 3);
            GMAF_CUDA(cudaGetLastError());
            GMAF_TRY(read_scalars(ctx, dsc_outer, ho));
            clk.collect();
        }
        inf.true_rel_residual = ho->true_rel;
        inf.rel_residual = ho->true_rel;
        if (ho->status != 0 || !std::isfinite(ho->true_rel)) {
            inf.status = GMAF_NONFINITE;
            break;
        }
        if (ho->normS == 0.0 || ho->true_rel <= opts->eps) {
            inf.status = GMAF_OK;
            break;
        }
        if (outer >= max_outer || total_inner >= opts->max_iter) break;
        // inner tolerance: a fixed reduction, but no further than the outer target needs
        double eps_in = 0.5 * opts->eps / ho->true_rel;
        if (eps_in < inner_floor) eps_in = inner_floor;
        if (eps_in > 0.5) eps_in = 0.5;
        h.eps = eps_in;
        h.max_iter = opts->max_iter - total_inner;
        GMAF_TRY(prepare<float>(ctx, run, ctx->graph32));
        k_make_b32<<<gs, kThreads, 0, s>>>((const double *)ctx->buf[B_R64], (float *)ctx->buf[B_B32],
                                           N, dsc_outer);
        GMAF_CUDA(cudaGetLastError());
        GMAF_TRY(pcg_once<float>(ctx, run, ctx->graph32, false, true));
        k_update_p64<<<gs, kThreads, 0, s>>>(p, (const float *)ctx->buf[B_X32], N, dsc_outer);
        GMAF_CUDA(cudaGetLastError());
        GMAF_TRY(read_scalars(ctx, dsc, hsc));
        total_inner += hsc->iter;
        ++outer;
        if (hsc->status != 0) {
            inf.status = hsc->status;
            break;
        }
        if (hsc->iter == 0) break;     // no progress possible
    }
    inf.iterations = total_inner;
    inf.outer_iterations = outer;
    *info = inf;
    return inf.status;
}

}  // namespace gmaf

// ------------------------------------------------------------------ allocation-free joint solve
//
// gmaf_solve_joint_noalloc: the FP64 joint solve for callers that may not
// allocate device memory.  All of its scratch (descriptor, scalars, partial
// sums, 1/D and the six PCG vectors) lives in one file-scope device array of
// GMAF_NOALLOC_SCRATCH_BYTES that every GPU loading the library holds until the
// process exits.  Host code cannot use the array's name as a device address, so
// the address is looked up once per device with cudaGetSymbolAddress and passed
// to the kernels.  The loop is driven from the host in chunks (no graph, no
// events, no pinned staging), so nothing here allocates.

namespace gmaf {

static __device__ __align__(256) unsigned char g_noalloc_scratch[GMAF_NOALLOC_SCRATCH_BYTES];

namespace {
constexpr size_t kNaDesc = 0;          // PcgDesc<double>
constexpr size_t kNaResid = 2048;      // ResidDesc
constexpr size_t kNaScal = 4096;       // Scalars of the run, Scalars of the residual
constexpr size_t kNaCslot = 8192;      // int[kMaxCond], identity coefficient map
constexpr size_t kNaPart = 16384;      // block partial sums
constexpr size_t kNaPartBytes = 65536;
constexpr size_t kNaVec = 131072;      // 1/D, r0, r1, u0, u1, z, v: N doubles each
constexpr int kNaMaxDevices = 64;
static_assert(sizeof(PcgDesc<double>) <= kNaResid - kNaDesc, "descriptor slot");
static_assert(sizeof(ResidDesc) <= kNaScal - kNaResid, "residual descriptor slot");
static_assert(2 * sizeof(Scalars) <= kNaCslot - kNaScal, "scalar slot");
static_assert(kNaPart + kNaPartBytes <= kNaVec, "partials slot");

std::mutex g_na_mutex;
void *g_na_base[kNaMaxDevices];

size_t round256(size_t b) { return (b + 255) & ~size_t(255); }

// Device address of the scratch array on the current device (looked up once per device).
int noalloc_base(char **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_status(e);
    if (dev < 0 || dev >= kNaMaxDevices) return GMAF_CUDA_ERROR;
    std::lock_guard<std::mutex> lock(g_na_mutex);
    if (!g_na_base[dev]) {
        void *ptr = nullptr;
        e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
        if (e != cudaSuccess || ptr == nullptr) return cuda_status(e == cudaSuccess ? cudaErrorInvalidSymbol : e);
        g_na_base[dev] = ptr;
    }
    *out = (char *)g_na_base[dev];
    return GMAF_OK;
}
}  // namespace

}  // namespace gmaf

extern "C" int gmaf_solve_joint_noalloc(const gmaf_grid *grid, int32_t n_cond, const double *D,
                                        const double *aE, const double *aN, const double *S,
                                        double *p, const gmaf_solver_opts *opts,
                                        void *cuda_stream, int32_t *iters_out,
                                        double *rel_res_out)
{
    using namespace gmaf;
    if (!grid || !D || !aE || !aN || !S || !p) return GMAF_INVALID_ARG;
    if (grid->n_theta < 3 || grid->n_z < 2 || n_cond < 1 || n_cond > kMaxCond) return GMAF_INVALID_ARG;
    if (!opts_valid(opts) || opts->precision != 0) return GMAF_INVALID_ARG;
    const int nth = grid->n_theta, nz = grid->n_z, K = n_cond;
    const long long n = (long long)nth * nz;
    const long long N = n * K;
    const size_t vec = round256((size_t)N * sizeof(double));
    if ((long long)nth * nz > (1LL << 31) - 1 || kNaVec + 7 * vec > (size_t)GMAF_NOALLOC_SCRATCH_BYTES)
        return GMAF_OUT_OF_MEMORY;
    char *base = nullptr;
    int st = noalloc_base(&base);
    if (st != GMAF_OK) return st;
    int dev = 0, num_sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return cuda_status(e);
    cudaStream_t s = (cudaStream_t)cuda_stream;

    constexpr int TX = TileCfg<double>::TX, TY = TileCfg<double>::TY;
    PcgDesc<double> h{};
    h.nth = nth;
    h.nz = nz;
    h.K = K;
    h.n = n;
    h.tiles_x = (nth + TX - 1) / TX;
    h.tiles_y = (nz + TY - 1) / TY;
    h.ntiles = (long long)h.tiles_x * h.tiles_y * K;
    h.precond = opts->precond;
    h.zero_init = opts->zero_init;
    h.use_cond = 0;
    const int grid_a = grid_for((const void *)k_phase_a<double, TX, TY>, h.ntiles, num_sms);
    const int grid_b = grid_for((const void *)k_phase_b<double, TX, TY, false>, h.ntiles, num_sms);
    const int grid_s = stream_grid(N, num_sms);
    int gm = grid_a > grid_b ? grid_a : grid_b;
    if (grid_s > gm) gm = grid_s;
    if ((size_t)2 * gm * sizeof(double) > kNaPartBytes) return GMAF_OUT_OF_MEMORY;
    double *vbase = (double *)(base + kNaVec);
    double *invD = vbase;
    double *vecs[6];
    for (int q = 0; q < 6; ++q) vecs[q] = (double *)(base + kNaVec + (size_t)(q + 1) * vec);
    Scalars *dsc = (Scalars *)(base + kNaScal);
    Scalars *dsc_res = dsc + 1;
    int *cslot = (int *)(base + kNaCslot);
    h.D = D;
    h.invD = invD;
    h.aE = aE;
    h.aN = aN;
    h.cslot = cslot;
    h.b = S;
    h.p = p;
    h.r[0] = vecs[0];
    h.r[1] = vecs[1];
    h.u[0] = vecs[2];
    h.u[1] = vecs[3];
    h.z = vecs[4];
    h.v = vecs[5];
    h.omega = opts->omega;
    h.c1 = opts->omega * (2.0 - opts->omega);
    h.eps = opts->eps;
    h.max_iter = opts->max_iter;
    h.sc = dsc;
    h.partials = (double *)(base + kNaPart);
    PcgDesc<double> *d_desc = (PcgDesc<double> *)(base + kNaDesc);
    ResidDesc *d_rdesc = (ResidDesc *)(base + kNaResid);
    ResidDesc rd{};
    rd.nth = nth;
    rd.nz = nz;
    rd.K = K;
    rd.n = n;
    rd.D = D;
    rd.aE = aE;
    rd.aN = aN;
    rd.cslot = cslot;
    rd.S = S;
    rd.p = p;
    rd.sc = dsc_res;
    rd.partials = h.partials;
    int slots[kMaxCond];
    for (int k = 0; k < K; ++k) slots[k] = k;

    // The array keeps the previous call's contents: clear the scalars and the
    // reduction tickets, which must start at zero.  The copies below come from
    // pageable (stack) memory and have consumed their sources when they return.
    e = cudaMemsetAsync(base + kNaScal, 0, kNaCslot - kNaScal, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(cslot, slots, (size_t)K * sizeof(int), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(d_desc, &h, sizeof(h), cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return cuda_status(e);
    k_invd64<<<stream_grid(N, num_sms), kThreads, 0, s>>>(D, invD, N);

    Scalars hs{}, hr{};
    int restarted = 0;
    bool keep = false, init_r = true;
    int status = GMAF_NOT_CONVERGED;
    double true_rel = 0.0;
    for (;;) {
        k_reset<<<1, 32, 0, s>>>(dsc, keep ? 1 : 0);
        if (init_r) k_init_r<double><<<grid_s, kThreads, 0, s>>>(d_desc);
        k_phase_b<double, TX, TY, true><<<grid_b, kThreads, 0, s>>>(d_desc);
        e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_status(e);
        const int chunk = 16;
        for (int it = 0; it <= opts->max_iter + chunk; it += chunk) {
            int done = 0;
            e = cudaMemcpyAsync(&done, &dsc->done, sizeof(int), cudaMemcpyDeviceToHost, s);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s);
            if (e != cudaSuccess) return cuda_status(e);
            if (done) break;
            for (int q = 0; q < chunk; ++q) {
                k_phase_a<double, TX, TY><<<grid_a, kThreads, 0, s>>>(d_desc);
                k_phase_b<double, TX, TY, false><<<grid_b, kThreads, 0, s>>>(d_desc);
            }
            e = cudaGetLastError();
            if (e != cudaSuccess) return cuda_status(e);
        }
        k_finalize<double><<<grid_s, kThreads, 0, s>>>(d_desc);
        e = cudaMemcpyAsync(&hs, dsc, sizeof(Scalars), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return cuda_status(e);
        // true residual S - A p into r[iter & 1], where a restart reads it
        rd.r = h.r[hs.iter & 1];
        e = cudaMemcpyAsync(d_rdesc, &rd, sizeof(rd), cudaMemcpyHostToDevice, s);
        if (e != cudaSuccess) return cuda_status(e);
        k_resid64<<<grid_s, kThreads, 0, s>>>(d_rdesc);
        e = cudaMemcpyAsync(&hr, dsc_res, sizeof(Scalars), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return cuda_status(e);
        true_rel = hr.true_rel;
        if (hs.zero_rhs) {
            e = cudaMemsetAsync(p, 0, (size_t)N * sizeof(double), s);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s);
            if (e != cudaSuccess) return cuda_status(e);
            true_rel = 0.0;
        }
        if (hs.status != 0 || hr.status != 0) {
            status = hs.status != 0 ? hs.status : hr.status;
            break;
        }
        if ((hs.converged || hs.zero_rhs) && true_rel <= 10.0 * opts->eps) {
            status = GMAF_OK;
            break;
        }
        if (restarted || hs.iter >= opts->max_iter) {
            status = GMAF_NOT_CONVERGED;
            break;
        }
        restarted = 1;
        keep = true;
        init_r = false;
    }
    if (iters_out) *iters_out = hs.iter;
    if (rel_res_out) *rel_res_out = true_rel;
    return status;
}

