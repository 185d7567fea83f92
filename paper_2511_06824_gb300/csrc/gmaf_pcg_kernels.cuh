// Device code of the joint PCG: accumulation, reductions, the strip-marching
// phase kernels (single joint system and batched groups), initialisation,
// residual and mixed-precision glue kernels.  Included by gmaf_pcg.cu (solver
// driver) and gmaf_server.cu (batched serving).
//
// Table 1 (with r0 = S - A p0) on the block-diagonal joint system of Eq. 3.7-3.8,
// one set of scalars per joint system and the synchronized criterion of Eq. 3.9;
// preconditioner ASSOR-II (Eq. 3.3-3.6) or Jacobi (Eq. 2.8).
#pragma once

#include <cmath>

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
    // add(s, 1) without the TwoProduct: s * 1 is exact (error term 0), so this is
    // bitwise the same as add(s, 1.0f) in fewer instructions
    __device__ __forceinline__ void add_sum(float p)
    {
        const float s = __fadd_rn(hi, p);
        const float bb = __fsub_rn(s, hi);
        const float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(p, bb));
        hi = s;
        lo = __fadd_rn(lo, e);
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

// ------------------------------------------------------------------ strip-marching tiles
//
// A task is one condition x one strip of W = 32 * VEC consecutive columns x TY
// rows.  One warp owns a task: lane l holds columns i0 + l*VEC .. +VEC-1 (one
// 16-byte vector per field and row) and the warp marches down the rows keeping
// the rows above and below in registers; the theta neighbours of a row go
// through a one-row shared buffer of the warp (slot s <-> column i0 - 2 + s in
// phase B, i0 - 1 + s in phase A) filled by the owners and, for the halo
// columns, by lanes 0..3.  Column indices are reduced modulo n_theta once per
// task, so the periodic wrap costs nothing per cell; lanes whose columns lie
// beyond n_theta compute the wrapped columns (their values are neighbours of the
// owned ones) but store nothing.  Requires n_theta % VEC == 0 and 16-byte
// aligned arrays for VEC > 1.
//
// Tasks are numbered with the condition fastest, so the warps working on one
// spatial strip at the same time read a shared coefficient slot once from DRAM.

constexpr int kWarps = kThreads / 32;

template <typename T, int VEC>
struct Vec;
template <typename T>
struct Vec<T, 1> {
    static __device__ __forceinline__ void ld(const T *p, T (&x)[1]) { x[0] = __ldg(p); }
    static __device__ __forceinline__ void ldrw(const T *p, T (&x)[1]) { x[0] = *p; }
    static __device__ __forceinline__ void st(T *p, const T (&x)[1]) { *p = x[0]; }
};
template <>
struct Vec<float, 4> {
    static __device__ __forceinline__ void ld(const float *p, float (&x)[4])
    {
        const float4 t = __ldg(reinterpret_cast<const float4 *>(p));
        x[0] = t.x; x[1] = t.y; x[2] = t.z; x[3] = t.w;
    }
    static __device__ __forceinline__ void ldrw(const float *p, float (&x)[4])
    {
        const float4 t = *reinterpret_cast<const float4 *>(p);
        x[0] = t.x; x[1] = t.y; x[2] = t.z; x[3] = t.w;
    }
    static __device__ __forceinline__ void st(float *p, const float (&x)[4])
    {
        *reinterpret_cast<float4 *>(p) = make_float4(x[0], x[1], x[2], x[3]);
    }
};
template <>
struct Vec<float, 8> {
    static __device__ __forceinline__ void ld(const float *p, float (&x)[8])
    {
        const float4 a = __ldg(reinterpret_cast<const float4 *>(p));
        const float4 b = __ldg(reinterpret_cast<const float4 *>(p) + 1);
        x[0] = a.x; x[1] = a.y; x[2] = a.z; x[3] = a.w; x[4] = b.x; x[5] = b.y; x[6] = b.z; x[7] = b.w;
    }
    static __device__ __forceinline__ void ldrw(const float *p, float (&x)[8])
    {
        const float4 a = *reinterpret_cast<const float4 *>(p);
        const float4 b = *(reinterpret_cast<const float4 *>(p) + 1);
        x[0] = a.x; x[1] = a.y; x[2] = a.z; x[3] = a.w; x[4] = b.x; x[5] = b.y; x[6] = b.z; x[7] = b.w;
    }
    static __device__ __forceinline__ void st(float *p, const float (&x)[8])
    {
        reinterpret_cast<float4 *>(p)[0] = make_float4(x[0], x[1], x[2], x[3]);
        reinterpret_cast<float4 *>(p)[1] = make_float4(x[4], x[5], x[6], x[7]);
    }
};
template <>
struct Vec<float, 2> {
    static __device__ __forceinline__ void ld(const float *p, float (&x)[2])
    {
        const float2 t = __ldg(reinterpret_cast<const float2 *>(p));
        x[0] = t.x; x[1] = t.y;
    }
    static __device__ __forceinline__ void ldrw(const float *p, float (&x)[2])
    {
        const float2 t = *reinterpret_cast<const float2 *>(p);
        x[0] = t.x; x[1] = t.y;
    }
    static __device__ __forceinline__ void st(float *p, const float (&x)[2])
    {
        *reinterpret_cast<float2 *>(p) = make_float2(x[0], x[1]);
    }
};
template <>
struct Vec<double, 2> {
    static __device__ __forceinline__ void ld(const double *p, double (&x)[2])
    {
        const double2 t = __ldg(reinterpret_cast<const double2 *>(p));
        x[0] = t.x; x[1] = t.y;
    }
    static __device__ __forceinline__ void ldrw(const double *p, double (&x)[2])
    {
        const double2 t = *reinterpret_cast<const double2 *>(p);
        x[0] = t.x; x[1] = t.y;
    }
    static __device__ __forceinline__ void st(double *p, const double (&x)[2])
    {
        *reinterpret_cast<double2 *>(p) = make_double2(x[0], x[1]);
    }
};

// Dot-product accumulation: a row's VEC products are summed in T, the row sums
// are accumulated with Acc<T> (exact two-float form for float), and the totals
// are reduced in FP64 across lanes and blocks.
template <typename T>
struct RowAcc {
    Acc<T> acc;
    __device__ __forceinline__ void add_row(T s)
    {
        if constexpr (sizeof(T) == 4)
            acc.add_sum(s);
        else
            acc.add(s, T(1));
    }
    __device__ __forceinline__ double value() const { return acc.value(); }
};

struct Task {
    int cond, i0, j0, jend;
};

template <int W, int TY>
__device__ __forceinline__ Task task_of(long long t, int K, int tiles_x, int nz)
{
    Task r;
    r.cond = (int)(t % K);
    const long long sp = t / K;
    const int ty = (int)(sp / tiles_x);
    const int tx = (int)(sp - (long long)ty * tiles_x);
    r.i0 = tx * W;
    r.j0 = ty * TY;
    r.jend = min(r.j0 + TY, nz);
    return r;
}

// The same with the task height given at run time (the batched kernels, whose
// groups each have their own).
template <int W>
__device__ __forceinline__ Task task_of_rows(long long t, int K, int tiles_x, int nz, int ty)
{
    Task r;
    r.cond = (int)(t % K);
    const long long sp = t / K;
    const int tyi = (int)(sp / tiles_x);
    const int tx = (int)(sp - (long long)tyi * tiles_x);
    r.i0 = tx * W;
    r.j0 = tyi * ty;
    r.jend = min(r.j0 + ty, nz);
    return r;
}

// Static schedule of a phase (SCHED = 1).  The spatial rows of one condition,
// L = tiles_x * nz (tile column tx, then row j), are cut into G groups of
// consecutive rows; item (group g, condition c) = g * K + c goes to warp
// item mod P (P = warps of the launch), so the warps of one block cover the
// same rows of several conditions at once.  f(task) is called for each piece of
// a warp's items (a piece never crosses a tile column); REV walks the items and
// the pieces of each item in the reverse order.
template <bool REV, typename F>
__device__ __forceinline__ void static_pieces(int K, int tiles_x, int nz, int W, long long G,
                                              long long P, long long gw, F &&f)
{
    const long long L = (long long)tiles_x * nz;
    const long long items = G * K;
    if (gw >= items) return;
    const long long mine = (items - 1 - gw) / P + 1;
    for (long long m = 0; m < mine; ++m) {
        const long long it = gw + (REV ? mine - 1 - m : m) * P;
        const long long g = it / K;
        const int cond = (int)(it - g * K);
        const long long lo = g * L / G, hi = (g + 1) * L / G;
        if (!REV) {
            for (long long a = lo; a < hi;) {
                const long long tx = a / nz;
                const long long e = min(hi, (tx + 1) * nz);
                const Task tk{cond, (int)(tx * W), (int)(a - tx * nz), (int)(e - tx * nz)};
                f(tk);
                a = e;
            }
        } else {
            for (long long b = hi; b > lo;) {
                const long long tx = (b - 1) / nz;
                const long long a = max(lo, tx * nz);
                const Task tk{cond, (int)(tx * W), (int)(a - tx * nz), (int)(b - tx * nz)};
                f(tk);
                b = a;
            }
        }
    }
}

__device__ __forceinline__ int wrap_col(int c, int n)
{
    int r = c % n;
    return r < 0 ? r + n : r;
}

// Next task of the warp from the kernel's task counter (one atomic per task).
__device__ __forceinline__ unsigned next_task(unsigned *ctr, int lane)
{
    unsigned t = 0;
    if (lane == 0) t = atomicAdd(ctr, 1u);
    return __shfl_sync(0xffffffffu, t, 0);
}

// Where a phase launch publishes its sums.
struct PcgReduce {
    double *partials;
    double *chunk_sum;
    unsigned *chunk_ctr;
};

template <typename T>
__device__ __forceinline__ PcgReduce reducer_of(const PcgDesc<T> &d)
{
    return PcgReduce{d.partials, d.chunk_sum, d.chunk_ctr};
}

// Publish NV per-task sums (warp-reduced in a fixed order) at partials[t * NV + q].
template <int NV>
__device__ __forceinline__ void publish_task(const double (&v)[NV], double *partials, unsigned t,
                                             int lane)
{
#pragma unroll
    for (int q = 0; q < NV; ++q) {
        const double s = warp_sum_d(v[q]);
        if (lane == 0) partials[(size_t)t * NV + q] = s;
    }
}

// After every task of the launch is published: the last block (by ticket)
// adds the n sums (entry i's q-th at sums[i * stride + q]) in entry order, so
// the totals depend neither on the grid nor on which warp ran which task.
// Also rearms the task counter.
template <int NV>
__device__ __forceinline__ bool reduce_tasks(const double *sums, unsigned n, int stride,
                                             unsigned *ticket, unsigned *task_ctr,
                                             double (&tot)[NV])
{
    __shared__ double red[NV][32];
    __shared__ int s_last;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned t = atomicAdd(ticket, 1u);
        s_last = (t == gridDim.x - 1);
    }
    __syncthreads();
    if (!s_last) return false;
    __threadfence();
    // each thread adds the entries threadIdx.x, + blockDim.x, ... in that order;
    // the unrolled loop keeps several L2 loads in flight
    double acc[NV];
#pragma unroll
    for (int q = 0; q < NV; ++q) acc[q] = 0.0;
#pragma unroll 4
    for (unsigned t = threadIdx.x; t < n; t += blockDim.x) {
#pragma unroll
        for (int q = 0; q < NV; ++q) acc[q] += __ldcg(&sums[(size_t)t * stride + q]);
    }
#pragma unroll
    for (int q = 0; q < NV; ++q) {
        const double s = warp_sum_d(acc[q]);
        if (lane == 0) red[q][wid] = s;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
#pragma unroll
        for (int q = 0; q < NV; ++q) {
            double t = 0.0;
            for (int w = 0; w < nw; ++w) t += red[q][w];
            tot[q] = t;
        }
        *ticket = 0u;
        *task_ctr = 0u;
    }
    return true;
}

// Two-level reduction.  The publishing units (tasks, or warps under the static
// schedule) form chunks of kChunk consecutive ids.  A unit publishes its sums
// and counts itself in its chunk; the warp that completes a chunk adds the
// chunk's sums (a fixed butterfly over the units in id order), stores the chunk
// sum and rearms the counter.  The last block then adds only the chunk sums, in
// chunk order: the same determinism as one level, and the serial work left after
// the last task shrinks from one sum per unit (adds on one SM's FP64 pipe) to
// one per chunk.
constexpr int kChunk = 32;

template <int NV>
__device__ __forceinline__ void publish_unit(const double (&v)[NV], const PcgReduce &rd,
                                             unsigned units, unsigned t, int lane)
{
    publish_task<NV>(v, rd.partials, t, lane);
    if (!rd.chunk_sum) return;
    const unsigned c = t / kChunk;
    const unsigned cnt = min((unsigned)kChunk, units - c * kChunk);
    unsigned prev = 0;
    if (lane == 0) {
        __threadfence();
        prev = atomicAdd(&rd.chunk_ctr[c], 1u);
    }
    prev = __shfl_sync(0xffffffffu, prev, 0);
    if (prev != cnt - 1) return;
    __threadfence();
    const unsigned u = c * kChunk + (unsigned)lane;
#pragma unroll
    for (int q = 0; q < NV; ++q) {
        const double x = warp_sum_d((unsigned)lane < cnt ? __ldcg(&rd.partials[(size_t)u * NV + q]) : 0.0);
        if (lane == 0) rd.chunk_sum[(size_t)c * 2 + q] = x;
    }
    if (lane == 0) rd.chunk_ctr[c] = 0u;
}

// The last block's totals: over the chunk sums, or (one level) the unit sums.
template <int NV>
__device__ __forceinline__ bool reduce_units(const PcgReduce &rd, unsigned units, unsigned *ticket,
                                             unsigned *task_ctr, double (&tot)[NV])
{
    if (rd.chunk_sum)
        return reduce_tasks<NV>(rd.chunk_sum, (units + kChunk - 1) / kChunk, 2, ticket, task_ctr, tot);
    return reduce_tasks<NV>(rd.partials, units, NV, ticket, task_ctr, tot);
}

// ------------------------------------------------------------------ phase A
//   p += alpha' u';  u = z + beta u';  v = A u;  partial u.v
// Marching: at row jr the warp forms u(jr) and outputs v(jr - 1), which needs
// u(jr - 2) (register), u(jr - 1) and its row neighbours (shared row) and u(jr).
// The loads of row jr + 1 are issued before row jr is processed.
// Shared row slot s holds column i0 - 4 + s (own columns start 16-byte aligned).

template <typename T, int VEC>
struct RowA {
    T z[VEC], uo[VEC], D[VEC], e[VEC], n[VEC], p[VEC];
    T hz, huo, he;
};

// One task of phase A; returns the lane's share of the task's u.v.  UP marches
// the rows from the top of the task down to its bottom (jend -> j0): the stencil
// is symmetric in z, so only the roles of the two aN couplings swap.
// first: 1 = u = z (initial iteration), else u = z + beta u' (2: first iteration
// after a reliable update of the residual).  pend: alpha u terms not yet in p;
// this body adds the pending one (p += alpha' u') whenever there is one.
template <typename T, int VEC, bool UP>
__device__ __forceinline__ double run_task_a(const PcgDesc<T> &d, const Task &tk, int k, int first,
                                             int pend, T alpha_prev, T beta, T *ub, T *ab, int lane)
{
    constexpr int W = 32 * VEC;
    const bool uz = first == 1;      // u = z
    const bool nop = pend == 0;      // no p update
    const int nth = d.nth, nz = d.nz;
    const long long n = d.n;
    const T *uo_base = d.u[(k + 1) & 1];
    T *un_base = d.u[k & 1];
        RowAcc<T> acc;
        const size_t off = (size_t)tk.cond * (size_t)n;
        const size_t coff = (size_t)d.cslot[tk.cond] * (size_t)n;
        const T *z = d.z + off;
        const T *uo = uo_base + off;
        T *un = un_base + off;
        T *vv = d.v + off;
        T *pp = d.p + off;
        const T *D = d.D + coff;
        const T *aE = d.aE + coff;
        const T *aN = d.aN + coff;
        const int c0 = tk.i0 + lane * VEC;
        const bool owned = c0 < nth;
        const int g0 = wrap_col(c0, nth);
        const int sown = 4 + lane * VEC;
        // halo: lane 0 -> column i0 - 1 (slot 3), lane 1 -> column i0 + W (slot W + 4);
        // branch-free: every lane loads (lanes 2..31 at lane 1's column) and lanes
        // without a halo column store into the spare slot W + 7
        const int hg = wrap_col(lane == 0 ? tk.i0 - 1 : tk.i0 + W, nth);
        const int hslot = lane == 0 ? 3 : W + 4;
        const int hslot_u = lane < 2 ? hslot : W + 7;
        const int hslot_a = lane == 0 ? hslot : W + 7;

        auto load_row = [&](int jr, RowA<T, VEC> &R) {
            if (jr < 0 || jr >= nz) {
#pragma unroll
                for (int q = 0; q < VEC; ++q) R.z[q] = R.uo[q] = R.D[q] = R.e[q] = R.n[q] = R.p[q] = T(0);
                R.hz = R.huo = R.he = T(0);
                return;
            }
            const size_t q0 = (size_t)jr * nth + g0;
            Vec<T, VEC>::ld(z + q0, R.z);
            if (!uz) {
                Vec<T, VEC>::ld(uo + q0, R.uo);
            } else {
#pragma unroll
                for (int q = 0; q < VEC; ++q) R.uo[q] = T(0);
            }
            Vec<T, VEC>::ld(aN + q0, R.n);
            if (jr >= tk.j0 && jr < tk.jend) {
                Vec<T, VEC>::ld(D + q0, R.D);
                Vec<T, VEC>::ld(aE + q0, R.e);
                if (!nop && owned) {
                    Vec<T, VEC>::ldrw(pp + q0, R.p);
                } else {
#pragma unroll
                    for (int q = 0; q < VEC; ++q) R.p[q] = T(0);
                }
            } else {
#pragma unroll
                for (int q = 0; q < VEC; ++q) R.D[q] = R.e[q] = R.p[q] = T(0);
            }
            const size_t qh = (size_t)jr * nth + hg;
            R.hz = __ldg(z + qh);
            R.huo = uz ? T(0) : __ldg(uo + qh);
            R.he = __ldg(aE + qh);
        };

        T u_m1[VEC], u_m2[VEC], uo_m1[VEC], D_m1[VEC], e_m1[VEC], n_m1[VEC], n_m2[VEC], p_m1[VEC];
#pragma unroll
        for (int q = 0; q < VEC; ++q)
            u_m1[q] = u_m2[q] = uo_m1[q] = D_m1[q] = e_m1[q] = n_m1[q] = n_m2[q] = p_m1[q] = T(0);
        RowA<T, VEC> nx;
        constexpr int step = UP ? -1 : 1;
        const int jfirst = UP ? tk.jend : tk.j0 - 1;
        const int jlast = UP ? tk.j0 - 1 : tk.jend;
        load_row(jfirst, nx);
        for (int jr = jfirst; UP ? jr >= jlast : jr <= jlast; jr += step) {
            const RowA<T, VEC> cur = nx;
            if (jr != jlast) load_row(jr + step, nx);
            T u[VEC];
#pragma unroll
            for (int q = 0; q < VEC; ++q) u[q] = uz ? cur.z[q] : cur.z[q] + beta * cur.uo[q];
            const T hu = uz ? cur.hz : cur.hz + beta * cur.huo;
            // output row jo (the previous step's row): its u row and aE row are in
            // the shared buffers; u_m2 is the row beyond jo, u the row before it
            const int jo = jr - step;
            if (jo >= tk.j0 && jo < tk.jend) {
                T vout[VEC];
                T rowsum = T(0);
#pragma unroll
                for (int q = 0; q < VEC; ++q) {
                    const int s = sown + q;
                    const T uE = (q < VEC - 1) ? u_m1[q + 1] : ub[s + 1];
                    const T uW = (q > 0) ? u_m1[q - 1] : ub[s - 1];
                    const T aW = (q > 0) ? e_m1[q - 1] : ab[s - 1];
                    if (UP)   // n_m1 = aN(jo) couples jo + 1 (u_m2); cur.n = aN(jo - 1) couples u
                        vout[q] = D_m1[q] * u_m1[q] - e_m1[q] * uE - aW * uW - n_m1[q] * u_m2[q] -
                                  cur.n[q] * u[q];
                    else      // n_m1 = aN(jo) couples jo + 1 (u); n_m2 = aN(jo - 1) couples u_m2
                        vout[q] = D_m1[q] * u_m1[q] - e_m1[q] * uE - aW * uW - n_m1[q] * u[q] -
                                  n_m2[q] * u_m2[q];
                    rowsum += u_m1[q] * vout[q];
                }
                if (owned) {
                    const size_t qo = (size_t)jo * nth + g0;
                    Vec<T, VEC>::st(un + qo, u_m1);
                    Vec<T, VEC>::st(vv + qo, vout);
                    if (!nop) {
                        T pn[VEC];
#pragma unroll
                        for (int q = 0; q < VEC; ++q) pn[q] = p_m1[q] + alpha_prev * uo_m1[q];
                        Vec<T, VEC>::st(pp + qo, pn);
                    }
                    acc.add_row(rowsum);
                }
            }
            __syncwarp();
            Vec<T, VEC>::st(ub + sown, u);
            Vec<T, VEC>::st(ab + sown, cur.e);
            ub[hslot_u] = hu;
            ab[hslot_a] = cur.he;
            __syncwarp();
#pragma unroll
            for (int q = 0; q < VEC; ++q) {
                u_m2[q] = u_m1[q];
                u_m1[q] = u[q];
                uo_m1[q] = cur.uo[q];
                n_m2[q] = n_m1[q];
                n_m1[q] = cur.n[q];
                D_m1[q] = cur.D[q];
                e_m1[q] = cur.e[q];
                p_m1[q] = cur.p[q];
            }
        }
    return acc.value();
}

// Scalar update after the u.v reduction (alpha = d / u.v).  added: the phase
// added the pending p updates; otherwise the last alpha stays pending as alpha_pp.
__device__ __forceinline__ void finish_a(Scalars *sc, double uv, bool added)
{
    if (added)
        sc->pending = 0;
    else
        sc->alpha_pp = sc->alpha;
    if (!finite_d(uv) || !(uv > 0.0) || !finite_d(sc->d)) {
        sc->status = GMAF_NONFINITE;
        sc->done = 1;
    } else {
        sc->alpha = sc->d / uv;
    }
}

// SCHED 0: dynamic tasks of TY rows, marched downward.  SCHED 1: the static
// schedule, marched upward, mirroring phase B (which marches downward), so each
// phase starts on the rows the other touched last and finds them in L2.
template <typename T, int VEC, int TY, int MINB, int SCHED>
__global__ void __launch_bounds__(kThreads, MINB) k_phase_a(const PcgDesc<T> *__restrict__ dp)
{
    constexpr int W = 32 * VEC;
    constexpr int NB = W + 8;
    const PcgDesc<T> &d = *dp;
    Scalars *sc = d.sc;
    __shared__ __align__(16) T su[kWarps][NB];
    __shared__ __align__(16) T sa[kWarps][NB];
    __shared__ int s_done, s_k, s_first, s_pend;
    __shared__ double s_alpha, s_beta;
    if (threadIdx.x == 0) {
        s_done = sc->done;
        s_k = sc->iter;
        s_first = sc->first;
        s_pend = sc->pending;
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
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
    unsigned ntasks;
    if (SCHED == 0) {
        ntasks = (unsigned)d.ntiles;
        for (unsigned t = next_task(&sc->task_ctr[0], lane); t < ntasks;
             t = next_task(&sc->task_ctr[0], lane)) {
            const Task tk = task_of<W, TY>(t, d.K, d.tiles_x, d.nz);
            const double val[1] = {run_task_a<T, VEC, false>(d, tk, s_k, s_first, s_pend, (T)s_alpha,
                                                              (T)s_beta, su[wp], sa[wp], lane)};
            publish_unit<1>(val, reducer_of(d), ntasks, t, lane);
        }
    } else {
        ntasks = gridDim.x * kWarps;
        const unsigned gw = blockIdx.x * kWarps + wp;
        double v = 0.0;
        static_pieces<true>(d.K, d.tiles_x, d.nz, W, d.sgroups, ntasks, gw, [&](const Task &tk) {
            v += run_task_a<T, VEC, true>(d, tk, s_k, s_first, s_pend, (T)s_alpha, (T)s_beta, su[wp],
                                          sa[wp], lane);
        });
        const double val[1] = {v};
        publish_unit<1>(val, reducer_of(d), ntasks, gw, lane);
    }
    double tot[1];
    if (reduce_units<1>(reducer_of(d), ntasks, &sc->ticket[kTicketA], &sc->task_ctr[0], tot) &&
        threadIdx.x == 0)
        finish_a(sc, tot[0], s_pend > 0);
}

// ------------------------------------------------------------------ phase B
//   r -= alpha v;  z = M^-1 r;  partial r.z, r.r
// The stored diagonal d.invD is omega D^-1 for ASSOR-II (D^-1 for Jacobi), so y,
// w and z below are omega times those of Eq. 3.5-3.6 (PCG is invariant under a
// constant factor on the preconditioner, as it is under the c1 left out of z).
// Marching: at row jr the warp forms r(jr), y = omega D^-1 r (shared row), the first
// ASSOR pass w(jr) (needs y(jr - 1) in registers and the row neighbours of
// y(jr)), and the second pass z(jr - 1) (needs w(jr) in registers and the row
// neighbours of w(jr - 1), still in the shared row).  Halo columns i0 - 2 ..
// i0 - 1 and i0 + W .. i0 + W + 1 are formed by lanes 0..3.  The loads of row
// jr + 1 are issued before row jr is processed.  Shared row slot s holds column
// i0 - 4 + s.

template <typename T, int VEC>
struct RowB {
    T r[VEC], v[VEC], dI[VEC], e[VEC], n[VEC];
    T hr, hv, hd, he, hn;
};

// One task of phase B; writes the lane's shares of the task's r.z and r.r.
// One body serves every task (a second, specialised copy of this unrolled body
// measured slower: the kernel is sensitive to its code size).  In FP32 the halo
// work is branch-free: every lane issues the halo loads, lanes 4..31 at lane
// 3's column (same address, no extra traffic) and into a spare shared slot.  In
// FP64, bound by the FP64 pipe, only the lanes that own a halo column do it.
template <typename T, int VEC, bool INIT>
__device__ __forceinline__ void run_task_b(const PcgDesc<T> &d, const Task &tk, int k, T alpha,
                                           T *yb, T *wb, T *ab, int lane, double (&out)[2])
{
    constexpr int W = 32 * VEC;
    constexpr int kSpare = W + 7;      // shared slot written by lanes without a halo column
    constexpr bool BF = sizeof(T) == 4;
    const int nth = d.nth, nz = d.nz;
    const long long n = d.n;
    const bool assor = (d.precond == 1);
    const T *ro_base = d.r[k & 1];
    T *rn_base = d.r[(k + 1) & 1];
        RowAcc<T> arz, arr;
        const size_t off = (size_t)tk.cond * (size_t)n;
        const size_t coff = (size_t)d.cslot[tk.cond] * (size_t)n;
        const T *ro = ro_base + off;
        const T *vv = d.v + off;
        T *rn = rn_base + off;
        T *zo = d.z + off;
        const T *invD = d.invD + coff;
        const T *aE = d.aE + coff;
        const T *aN = d.aN + coff;
        const int c0 = tk.i0 + lane * VEC;
        const bool owned = c0 < nth;
        const int g0 = wrap_col(c0, nth);
        // n_theta % VEC == 0: only element 0 of a lane can be column 0 and only
        // element VEC - 1 column n_theta - 1 (the seam tests below are static otherwise)
        const bool at_w = g0 == 0, at_e = g0 + VEC == nth;
        const int sown = 4 + lane * VEC;
        // halo: lanes 0..3 -> columns i0-2, i0-1 (slots 2, 3), i0+W, i0+W+1 (slots W+4, W+5)
        const int hl = lane < 4 ? lane : 3;
        const int hoff = hl < 2 ? hl - 2 : W + (hl - 2);
        const int hg = wrap_col(tk.i0 + hoff, nth);
        const int hs = hl < 2 ? hl + 2 : W + 2 + hl;          // the halo column's slot
        const int hslot_y = lane < 4 ? hs : kSpare;            // y, aE of lanes 0..3
        const int hslot_w = (lane == 1 || lane == 2) ? hs : kSpare;   // w of lanes 1, 2

        auto load_row = [&](int jr, RowB<T, VEC> &R) {
            if (jr < 0 || jr >= nz) {
#pragma unroll
                for (int q = 0; q < VEC; ++q) R.r[q] = R.v[q] = R.dI[q] = R.e[q] = R.n[q] = T(0);
                R.hr = R.hv = R.hd = R.he = R.hn = T(0);
                return;
            }
            const size_t q0 = (size_t)jr * nth + g0;
            Vec<T, VEC>::ld(ro + q0, R.r);
            if (!INIT) {
                Vec<T, VEC>::ld(vv + q0, R.v);
            } else {
#pragma unroll
                for (int q = 0; q < VEC; ++q) R.v[q] = T(0);
            }
            Vec<T, VEC>::ld(invD + q0, R.dI);
            Vec<T, VEC>::ld(aE + q0, R.e);
            Vec<T, VEC>::ld(aN + q0, R.n);
            R.hr = R.hv = R.hd = R.he = R.hn = T(0);
            if (BF || lane < 4) {
                const size_t qh = (size_t)jr * nth + hg;
                R.hr = __ldg(ro + qh);
                if (!INIT) R.hv = __ldg(vv + qh);
                R.hd = __ldg(invD + qh);
                R.he = __ldg(aE + qh);
                R.hn = __ldg(aN + qh);
            }
        };

        T y_m1[VEC], w_m1[VEC], od_m1[VEC], n_m1[VEC], e_m1[VEC], r_m1[VEC];
#pragma unroll
        for (int q = 0; q < VEC; ++q) y_m1[q] = w_m1[q] = od_m1[q] = n_m1[q] = e_m1[q] = r_m1[q] = T(0);
        T hy_m1 = T(0), hn_m1 = T(0), he_m1 = T(0);
        RowB<T, VEC> nx;
        load_row(tk.j0 - 1, nx);
        for (int jr = tk.j0 - 1; jr <= tk.jend; ++jr) {
            const RowB<T, VEC> cur = nx;
            if (jr + 1 <= tk.jend) load_row(jr + 1, nx);
            const bool inrow = jr >= 0 && jr < nz;
            T r1[VEC], y[VEC];
#pragma unroll
            for (int q = 0; q < VEC; ++q) {
                r1[q] = INIT ? cur.r[q] : cur.r[q] - alpha * cur.v[q];
                y[q] = r1[q] * cur.dI[q];
            }
            const T hy = (INIT ? cur.hr : cur.hr - alpha * cur.hv) * cur.hd;
            Vec<T, VEC>::st(yb + sown, y);
            Vec<T, VEC>::st(ab + sown, cur.e);
            if (BF || lane < 4) {
                yb[hslot_y] = hy;
                ab[hslot_y] = cur.he;
            }
            // FP32: aE(jr - 1, n_theta - 1), the wrapped west coupling of column 0 in
            // the second pass, from lane 1 (column i0 - 1, which is n_theta - 1 when
            // i0 = 0); FP64 loads it where it is needed
            T aw_wrap = T(0);
            if (BF) aw_wrap = __shfl_sync(0xffffffffu, he_m1, 1);
            __syncwarp();
            // first ASSOR pass on row jr: w = y + omega D^-1 (lower couplings) y
            T w[VEC], od[VEC];                 // od = omega D^-1, reused by the second pass
            T hw = T(0);
#pragma unroll
            for (int q = 0; q < VEC; ++q) w[q] = od[q] = T(0);
            if (assor && inrow && jr >= tk.j0) {
#pragma unroll
                for (int q = 0; q < VEC; ++q) {
                    const int s = sown + q;
                    T sum = T(0);
                    if (jr > 0) sum += n_m1[q] * y_m1[q];                            // south
                    if (q > 0 || !at_w)                                                // west
                        sum += ((q > 0) ? cur.e[q - 1] : ab[s - 1]) * ((q > 0) ? y[q - 1] : yb[s - 1]);
                    if (q == VEC - 1 && at_e)                                          // east, wrapped
                        sum += cur.e[q] * ((q < VEC - 1) ? y[q + 1] : yb[s + 1]);
                    od[q] = cur.dI[q];
                    w[q] = y[q] + od[q] * sum;
                }
                // halo w (used for lanes 1, 2; in FP32 the others compute and discard it)
                if (BF || lane == 1 || lane == 2) {
                    T sum = T(0);
                    if (jr > 0) sum += hn_m1 * hy_m1;
                    if (hg > 0) sum += ab[hs - 1] * yb[hs - 1];
                    if (hg == nth - 1) sum += cur.he * yb[hs + 1];
                    hw = hy + cur.hd * sum;
                }
            }
            // second pass on row jo = jr - 1: z = w + omega D^-1 (upper couplings) w.
            // The constant factor c1 = omega (2 - omega) of Eq. 3.6 is left out: PCG is
            // invariant under scaling the preconditioner by a positive constant (alpha
            // takes the inverse factor; p and r are unchanged), and it saves an FP64
            // multiply per cell where FP64 arithmetic bounds the phase
            const int jo = jr - 1;
            if (jo >= tk.j0 && jo < tk.jend) {
                T zz[VEC];
                T rz = T(0), rr = T(0);
#pragma unroll
                for (int q = 0; q < VEC; ++q) {
                    if (assor) {
                        const int s = sown + q;
                        T sum = T(0);
                        if (jo < nz - 1) sum += n_m1[q] * w[q];                                          // north
                        if (q < VEC - 1 || !at_e) sum += e_m1[q] * ((q < VEC - 1) ? w_m1[q + 1] : wb[s + 1]);  // east
                        if (q == 0 && at_w)                                                              // west, wrapped
                            sum += (BF ? aw_wrap : __ldg(aE + (size_t)jo * nth + nth - 1)) *
                                   ((q > 0) ? w_m1[q - 1] : wb[s - 1]);
                        zz[q] = w_m1[q] + od_m1[q] * sum;      // Eq. 3.6 without its factor c1
                    } else {
                        zz[q] = y_m1[q];
                    }
                    rz += r_m1[q] * zz[q];
                    rr += r_m1[q] * r_m1[q];
                }
                if (owned) {
                    const size_t qo = (size_t)jo * nth + g0;
                    Vec<T, VEC>::st(zo + qo, zz);
                    if (!INIT) Vec<T, VEC>::st(rn + qo, r_m1);
                    arz.add_row(rz);
                    arr.add_row(rr);
                }
            }
            __syncwarp();
            if (assor) {
                Vec<T, VEC>::st(wb + sown, w);
                if (BF || lane == 1 || lane == 2) wb[hslot_w] = hw;
            }
            __syncwarp();
#pragma unroll
            for (int q = 0; q < VEC; ++q) {
                y_m1[q] = y[q];
                w_m1[q] = w[q];
                od_m1[q] = od[q];
                n_m1[q] = cur.n[q];
                e_m1[q] = cur.e[q];
                r_m1[q] = r1[q];
            }
            hy_m1 = hy;
            hn_m1 = cur.hn;
            he_m1 = cur.he;
        }
    out[0] = arz.value();
    out[1] = arr.value();
}

// Scalar update after the r.z, r.r reductions: convergence test (Eq. 3.9), beta,
// loop guard.  Returns 1 when the run is done.
template <bool INIT>
__device__ __forceinline__ int finish_b(Scalars *sc, double rz, double rr, int k, double eps,
                                        int max_iter, int guard_limit)
{
    const double rel = sqrt(rr) / sc->normS;
    sc->rel = rel;
    int done = 0;
    if (INIT) {
        // reliable update (mixed precision): r was replaced by the FP64 residual;
        // continue with u = z + beta u', the old direction converted to the new
        // units (old d = r.z of the last iteration, in units cscale times smaller)
        if (sc->cont && finite_d(rz) && finite_d(sc->d) && sc->d > 0.0 && sc->cscale > 0.0) {
            sc->beta = rz / (sc->cscale * sc->d);
            sc->first = 2;
        } else {
            sc->first = 1;
        }
        sc->cont = 0;
        sc->d = rz;
        sc->pending = 0;
        if (sc->zero_rhs) {
            sc->converged = 1;
            done = 1;
        } else if (!finite_d(rz) || !finite_d(rr)) {
            sc->status = GMAF_NONFINITE;
            done = 1;
        } else if (rel <= eps) {
            sc->converged = 1;
            done = 1;
        } else if (sc->iter >= max_iter) {
            done = 1;
        }
    } else {
        const int it = k + 1;
        sc->iter = it;
        sc->first = 0;
        sc->pending += 1;             // alpha u of this iteration
        if (!finite_d(rz) || !finite_d(rr)) {
            sc->status = GMAF_NONFINITE;
            done = 1;
        } else if (rel <= eps) {
            sc->converged = 1;
            done = 1;
        } else if (it >= max_iter) {
            done = 1;
        } else {
            sc->beta = rz / sc->d;
            sc->d = rz;
        }
        // loop guard: never more bodies than iterations (a host-set limit can lower it)
        if (sc->guard > (guard_limit > 0 ? guard_limit : max_iter + 4)) {
            sc->status = GMAF_TIMEOUT;
            done = 1;
        }
    }
    sc->done = done;
    return done;
}

// SCHED 0: dynamic tasks of TY rows, claimed in the reverse of phase A's order.
// SCHED 1: the static schedule in forward order (phase A walks it backward).
template <typename T, int VEC, int TY, int MINB, bool INIT, int SCHED>
__global__ void __launch_bounds__(kThreads, MINB) k_phase_b(const PcgDesc<T> *__restrict__ dp)
{
    constexpr int W = 32 * VEC;
    constexpr int NB = W + 8;
    const PcgDesc<T> &d = *dp;
    Scalars *sc = d.sc;
    __shared__ __align__(16) T sy[kWarps][NB];
    __shared__ __align__(16) T sw[kWarps][NB];
    __shared__ __align__(16) T sa[kWarps][NB];
    __shared__ int s_done, s_k;
    __shared__ double s_alpha;
    if (threadIdx.x == 0) {
        s_done = sc->done;
        s_k = sc->iter;
        s_alpha = sc->alpha;
    }
    __syncthreads();
    if (s_done) return;
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
    unsigned ntasks;
    if (SCHED == 0) {
        ntasks = (unsigned)d.ntiles;
        // tasks are claimed in the reverse of phase A's order; partials stay
        // indexed by task, so the totals do not depend on the order
        for (unsigned c = next_task(&sc->task_ctr[1], lane); c < ntasks;
             c = next_task(&sc->task_ctr[1], lane)) {
            const unsigned t = ntasks - 1u - c;
            // d.ty: a batched group's own task height (its initial pass runs here)
            const Task tk = task_of_rows<W>(t, d.K, d.tiles_x, d.nz, d.ty > 0 ? d.ty : TY);
            double val[2];
            run_task_b<T, VEC, INIT>(d, tk, s_k, (T)s_alpha, sy[wp], sw[wp], sa[wp], lane, val);
            publish_unit<2>(val, reducer_of(d), ntasks, t, lane);
        }
    } else {
        ntasks = gridDim.x * kWarps;
        const unsigned gw = blockIdx.x * kWarps + wp;
        double v[2] = {0.0, 0.0};
        static_pieces<false>(d.K, d.tiles_x, d.nz, W, d.sgroups, ntasks, gw, [&](const Task &tk) {
            double val[2];
            run_task_b<T, VEC, INIT>(d, tk, s_k, (T)s_alpha, sy[wp], sw[wp], sa[wp], lane, val);
            v[0] += val[0];
            v[1] += val[1];
        });
        publish_unit<2>(v, reducer_of(d), ntasks, gw, lane);
    }
    double tot[2];
    if (reduce_units<2>(reducer_of(d), ntasks, &sc->ticket[kTicketB], &sc->task_ctr[1], tot) &&
        threadIdx.x == 0) {
        const int done = finish_b<INIT>(sc, tot[0], tot[1], s_k, d.eps, d.max_iter, d.guard_limit);
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

// The p updates still pending after the last iteration (phase A adds them
// otherwise): alpha u of the last iteration, and with two pending the one before
// (alpha_pp, the other u buffer), added first.
template <typename T>
__global__ void __launch_bounds__(kThreads) k_finalize(const PcgDesc<T> *__restrict__ dp)
{
    const PcgDesc<T> &d = *dp;
    Scalars *sc = d.sc;
    const int pend = sc->pending;
    if (!pend) return;
    const T alpha = (T)sc->alpha;
    const T alpha_pp = (T)sc->alpha_pp;
    const T *u = d.u[(sc->iter + 1) & 1];
    const T *upp = d.u[sc->iter & 1];
    const long long N = d.n * d.K;
    for (long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x; g < N;
         g += (long long)gridDim.x * blockDim.x) {
        T x = d.p[g];
        if (pend == 2) x += alpha_pp * upp[g];
        d.p[g] = x + alpha * u[g];
    }
}

// Reliable update of the mixed-precision inner solve: keep the iteration count,
// the direction u and d = r.z; the next initial pass continues the recurrence from
// the new residual, whose units are cscale times those of the last one.
static __global__ void k_continue(Scalars *sc, double cscale)
{
    if (threadIdx.x != 0) return;
    sc->cont = 1;
    sc->cscale = cscale;
    sc->done = 0;
    sc->converged = 0;
    sc->status = 0;
    sc->pending = 0;
    sc->guard = 0;
    sc->zero_rhs = 0;
    for (int q = 0; q < 6; ++q) sc->ticket[q] = 0u;
    sc->task_ctr[0] = 0u;
    sc->task_ctr[1] = 0u;
}

static __global__ void k_reset(Scalars *sc, int keep_iter)
{
    if (threadIdx.x != 0) return;
    if (!keep_iter) sc->iter = 0;
    sc->cont = 0;
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
    sc->task_ctr[0] = 0u;
    sc->task_ctr[1] = 0u;
}

// ------------------------------------------------------------------ FP64 residual, conversions

// r = S - A p (FP64), partial ||r||^2 and ||S||^2; last block sets true_rel and rnorm.
static __global__ void __launch_bounds__(kThreads) k_resid64(const ResidDesc *__restrict__ dp)
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

// The stored diagonal of FP64 coefficient slots, w / D: w = omega for ASSOR-II, whose two passes then use
// it as omega D^-1 directly (y, w and z come out scaled by omega, which PCG does
// not see: alpha takes the inverse factor), w = 1 for Jacobi.
static __global__ void k_invd64(const double *__restrict__ D, double *__restrict__ invD, long long m,
                                double w)
{
    for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < m;
         q += (long long)gridDim.x * blockDim.x)
        invD[q] = w / D[q];
}

// FP32 copies of the coefficient slots scaled by a power of two so that the
// FP32 entries are of order one: A32 = scale * A; the stored diagonal is w / D32
// (w = omega for ASSOR-II, 1 for Jacobi, as k_invd64).
static __global__ void k_to_f32(const double *__restrict__ D, const double *__restrict__ aE,
                         const double *__restrict__ aN, float *__restrict__ D32,
                         float *__restrict__ invD32, float *__restrict__ aE32,
                         float *__restrict__ aN32, long long m, Scalars *sc, double w)
{
    const double scale = ldexp(1.0, -ilogb(D[0]));
    if (blockIdx.x == 0 && threadIdx.x == 0) sc->scale = scale;
    for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < m;
         q += (long long)gridDim.x * blockDim.x) {
        const double dd = D[q] * scale;
        D32[q] = (float)dd;
        invD32[q] = (float)(w / dd);
        aE32[q] = (float)(aE[q] * scale);
        aN32[q] = (float)(aN[q] * scale);
    }
}

// b32 = r64 / ||r64|| (unit-norm right-hand side of the inner FP32 solve).
static __global__ void k_make_b32(const double *__restrict__ r64, float *__restrict__ b32, long long N,
                           const Scalars *__restrict__ outer)
{
    const double inv = 1.0 / outer->rnorm;
    for (long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x; g < N;
         g += (long long)gridDim.x * blockDim.x)
        b32[g] = (float)(r64[g] * inv);
}

// p64 += scale * ||r64|| * x32  (delta = A^-1 r64 = scale ||r64|| (scale A)^-1 (r64/||r64||)).
static __global__ void k_update_p64(double *__restrict__ p, const float *__restrict__ x, long long N,
                             const Scalars *__restrict__ outer)
{
    const double f = outer->scale * outer->rnorm;
    for (long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x; g < N;
         g += (long long)gridDim.x * blockDim.x)
        p[g] = fma(f, (double)x[g], p[g]);
}


// ------------------------------------------------------------------ phase B, staged rows
//
// Same arithmetic and order as run_task_b, but the five input rows (r, v, 1/D,
// aE, aN with their halo columns) are staged by cp.async into a per-warp ring of
// D + 1 rows in shared memory, D rows ahead of the row being processed, so the
// loads in flight do not occupy registers.  One commit group per row (empty
// groups keep the count uniform); row jr is consumed after wait_group(D).
// 16-byte copies need VEC * sizeof(T) == 16 and aligned rows.

__device__ __forceinline__ unsigned smem_u32(const void *p)
{
    return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void cp_async16(void *s, const void *g)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(smem_u32(s)), "l"(g) : "memory");
}
template <int BYTES>
__device__ __forceinline__ void cp_async_small(void *s, const void *g)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(smem_u32(s)), "l"(g), "n"(BYTES)
                 : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait()
{
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// ------------------------------------------------------------------ phase A, staged rows
//
// Same arithmetic and order as run_task_a (forward marching), but the six input
// rows (z, u', D, aE, aN, p) and the halo columns (z, u' of lanes 0 and 1, aE of
// lane 0) are staged by cp.async into a per-warp ring of D + 1 rows, D rows
// ahead.  A row's values move to registers (and the aE and u rows to their own
// shared rows) when it is consumed, so the slot that the next copy overwrites is
// never read again.
//
// PAIR: the p updates are applied every second iteration, two at a time
// (p += alpha_pp u'' + alpha' u', u'' the direction before u', read from the u
// buffer this phase overwrites, before it does): on average 2 fewer bytes per
// unknown in FP32 than reading and writing p every iteration.

template <typename T, int VEC, bool PAIR = false>
struct RingA {
    static constexpr int W = 32 * VEC, NB = W + 8, NF = PAIR ? 7 : 6;
    // elements per warp: (D+1) staged rows of NF fields, plus the u and aE rows
    __host__ __device__ static constexpr int per_warp(int D) { return (D + 1) * NF * NB + 2 * NB; }
};

// DREC: the diagonal is not staged but rebuilt from the couplings the row step
// already holds, D = aE + aW + aN + aS (+ the Dirichlet term of the first and last
// rows, read from d.dbnd), as the assembly forms it; 4 bytes fewer per unknown and
// coefficient slot.
template <typename T, int VEC, int TY, int D, bool PAIR = false, bool DREC = false>
__device__ __forceinline__ double run_task_a_staged(const PcgDesc<T> &d, const Task &tk, int k,
                                                    int first, int pend, T alpha_prev, T alpha_pp,
                                                    T beta, T *ring, T *ub, T *ab, int lane)
{
    const bool uz = first == 1;      // u = z (modes of `first` as in run_task_a)
    // p updates: with PAIR only when two are pending (both added), else the pending one
    const bool two = PAIR && pend == 2;
    const bool nop = PAIR ? !two : pend == 0;
    constexpr int W = 32 * VEC;
    constexpr int NB = W + 8, NF = RingA<T, VEC, PAIR>::NF, SLOT = NF * NB;
    constexpr int CH = 16 / (int)sizeof(T);
    static_assert(VEC % CH == 0, "whole 16-byte chunks per lane");
    const int nth = d.nth, nz = d.nz;
    const long long n = d.n;
    RowAcc<T> acc;
    const size_t off = (size_t)tk.cond * (size_t)n;
    const size_t coff = (size_t)d.cslot[tk.cond] * (size_t)n;
    const T *uo_base = d.u[(k + 1) & 1];
    T *un = d.u[k & 1] + off;
    T *vv = d.v + off;
    T *pp = d.p + off;
    const int c0 = tk.i0 + lane * VEC;
    const bool owned = c0 < nth;
    const int g0 = wrap_col(c0, nth);
    const int sown = 4 + lane * VEC;
    // halo: lane 0 -> column i0 - 1 (slot 3), lane 1 -> column i0 + W (slot W + 4);
    // the other lanes read lane 1's slot and write the spare slot W + 7
    const int hg = wrap_col(lane == 0 ? tk.i0 - 1 : tk.i0 + W, nth);
    const int hs = lane == 0 ? 3 : W + 4;
    const int hslot_u = lane < 2 ? hs : W + 7;
    const int hslot_a = lane == 0 ? hs : W + 7;
    // fields: 0 z, 1 u', 2 D, 3 aE, 4 aN, 5 p (, 6 u'': the direction before u')
    const T *src[7] = {d.z + off, uo_base + off, d.D + coff, d.aE + coff, d.aN + coff, pp, un};

    // ring slot of row jr: (jr - (j0 - 1)) mod (D + 1), passed in by the caller
    auto issue = [&](int jr, int sl) {
        if (jr >= 0 && jr < nz && jr >= tk.j0 - 1 && jr <= tk.jend) {
            T *slot = ring + sl * SLOT;
            const size_t rq = (size_t)jr * nth;
            const bool in = jr >= tk.j0 && jr < tk.jend;
#pragma unroll
            for (int f = 0; f < NF; ++f) {
                if ((uz && f == 1) || (nop && f == 5)) continue;     // no u' / no p update
                if (f == 6 && !two) continue;
                if (DREC && f == 2) continue;                        // D rebuilt, not copied
                if (!in && (f == 2 || f == 3 || f >= 5)) continue;
                if (!owned && f >= 5) continue;
#pragma unroll
                for (int c = 0; c < VEC; c += CH) cp_async16(slot + f * NB + sown + c, src[f] + rq + g0 + c);
            }
            if (lane < 2) {
                cp_async_small<sizeof(T)>(slot + hs, src[0] + rq + hg);
                if (!uz) cp_async_small<sizeof(T)>(slot + NB + hs, src[1] + rq + hg);
                if (lane == 0) cp_async_small<sizeof(T)>(slot + 3 * NB + hs, src[3] + rq + hg);
            }
        }
        cp_commit();
    };

    T u_m1[VEC], u_m2[VEC], uo_m1[VEC], D_m1[VEC], e_m1[VEC], n_m1[VEC], n_m2[VEC], p_m1[VEC];
    T upp_m1[VEC];
#pragma unroll
    for (int q = 0; q < VEC; ++q)
        u_m1[q] = u_m2[q] = uo_m1[q] = D_m1[q] = e_m1[q] = n_m1[q] = n_m2[q] = p_m1[q] = upp_m1[q] = T(0);
#pragma unroll
    for (int q = 0; q < D; ++q) issue(tk.j0 - 1 + q, q);
    // one row step: row jr in ring slot sl
    auto step = [&](const int jr, const int sl) {
        issue(jr + D, sl == 0 ? D : sl - 1);
        cp_wait<D>();
        __syncwarp();
        const T *cur = ring + sl * SLOT;
        const bool inrow = jr >= 0 && jr < nz;
        const bool in = inrow && jr >= tk.j0 && jr < tk.jend;
        T zv[VEC], uov[VEC], Dv[VEC], ev[VEC], nv[VEC], pv[VEC], uppv[VEC];
#pragma unroll
        for (int q = 0; q < VEC; ++q) zv[q] = uov[q] = Dv[q] = ev[q] = nv[q] = pv[q] = uppv[q] = T(0);
        T hz = T(0), huo = T(0), he = T(0);
        if (inrow) {
            Vec<T, VEC>::ldrw(cur + sown, zv);
            if (!uz) Vec<T, VEC>::ldrw(cur + NB + sown, uov);
            Vec<T, VEC>::ldrw(cur + 4 * NB + sown, nv);
            if (in) {
                if constexpr (!DREC) Vec<T, VEC>::ldrw(cur + 2 * NB + sown, Dv);
                Vec<T, VEC>::ldrw(cur + 3 * NB + sown, ev);
                if (!nop) Vec<T, VEC>::ldrw(cur + 5 * NB + sown, pv);
                if (two) Vec<T, VEC>::ldrw(cur + 6 * NB + sown, uppv);
            }
            hz = cur[hs];
            if (!uz) huo = cur[NB + hs];
            he = cur[3 * NB + hs];
        }
        T u[VEC];
#pragma unroll
        for (int q = 0; q < VEC; ++q) u[q] = uz ? zv[q] : zv[q] + beta * uov[q];
        const T hu = uz ? hz : hz + beta * huo;
        const int jo = jr - 1;
        if (jo >= tk.j0 && jo < tk.jend) {
            T vout[VEC];
            T rowsum = T(0);
            T bnd[VEC];
            if constexpr (DREC) {
                // Dirichlet term of the first and last rows: d.dbnd[slot][0 or 1][n_theta]
#pragma unroll
                for (int q = 0; q < VEC; ++q) bnd[q] = T(0);
                if (jo == 0 || jo == nz - 1)
                    Vec<T, VEC>::ld(d.dbnd + ((size_t)d.cslot[tk.cond] * 2 + (jo == 0 ? 0 : 1)) * nth + g0,
                                    bnd);
            }
#pragma unroll
            for (int q = 0; q < VEC; ++q) {
                const int s = sown + q;
                const T uE = (q < VEC - 1) ? u_m1[q + 1] : ub[s + 1];
                const T uW = (q > 0) ? u_m1[q - 1] : ub[s - 1];
                const T aW = (q > 0) ? e_m1[q - 1] : ab[s - 1];
                T dg;
                if constexpr (DREC)
                    dg = (((e_m1[q] + aW) + n_m1[q]) + n_m2[q]) + bnd[q];
                else
                    dg = D_m1[q];
                vout[q] = dg * u_m1[q] - e_m1[q] * uE - aW * uW - n_m1[q] * u[q] -
                          n_m2[q] * u_m2[q];
                rowsum += u_m1[q] * vout[q];
            }
            if (owned) {
                const size_t qo = (size_t)jo * nth + g0;
                Vec<T, VEC>::st(un + qo, u_m1);
                Vec<T, VEC>::st(vv + qo, vout);
                if (!nop) {
                    T pn[VEC];
#pragma unroll
                    for (int q = 0; q < VEC; ++q)
                        pn[q] = (two ? p_m1[q] + alpha_pp * upp_m1[q] : p_m1[q]) + alpha_prev * uo_m1[q];
                    Vec<T, VEC>::st(pp + qo, pn);
                }
                acc.add_row(rowsum);
            }
        }
        __syncwarp();
        Vec<T, VEC>::st(ub + sown, u);
        Vec<T, VEC>::st(ab + sown, ev);
        ub[hslot_u] = hu;
        ab[hslot_a] = he;
        __syncwarp();
#pragma unroll
        for (int q = 0; q < VEC; ++q) {
            u_m2[q] = u_m1[q];
            u_m1[q] = u[q];
            uo_m1[q] = uov[q];
            n_m2[q] = n_m1[q];
            n_m1[q] = nv[q];
            D_m1[q] = Dv[q];
            e_m1[q] = ev[q];
            p_m1[q] = pv[q];
            upp_m1[q] = uppv[q];
        }
    };
    int sl = 0;
    for (int jr = tk.j0 - 1; jr <= tk.jend; ++jr) {
        step(jr, sl);
        sl = sl == D ? 0 : sl + 1;
    }
    cp_wait<0>();
    __syncwarp();
    return acc.value();
}

// FP32: the p updates are paired (PAIR above); FP64 adds one every iteration.
// DREC: the diagonal rebuilt from the couplings (run_task_a_staged).
template <typename T, int VEC, int TY, int MINB, int D, int NT = kThreads, bool DREC = false>
__global__ void __launch_bounds__(NT, MINB) k_phase_a_staged(const PcgDesc<T> *__restrict__ dp)
{
    constexpr bool PAIR = sizeof(T) == 4;
    using R = RingA<T, VEC, PAIR>;
    constexpr int W = 32 * VEC;
    const PcgDesc<T> &d = *dp;
    Scalars *sc = d.sc;
    extern __shared__ __align__(16) unsigned char g_dyn_smem_a[];
    __shared__ int s_done, s_k, s_first, s_pend;
    __shared__ double s_alpha, s_beta, s_alpha_pp;
    if (threadIdx.x == 0) {
        s_done = sc->done;
        s_k = sc->iter;
        s_first = sc->first;
        s_pend = sc->pending;
        s_alpha = sc->alpha;
        s_alpha_pp = sc->alpha_pp;
        s_beta = sc->beta;
        if (blockIdx.x == 0) {
            // stop unless phase B's last block asks for another iteration
            if (d.use_cond) cudaGraphSetConditional(d.cond, 0u);
            sc->guard += 1;
        }
    }
    __syncthreads();
    if (s_done) return;
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
    T *mine = reinterpret_cast<T *>(g_dyn_smem_a) + (size_t)wp * R::per_warp(D);
    T *ring = mine;
    T *ub = mine + (D + 1) * R::NF * R::NB;
    T *ab = ub + R::NB;
    const unsigned ntasks = (unsigned)d.ntiles;
    // (tasks are claimed one at a time, when the warp is free: claiming the next one
    // early scatters the tasks that run together and costs their L2 sharing, 8 %)
    for (unsigned t = next_task(&sc->task_ctr[0], lane); t < ntasks;
         t = next_task(&sc->task_ctr[0], lane)) {
        const Task tk = task_of_rows<W>(t, d.K, d.tiles_x, d.nz, d.ty > 0 ? d.ty : TY);
        const double val[1] = {run_task_a_staged<T, VEC, TY, D, PAIR, DREC>(
            d, tk, s_k, s_first, s_pend, (T)s_alpha, (T)s_alpha_pp, (T)s_beta, ring, ub, ab, lane)};
        publish_unit<1>(val, reducer_of(d), ntasks, t, lane);
    }
    double tot[1];
    if (reduce_units<1>(reducer_of(d), ntasks, &sc->ticket[kTicketA], &sc->task_ctr[0], tot) &&
        threadIdx.x == 0)
        finish_a(sc, tot[0], PAIR ? s_pend == 2 : s_pend > 0);
}

template <typename T, int VEC>
struct RingB {
    static constexpr int W = 32 * VEC, NB = W + 8, NF = 5;
    // elements per warp: (D+1) staged rows of NF fields, plus the y and w rows
    __host__ __device__ static constexpr int per_warp(int D) { return (D + 1) * NF * NB + 2 * NB; }
};

// Only lanes 0..3 issue the halo copies (copies of one word from many lanes into
// one shared slot serialise).  FP32: one body for every task, branch-free halo
// arithmetic as in run_task_b (reading lane 3's column).  FP64 (bound by the
// FP64 pipe, where it measured faster): interior tasks take a second body
// (EDGE = false: the strip and its halo touch neither theta edge, 2 <= i0 and
// i0 + W + 2 <= n_theta), with the periodic-wrap tests compiled out.
template <typename T, int VEC, int TY, bool INIT, int D, bool EDGE>
__device__ __forceinline__ void run_task_b_staged(const PcgDesc<T> &d, const Task &tk, int k,
                                                  T alpha, T *ring, T *yb, T *wb, int lane,
                                                  double (&out)[2])
{
    constexpr int W = 32 * VEC;
    constexpr int NB = W + 8, NF = 5, SLOT = NF * NB;
    constexpr int kSpare = W + 7;
    constexpr bool BF = sizeof(T) == 4;
    constexpr int CH = 16 / (int)sizeof(T);      // elements per 16-byte copy
    static_assert(VEC % CH == 0, "whole 16-byte chunks per lane");
    const int nth = d.nth, nz = d.nz;
    const long long n = d.n;
    const bool assor = (d.precond == 1);
    RowAcc<T> arz, arr;
    const size_t off = (size_t)tk.cond * (size_t)n;
    const size_t coff = (size_t)d.cslot[tk.cond] * (size_t)n;
    const int c0 = tk.i0 + lane * VEC;
    const bool owned = c0 < nth;
    const int g0 = EDGE ? wrap_col(c0, nth) : c0;
    // n_theta % VEC == 0: only element 0 of a lane can be column 0 and only
    // element VEC - 1 column n_theta - 1 (the seam tests below are static otherwise)
    const bool at_w = g0 == 0, at_e = g0 + VEC == nth;
    const int sown = 4 + lane * VEC;
    const int hl = lane < 4 ? lane : 3;
    const int hoff = hl < 2 ? hl - 2 : W + (hl - 2);
    const int hg = EDGE ? wrap_col(tk.i0 + hoff, nth) : tk.i0 + hoff;
    const int hs = hl < 2 ? hl + 2 : W + 2 + hl;
    const int hslot_y = lane < 4 ? hs : kSpare;
    const int hslot_w = (lane == 1 || lane == 2) ? hs : kSpare;
    const T *aE = d.aE + coff;
    // row pointers at row j0 - 1 (own columns / halo column); advanced by n_theta per row
    const long long row0 = (long long)(tk.j0 - 1) * nth;
    const T *src[NF] = {d.r[k & 1] + off, d.v + off, d.invD + coff, d.aE + coff, d.aN + coff};
    T *rn = d.r[(k + 1) & 1] + off + (long long)tk.j0 * nth + g0;
    T *zo = d.z + off + (long long)tk.j0 * nth + g0;

    // ring slot of row jr: (jr - (j0 - 1)) mod (D + 1), passed in by the caller
    auto issue = [&](int jr, int sl) {
        if (jr >= 0 && jr < nz && jr <= tk.jend) {
            T *slot = ring + sl * SLOT;
            const long long rq = row0 + (long long)(jr - tk.j0 + 1) * nth;
#pragma unroll
            for (int f = 0; f < NF; ++f) {
                if (INIT && f == 1) continue;
#pragma unroll
                for (int c = 0; c < VEC; c += CH) cp_async16(slot + f * NB + sown + c, src[f] + rq + g0 + c);
            }
            if (lane < 4) {
#pragma unroll
                for (int f = 0; f < NF; ++f) {
                    if (INIT && f == 1) continue;
                    cp_async_small<sizeof(T)>(slot + f * NB + hs, src[f] + rq + hg);
                }
            }
        }
        cp_commit();
    };

    T y_m1[VEC], w_m1[VEC], od_m1[VEC], n_m1[VEC], e_m1[VEC], r_m1[VEC];
#pragma unroll
    for (int q = 0; q < VEC; ++q) y_m1[q] = w_m1[q] = od_m1[q] = n_m1[q] = e_m1[q] = r_m1[q] = T(0);
    T hy_m1 = T(0), hn_m1 = T(0), he_m1 = T(0);
#pragma unroll
    for (int q = 0; q < D; ++q) issue(tk.j0 - 1 + q, q);
    // one row step: row jr in ring slot sl
    auto step = [&](const int jr, const int sl) {
        issue(jr + D, sl == 0 ? D : sl - 1);
        cp_wait<D>();
        __syncwarp();
        const T *cur = ring + sl * SLOT;
        const bool inrow = jr >= 0 && jr < nz;
        T r1[VEC], y[VEC], dI[VEC], ev[VEC], nv[VEC];
        T hy = T(0), hd = T(0), he = T(0), hn = T(0);
        if (inrow) {
            T rv[VEC], vx[VEC];
            Vec<T, VEC>::ldrw(cur + 0 * NB + sown, rv);
            if (!INIT) Vec<T, VEC>::ldrw(cur + 1 * NB + sown, vx);
            Vec<T, VEC>::ldrw(cur + 2 * NB + sown, dI);
            Vec<T, VEC>::ldrw(cur + 3 * NB + sown, ev);
            Vec<T, VEC>::ldrw(cur + 4 * NB + sown, nv);
#pragma unroll
            for (int q = 0; q < VEC; ++q) {
                r1[q] = INIT ? rv[q] : rv[q] - alpha * vx[q];
                y[q] = r1[q] * dI[q];
            }
            if (BF || lane < 4) {
                const T hr = INIT ? cur[hs] : cur[hs] - alpha * cur[NB + hs];
                hd = cur[2 * NB + hs];
                he = cur[3 * NB + hs];
                hn = cur[4 * NB + hs];
                hy = hr * hd;
            }
        } else {
#pragma unroll
            for (int q = 0; q < VEC; ++q) r1[q] = y[q] = dI[q] = ev[q] = nv[q] = T(0);
        }
        Vec<T, VEC>::st(yb + sown, y);
        if (BF || lane < 4) yb[hslot_y] = hy;
        // FP32: aE(jr - 1, n_theta - 1) from lane 1 (column i0 - 1): wrapped west
        // coupling of column 0; FP64 loads it where it is needed
        T aw_wrap = T(0);
        if (BF) aw_wrap = __shfl_sync(0xffffffffu, he_m1, 1);
        __syncwarp();
        T w[VEC], od[VEC];                       // od = omega D^-1, reused by the second pass
        T hw = T(0);
#pragma unroll
        for (int q = 0; q < VEC; ++q) w[q] = od[q] = T(0);
        if (assor && inrow && jr >= tk.j0) {
            const T *ab = cur + 3 * NB;          // aE of row jr with its halo
            const bool south = jr > 0;
#pragma unroll
            for (int q = 0; q < VEC; ++q) {
                const int s = sown + q;
                T sum = south ? n_m1[q] * y_m1[q] : T(0);
                const T aW = (q > 0) ? ev[q - 1] : ab[s - 1];
                const T yW = (q > 0) ? y[q - 1] : yb[s - 1];
                if (!EDGE || q > 0 || !at_w) sum += aW * yW;
                if (EDGE && q == VEC - 1 && at_e) sum += ev[q] * ((q < VEC - 1) ? y[q + 1] : yb[s + 1]);
                od[q] = dI[q];
                w[q] = y[q] + od[q] * sum;
            }
            if (BF || lane == 1 || lane == 2) {
                T sum = south ? hn_m1 * hy_m1 : T(0);
                if (!EDGE || hg > 0) sum += ab[hs - 1] * yb[hs - 1];
                if (EDGE && hg == nth - 1) sum += he * yb[hs + 1];
                hw = hy + hd * sum;
            }
        }
        const int jo = jr - 1;
        if (jo >= tk.j0 && jo < tk.jend) {
            T zz[VEC];
            T rz = T(0), rr = T(0);
            const bool north = jo < nz - 1;
#pragma unroll
            for (int q = 0; q < VEC; ++q) {
                if (assor) {
                    const int s = sown + q;
                    T sum = north ? n_m1[q] * w[q] : T(0);
                    const T wE = (q < VEC - 1) ? w_m1[q + 1] : wb[s + 1];
                    if (!EDGE || q < VEC - 1 || !at_e) sum += e_m1[q] * wE;
                    if (EDGE && q == 0 && at_w)
                        sum += (BF ? aw_wrap : __ldg(aE + (size_t)jo * nth + nth - 1)) *
                               ((q > 0) ? w_m1[q - 1] : wb[s - 1]);
                    zz[q] = w_m1[q] + od_m1[q] * sum;   // Eq. 3.6 without its factor c1
                } else {
                    zz[q] = y_m1[q];
                }
                rz += r_m1[q] * zz[q];
                rr += r_m1[q] * r_m1[q];
            }
            if (owned) {
                Vec<T, VEC>::st(zo, zz);
                if (!INIT) Vec<T, VEC>::st(rn, r_m1);
                arz.add_row(rz);
                arr.add_row(rr);
            }
            zo += nth;
            rn += nth;
        }
        __syncwarp();
        if (assor) {
            Vec<T, VEC>::st(wb + sown, w);
            if (BF || lane == 1 || lane == 2) wb[hslot_w] = hw;
        }
        __syncwarp();
#pragma unroll
        for (int q = 0; q < VEC; ++q) {
            y_m1[q] = y[q];
            w_m1[q] = w[q];
            od_m1[q] = od[q];
            n_m1[q] = nv[q];
            e_m1[q] = ev[q];
            r_m1[q] = r1[q];
        }
        hy_m1 = hy;
        hn_m1 = hn;
        he_m1 = he;
    };
    int sl = 0;
    for (int jr = tk.j0 - 1; jr <= tk.jend; ++jr) {
        step(jr, sl);
        sl = sl == D ? 0 : sl + 1;
    }
    cp_wait<0>();
    __syncwarp();
    out[0] = arz.value();
    out[1] = arr.value();
}

template <typename T, int VEC, int TY, int MINB, bool INIT, int D, int NT = kThreads>
__global__ void __launch_bounds__(NT, MINB) k_phase_b_staged(const PcgDesc<T> *__restrict__ dp)
{
    using R = RingB<T, VEC>;
    const PcgDesc<T> &d = *dp;
    Scalars *sc = d.sc;
    extern __shared__ __align__(16) unsigned char g_dyn_smem[];
    __shared__ int s_done, s_k;
    __shared__ double s_alpha;
    if (threadIdx.x == 0) {
        s_done = sc->done;
        s_k = sc->iter;
        s_alpha = sc->alpha;
    }
    __syncthreads();
    if (s_done) return;
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
    T *mine = reinterpret_cast<T *>(g_dyn_smem) + (size_t)wp * R::per_warp(D);
    T *ring = mine;
    T *yb = mine + (D + 1) * R::NF * R::NB;
    T *wb = yb + R::NB;
    const unsigned ntasks = (unsigned)d.ntiles;
    constexpr int W = 32 * VEC;
    for (unsigned c = next_task(&sc->task_ctr[1], lane); c < ntasks;
         c = next_task(&sc->task_ctr[1], lane)) {
        const unsigned t = ntasks - 1u - c;    // reverse of phase A's order (L2 reuse)
        double val[2];
        const Task tk = task_of_rows<W>(t, d.K, d.tiles_x, d.nz, d.ty > 0 ? d.ty : TY);
        if (sizeof(T) == 8 && tk.i0 >= 2 && tk.i0 + W + 2 <= d.nth)
            run_task_b_staged<T, VEC, TY, INIT, D, false>(d, tk, s_k, (T)s_alpha, ring, yb, wb, lane, val);
        else
            run_task_b_staged<T, VEC, TY, INIT, D, true>(d, tk, s_k, (T)s_alpha, ring, yb, wb, lane, val);
        publish_unit<2>(val, reducer_of(d), ntasks, t, lane);
    }
    double tot[2];
    if (reduce_units<2>(reducer_of(d), ntasks, &sc->ticket[kTicketB], &sc->task_ctr[1], tot) &&
        threadIdx.x == 0) {
        const int done = finish_b<INIT>(sc, tot[0], tot[1], s_k, d.eps, d.max_iter, d.guard_limit);
        if (d.use_cond) cudaGraphSetConditional(d.cond, done ? 0u : 1u);
    }
}

// ------------------------------------------------------------------ phase B, bulk-copied rows
//
// The arithmetic and order of run_task_b_staged (so the results are bitwise the
// same), with the ring filled differently: one lane per warp copies each field's
// whole row segment, columns i0 - 4 .. i0 + W + 3 (W + 8 elements, halo
// included), with cp.async.bulk global -> shared, completing on the ring slot's
// mbarrier (transaction count = the bytes of the row).  The other 31 lanes issue
// no copy instructions and take no address arithmetic for them.  Slot s of a
// field row holds column (i0 - 4 + s) mod n_theta; at the periodic seam a row is
// copied in two pieces (the 16-byte wrap piece and the rest).  Needs
// n_theta % 4 == 0 (16-byte pieces), n_theta >= W + 8 (at most one wrap per row)
// and 16-byte aligned fields.
//
// Every wait on an mbarrier is bounded: after kBarSpin failed polls the warp
// records GMAF_TIMEOUT in the run's scalars, stops, waits (again bounded) for
// the copies it still has in flight and leaves its task loop.

constexpr unsigned kBarSpin = 1u << 22;

__device__ __forceinline__ void mbar_init(unsigned long long *bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_init_fence()
{
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async_smem()
{
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_tx(unsigned long long *bar, unsigned tx)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(tx)
                 : "memory");
}
__device__ __forceinline__ void mbar_arrive(unsigned long long *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_test(unsigned long long *bar, unsigned parity)
{
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bounded wait for the phase of `parity` to complete; false if it never did.
__device__ __forceinline__ bool mbar_wait(unsigned long long *bar, unsigned parity)
{
    for (unsigned k = 0; k < kBarSpin; ++k)
        if (mbar_test(bar, parity)) return true;
    return false;
}
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, unsigned bytes,
                                         unsigned long long *bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

// The per-warp ring of D + 1 slots and their barriers, for one warp.
template <int D>
struct BulkRing {
    unsigned long long *bar;   // [D + 1] mbarriers
    unsigned parity;           // bit k: phase parity the next wait on slot k expects
    unsigned pend;             // bit k: slot k has a phase armed and not yet waited for
    bool ok;                   // false once a wait gave up
};

template <typename T, int VEC, int TY, bool INIT, int D>
__device__ __forceinline__ void run_task_b_bulk(const PcgDesc<T> &d, const Task &tk, int k, T alpha,
                                                T *ring, T *yb, T *wb, BulkRing<D> &br, int lane,
                                                double (&out)[2])
{
    constexpr int W = 32 * VEC;
    constexpr int NB = W + 8, NF = 5, SLOT = NF * NB;
    constexpr int kSpare = W + 7;
    constexpr bool BF = sizeof(T) == 4;
    const int nth = d.nth, nz = d.nz;
    const long long n = d.n;
    const bool assor = (d.precond == 1);
    RowAcc<T> arz, arr;
    const size_t off = (size_t)tk.cond * (size_t)n;
    const size_t coff = (size_t)d.cslot[tk.cond] * (size_t)n;
    const int c0 = tk.i0 + lane * VEC;
    const bool owned = c0 < nth;
    const int g0 = wrap_col(c0, nth);
    const bool at_w = g0 == 0, at_e = g0 + VEC == nth;   // (see run_task_b_staged)
    const int sown = 4 + lane * VEC;
    const int hl = lane < 4 ? lane : 3;
    const int hoff = hl < 2 ? hl - 2 : W + (hl - 2);
    const int hg = wrap_col(tk.i0 + hoff, nth);
    const int hs = hl < 2 ? hl + 2 : W + 2 + hl;
    const int hslot_y = lane < 4 ? hs : kSpare;
    const int hslot_w = (lane == 1 || lane == 2) ? hs : kSpare;
    T *rn = d.r[(k + 1) & 1] + off + (long long)tk.j0 * nth + g0;
    T *zo = d.z + off + (long long)tk.j0 * nth + g0;

    // copy pieces of a row segment (lane 0): columns [a, b) = [i0 - 4, i0 + W + 4)
    // mapped into [0, n_theta); a < 0 only when i0 = 0, b > n_theta only at the last tile
    const int a = tk.i0 - 4, b = tk.i0 + W + 4;
    const int m_lo = a < 0 ? 0 : a, m_hi = b < nth ? b : nth;
    const unsigned m_bytes = (unsigned)(m_hi - m_lo) * sizeof(T);
    const int m_dst = m_lo - a;
    const int x_src = a < 0 ? a + nth : 0;                 // the wrap piece
    const int x_dst = a < 0 ? 0 : nth - a;
    const unsigned x_bytes = a < 0 ? (unsigned)(-a) * sizeof(T) : (b > nth ? (unsigned)(b - nth) * sizeof(T) : 0u);
    const T *src[NF] = {d.r[k & 1] + off, d.v + off, d.invD + coff, d.aE + coff, d.aN + coff};
    constexpr int NFR = INIT ? NF - 1 : NF;                // fields copied (no v in the initial pass)
    const unsigned row_bytes = (unsigned)NFR * (unsigned)NB * sizeof(T);

    auto issue = [&](int jr) {
        if (jr > tk.jend || !br.ok) return;                 // rows past the task are never consumed
        br.pend |= 1u << ((jr + 1) % (D + 1));              // (uniform: every lane keeps the mask)
        if (lane == 0) {
            unsigned long long *bar = &br.bar[(jr + 1) % (D + 1)];
            if (jr >= 0 && jr < nz) {
                T *slot = ring + ((jr + 1) % (D + 1)) * SLOT;
                const long long rq = (long long)jr * nth;
                // the slot's last generic reads (an earlier row) precede the async writes
                fence_proxy_async_smem();
                mbar_arrive_tx(bar, row_bytes);
#pragma unroll
                for (int f = 0; f < NF; ++f) {
                    if (INIT && f == 1) continue;
                    T *dst = slot + f * NB;
                    bulk_g2s(dst + m_dst, src[f] + rq + m_lo, m_bytes, bar);
                    if (x_bytes) bulk_g2s(dst + x_dst, src[f] + rq + x_src, x_bytes, bar);
                }
            } else {
                mbar_arrive(bar);                           // boundary row: nothing to copy
            }
        }
    };

    T y_m1[VEC], w_m1[VEC], od_m1[VEC], n_m1[VEC], e_m1[VEC], r_m1[VEC];
#pragma unroll
    for (int q = 0; q < VEC; ++q) y_m1[q] = w_m1[q] = od_m1[q] = n_m1[q] = e_m1[q] = r_m1[q] = T(0);
    T hy_m1 = T(0), hn_m1 = T(0), he_m1 = T(0);
#pragma unroll
    for (int q = 0; q < D; ++q) issue(tk.j0 - 1 + q);
    for (int jr = tk.j0 - 1; jr <= tk.jend; ++jr) {
        issue(jr + D);
        const int sl = (jr + 1) % (D + 1);
        if (br.ok) {
            br.ok = mbar_wait(&br.bar[sl], (br.parity >> sl) & 1u);
            br.ok = __all_sync(0xffffffffu, br.ok);
        }
        if (!br.ok) break;
        br.parity ^= 1u << sl;
        br.pend &= ~(1u << sl);
        const T *cur = ring + sl * SLOT;
        const bool inrow = jr >= 0 && jr < nz;
        T r1[VEC], y[VEC], dI[VEC], ev[VEC], nv[VEC];
        T hy = T(0), hd = T(0), he = T(0), hn = T(0);
        if (inrow) {
            T rv[VEC], vx[VEC];
            Vec<T, VEC>::ldrw(cur + 0 * NB + sown, rv);
            if (!INIT) Vec<T, VEC>::ldrw(cur + 1 * NB + sown, vx);
            Vec<T, VEC>::ldrw(cur + 2 * NB + sown, dI);
            Vec<T, VEC>::ldrw(cur + 3 * NB + sown, ev);
            Vec<T, VEC>::ldrw(cur + 4 * NB + sown, nv);
#pragma unroll
            for (int q = 0; q < VEC; ++q) {
                r1[q] = INIT ? rv[q] : rv[q] - alpha * vx[q];
                y[q] = r1[q] * dI[q];
            }
            if (BF || lane < 4) {
                const T hr = INIT ? cur[hs] : cur[hs] - alpha * cur[NB + hs];
                hd = cur[2 * NB + hs];
                he = cur[3 * NB + hs];
                hn = cur[4 * NB + hs];
                hy = hr * hd;
            }
        } else {
#pragma unroll
            for (int q = 0; q < VEC; ++q) r1[q] = y[q] = dI[q] = ev[q] = nv[q] = T(0);
        }
        Vec<T, VEC>::st(yb + sown, y);
        if (BF || lane < 4) yb[hslot_y] = hy;
        T aw_wrap = T(0);
        if (BF) aw_wrap = __shfl_sync(0xffffffffu, he_m1, 1);
        __syncwarp();
        T w[VEC], od[VEC];
        T hw = T(0);
#pragma unroll
        for (int q = 0; q < VEC; ++q) w[q] = od[q] = T(0);
        if (assor && inrow && jr >= tk.j0) {
            const T *ab = cur + 3 * NB;
            const bool south = jr > 0;
#pragma unroll
            for (int q = 0; q < VEC; ++q) {
                const int s = sown + q;
                T sum = south ? n_m1[q] * y_m1[q] : T(0);
                const T aW = (q > 0) ? ev[q - 1] : ab[s - 1];
                const T yW = (q > 0) ? y[q - 1] : yb[s - 1];
                if (q > 0 || !at_w) sum += aW * yW;
                if (q == VEC - 1 && at_e) sum += ev[q] * ((q < VEC - 1) ? y[q + 1] : yb[s + 1]);
                od[q] = dI[q];
                w[q] = y[q] + od[q] * sum;
            }
            if (BF || lane == 1 || lane == 2) {
                T sum = south ? hn_m1 * hy_m1 : T(0);
                if (hg > 0) sum += ab[hs - 1] * yb[hs - 1];
                if (hg == nth - 1) sum += he * yb[hs + 1];
                hw = hy + hd * sum;
            }
        }
        const int jo = jr - 1;
        if (jo >= tk.j0 && jo < tk.jend) {
            T zz[VEC];
            T rz = T(0), rr = T(0);
            const bool north = jo < nz - 1;
#pragma unroll
            for (int q = 0; q < VEC; ++q) {
                if (assor) {
                    const int s = sown + q;
                    T sum = north ? n_m1[q] * w[q] : T(0);
                    const T wE = (q < VEC - 1) ? w_m1[q + 1] : wb[s + 1];
                    if (q < VEC - 1 || !at_e) sum += e_m1[q] * wE;
                    if (q == 0 && at_w)
                        sum += (BF ? aw_wrap : d.aE[coff + (size_t)jo * nth + nth - 1]) *
                               ((q > 0) ? w_m1[q - 1] : wb[s - 1]);
                    zz[q] = w_m1[q] + od_m1[q] * sum;   // Eq. 3.6 without its factor c1
                } else {
                    zz[q] = y_m1[q];
                }
                rz += r_m1[q] * zz[q];
                rr += r_m1[q] * r_m1[q];
            }
            if (owned) {
                Vec<T, VEC>::st(zo, zz);
                if (!INIT) Vec<T, VEC>::st(rn, r_m1);
                arz.add_row(rz);
                arr.add_row(rr);
            }
            zo += nth;
            rn += nth;
        }
        __syncwarp();
        if (assor) {
            Vec<T, VEC>::st(wb + sown, w);
            if (BF || lane == 1 || lane == 2) wb[hslot_w] = hw;
        }
        __syncwarp();
#pragma unroll
        for (int q = 0; q < VEC; ++q) {
            y_m1[q] = y[q];
            w_m1[q] = w[q];
            od_m1[q] = od[q];
            n_m1[q] = nv[q];
            e_m1[q] = ev[q];
            r_m1[q] = r1[q];
        }
        hy_m1 = hy;
        hn_m1 = hn;
        he_m1 = he;
    }
    out[0] = arz.value();
    out[1] = arr.value();
}

// After a wait gave up: wait (bounded) for every phase the warp still has
// outstanding, so that no copy lands in shared memory after the block exits.
template <int D>
__device__ __forceinline__ void bulk_drain(BulkRing<D> &br)
{
#pragma unroll
    for (int sl = 0; sl < D + 1; ++sl)
        if ((br.pend >> sl) & 1u) mbar_wait(&br.bar[sl], (br.parity >> sl) & 1u);
    br.pend = 0u;
}

template <typename T, int VEC, int TY, int MINB, bool INIT, int D>
__global__ void __launch_bounds__(kThreads, MINB) k_phase_b_bulk(const PcgDesc<T> *__restrict__ dp)
{
    using R = RingB<T, VEC>;
    const PcgDesc<T> &d = *dp;
    Scalars *sc = d.sc;
    extern __shared__ __align__(128) unsigned char g_dyn_smem_bk[];
    __shared__ __align__(8) unsigned long long s_bar[kWarps][D + 1];
    __shared__ int s_done, s_k;
    __shared__ double s_alpha;
    if (threadIdx.x == 0) {
        s_done = sc->done;
        s_k = sc->iter;
        s_alpha = sc->alpha;
    }
    __syncthreads();
    if (s_done) return;
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
    T *mine = reinterpret_cast<T *>(g_dyn_smem_bk) + (size_t)wp * R::per_warp(D);
    T *ring = mine;
    T *yb = mine + (D + 1) * R::NF * R::NB;
    T *wb = yb + R::NB;
    BulkRing<D> br{s_bar[wp], 0u, 0u, true};
    if (lane == 0) {
#pragma unroll
        for (int q = 0; q < D + 1; ++q) mbar_init(&br.bar[q], 1);
        mbar_init_fence();
    }
    __syncwarp();
    const unsigned ntasks = (unsigned)d.ntiles;
    constexpr int W = 32 * VEC;
    for (unsigned c = next_task(&sc->task_ctr[1], lane); c < ntasks;
         c = next_task(&sc->task_ctr[1], lane)) {
        const unsigned t = ntasks - 1u - c;    // reverse of phase A's order (L2 reuse)
        double val[2] = {0.0, 0.0};
        if (br.ok) {
            const Task tk = task_of_rows<W>(t, d.K, d.tiles_x, d.nz, d.ty > 0 ? d.ty : TY);
            run_task_b_bulk<T, VEC, TY, INIT, D>(d, tk, s_k, (T)s_alpha, ring, yb, wb, br, lane, val);
            if (!br.ok) {
                // a wait gave up: record it and drain (bounded) what is in flight; the
                // warp keeps publishing (zero) sums for the tasks it still takes, so the
                // launch's reductions complete, and the run ends with GMAF_TIMEOUT
                if (lane == 0) {
                    sc->status = GMAF_TIMEOUT;
                    __threadfence();
                }
                bulk_drain<D>(br);
            }
        }
        publish_unit<2>(val, reducer_of(d), ntasks, t, lane);
    }
    double tot[2];
    if (reduce_units<2>(reducer_of(d), ntasks, &sc->ticket[kTicketB], &sc->task_ctr[1], tot) &&
        threadIdx.x == 0) {
        int done = finish_b<INIT>(sc, tot[0], tot[1], s_k, d.eps, d.max_iter, d.guard_limit);
        if (sc->status == GMAF_TIMEOUT) {
            sc->done = 1;
            done = 1;
        }
        if (d.use_cond) cudaGraphSetConditional(d.cond, done ? 0u : 1u);
    }
}

}  // namespace gmaf
