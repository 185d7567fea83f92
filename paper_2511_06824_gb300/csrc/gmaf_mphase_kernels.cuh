// Batched PCG phase kernels: several joint systems of uneven grids in one
// persistent launch per CG phase, used by the continuous-batching server and by
// the asynchronized criterion (one condition per group).  Built on the task
// bodies of the joint phase kernels (gmaf_pcg_kernels.cuh).
#pragma once

#include "gmaf_pcg_kernels.cuh"

namespace gmaf {

// ------------------------------------------------------------------ batched groups
//
// Several joint systems ("groups": requests of uneven grids, each with its own
// scalars, synchronized criterion, buffers and task height d.ty) in one
// persistent launch per CG phase.  Global task t belongs to group g with task_off[g] <= t < task_off[g+1].
// Groups whose run is done are skipped (a device-side active mask).  Each task
// publishes its sums at its global index.  The sums of a group are reduced in
// two levels relative to the group (chunks of kChunk of its tasks, then its
// chunks), in a fixed order, so a group's iterates do not depend on the other
// groups; the warp that completes a group applies the group's scalar update at
// once, so groups finish in parallel, and the last block only tells whether
// any group is still active.

constexpr int kMaxGroups = 64;

template <typename T>
struct MultiDesc {
    int ngroups;
    unsigned total_tasks;
    unsigned task_off[kMaxGroups + 1];
    const PcgDesc<T> *groups;      // device array [ngroups]
    Scalars *msc;                  // tickets and task counters of the batched launches
    double *partials;              // [total_tasks][2]
    unsigned chunk_off[kMaxGroups + 1];   // first chunk of each group (kChunk tasks a chunk)
    double *chunk_sum;             // [chunks][2]
    unsigned *chunk_ctr;           // [chunks], zero between launches
    unsigned *group_ctr;           // [ngroups], zero between launches
};

// Task t of group g has published its NV sums at partials[t].  Counts it in its
// chunk; the warp completing the chunk stores the chunk sum (the chunk's tasks
// in order) and counts the chunk in the group; the warp completing the group
// gets the group's totals (its chunk sums in order) and returns true.
template <int NV, typename T>
__device__ __forceinline__ bool group_complete(const MultiDesc<T> &m, int g, unsigned t, int lane,
                                               double (&tot)[NV])
{
    const unsigned off = m.task_off[g], tl = t - off, ntl = m.task_off[g + 1] - off;
    const unsigned cl = tl / kChunk, c = m.chunk_off[g] + cl;
    const unsigned cnt = min((unsigned)kChunk, ntl - cl * kChunk);
    unsigned prev = 0;
    if (lane == 0) {
        __threadfence();
        prev = atomicAdd(&m.chunk_ctr[c], 1u);
    }
    prev = __shfl_sync(0xffffffffu, prev, 0);
    if (prev != cnt - 1) return false;
    __threadfence();
    const unsigned u = off + cl * kChunk + (unsigned)lane;
#pragma unroll
    for (int q = 0; q < NV; ++q) {
        const double x = warp_sum_d((unsigned)lane < cnt ? __ldcg(&m.partials[(size_t)u * NV + q]) : 0.0);
        if (lane == 0) m.chunk_sum[(size_t)c * 2 + q] = x;
    }
    const unsigned c0 = m.chunk_off[g], nch = m.chunk_off[g + 1] - c0;
    if (lane == 0) {
        m.chunk_ctr[c] = 0u;
        __threadfence();
        prev = atomicAdd(&m.group_ctr[g], 1u);
    }
    prev = __shfl_sync(0xffffffffu, prev, 0);
    if (prev != nch - 1) return false;
    __threadfence();
#pragma unroll
    for (int q = 0; q < NV; ++q) {
        double a = 0.0;
        for (unsigned i = (unsigned)lane; i < nch; i += 32) a += __ldcg(&m.chunk_sum[(size_t)(c0 + i) * 2 + q]);
        tot[q] = warp_sum_d(a);
    }
    if (lane == 0) m.group_ctr[g] = 0u;
    return true;
}

__device__ __forceinline__ int group_of(const unsigned *off, int ng, unsigned t)
{
    int lo = 0, hi = ng - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (off[mid] <= t) lo = mid; else hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ bool last_block(unsigned *ticket)
{
    __shared__ int s_last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned t = atomicAdd(ticket, 1u);
        s_last = (t == gridDim.x - 1);
    }
    __syncthreads();
    if (s_last) __threadfence();
    return s_last != 0;
}

// D > 0: the input rows are staged D rows ahead through a per-warp shared ring
// (dynamic shared memory of kWarps * RingA<T, VEC, PAIR>::per_warp(D) elements);
// in FP32 the staged phase pairs the p updates as the joint kernel does.
template <typename T, int VEC, int TY, int MINB, int D>
__global__ void __launch_bounds__(kThreads, MINB) k_mphase_a(const MultiDesc<T> *__restrict__ mp)
{
    constexpr bool PAIR = D > 0 && sizeof(T) == 4;
    constexpr int W = 32 * VEC;
    constexpr int NB = W + 8;
    const MultiDesc<T> &m = *mp;
    __shared__ int s_idle;
    if (threadIdx.x == 0) s_idle = m.msc->done;    // every group finished earlier this round
    __syncthreads();
    if (s_idle) return;
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
    T *ring = nullptr, *ub, *ab;
    if constexpr (D > 0) {
        extern __shared__ __align__(16) unsigned char g_dyn_smem_ma[];
        ring = reinterpret_cast<T *>(g_dyn_smem_ma) + (size_t)wp * RingA<T, VEC, PAIR>::per_warp(D);
        ub = ring + (D + 1) * RingA<T, VEC, PAIR>::NF * NB;
        ab = ub + NB;
    } else {
        __shared__ __align__(16) T su[kWarps][NB];
        __shared__ __align__(16) T sa[kWarps][NB];
        ub = su[wp];
        ab = sa[wp];
    }
    for (unsigned t = next_task(&m.msc->task_ctr[0], lane); t < m.total_tasks;
         t = next_task(&m.msc->task_ctr[0], lane)) {
        const int g = group_of(m.task_off, m.ngroups, t);
        const PcgDesc<T> &d = m.groups[g];
        int done = 0, k = 0, first = 0, pend = 0;
        double alpha = 0.0, beta = 0.0, alpha_pp = 0.0;
        if (lane == 0) {
            done = d.sc->done;
            k = d.sc->iter;
            first = d.sc->first;
            pend = d.sc->pending;
            alpha = d.sc->alpha;
            alpha_pp = d.sc->alpha_pp;
            beta = d.sc->beta;
        }
        done = __shfl_sync(0xffffffffu, done, 0);
        k = __shfl_sync(0xffffffffu, k, 0);
        first = __shfl_sync(0xffffffffu, first, 0);
        pend = __shfl_sync(0xffffffffu, pend, 0);
        alpha = __shfl_sync(0xffffffffu, alpha, 0);
        alpha_pp = __shfl_sync(0xffffffffu, alpha_pp, 0);
        beta = __shfl_sync(0xffffffffu, beta, 0);
        double val[1] = {0.0};
        if (!done) {
            const Task tk = task_of_rows<W>(t - m.task_off[g], d.K, d.tiles_x, d.nz, d.ty > 0 ? d.ty : TY);
            if constexpr (D > 0)
                val[0] = run_task_a_staged<T, VEC, TY, D, PAIR>(d, tk, k, first, pend, (T)alpha,
                                                                (T)alpha_pp, (T)beta, ring, ub, ab, lane);
            else
                val[0] = run_task_a<T, VEC, false>(d, tk, k, first, pend, (T)alpha, (T)beta, ub, ab,
                                                   lane);
        }
        publish_task<1>(val, m.partials, t, lane);
        double tot[1];
        if (group_complete<1>(m, g, t, lane, tot) && lane == 0 && !done) {   // active all launch
            d.sc->guard += 1;
            finish_a(d.sc, tot[0], PAIR ? pend == 2 : pend > 0);
        }
    }
    if (!last_block(&m.msc->ticket[kTicketA])) return;
    if (threadIdx.x == 0) {
        m.msc->ticket[kTicketA] = 0u;
        m.msc->task_ctr[0] = 0u;
    }
}

// D > 0: staged D rows ahead (dynamic shared memory of kWarps *
// RingB<T, VEC>::per_warp(D) elements).
template <typename T, int VEC, int TY, int MINB, int D>
__global__ void __launch_bounds__(kThreads, MINB) k_mphase_b(const MultiDesc<T> *__restrict__ mp)
{
    constexpr int W = 32 * VEC;
    constexpr int NB = W + 8;
    const MultiDesc<T> &m = *mp;
    __shared__ int s_idle;
    if (threadIdx.x == 0) s_idle = m.msc->done;
    __syncthreads();
    if (s_idle) return;
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
    T *ring = nullptr, *yb, *wb, *ab = nullptr;
    if constexpr (D > 0) {
        extern __shared__ __align__(16) unsigned char g_dyn_smem_mb[];
        ring = reinterpret_cast<T *>(g_dyn_smem_mb) + (size_t)wp * RingB<T, VEC>::per_warp(D);
        yb = ring + (D + 1) * RingB<T, VEC>::NF * NB;
        wb = yb + NB;
    } else {
        __shared__ __align__(16) T sy[kWarps][NB];
        __shared__ __align__(16) T sw[kWarps][NB];
        __shared__ __align__(16) T sa[kWarps][NB];
        yb = sy[wp];
        wb = sw[wp];
        ab = sa[wp];
    }
    for (unsigned c = next_task(&m.msc->task_ctr[1], lane); c < m.total_tasks;
         c = next_task(&m.msc->task_ctr[1], lane)) {
        const unsigned t = m.total_tasks - 1u - c;    // reverse of phase A's order (L2 reuse)
        const int g = group_of(m.task_off, m.ngroups, t);
        const PcgDesc<T> &d = m.groups[g];
        int done = 0, k = 0;
        double alpha = 0.0;
        if (lane == 0) {
            done = d.sc->done;
            k = d.sc->iter;
            alpha = d.sc->alpha;
        }
        done = __shfl_sync(0xffffffffu, done, 0);
        k = __shfl_sync(0xffffffffu, k, 0);
        alpha = __shfl_sync(0xffffffffu, alpha, 0);
        double val[2] = {0.0, 0.0};
        if (!done) {
            const Task tk = task_of_rows<W>(t - m.task_off[g], d.K, d.tiles_x, d.nz, d.ty > 0 ? d.ty : TY);
            if constexpr (D > 0) {
                // FP64: interior tiles take the body without the periodic-wrap tests
                if constexpr (sizeof(T) == 8) {
                    if (tk.i0 >= 2 && tk.i0 + W + 2 <= d.nth)
                        run_task_b_staged<T, VEC, TY, false, D, false>(d, tk, k, (T)alpha, ring, yb, wb,
                                                                       lane, val);
                    else
                        run_task_b_staged<T, VEC, TY, false, D, true>(d, tk, k, (T)alpha, ring, yb, wb,
                                                                      lane, val);
                } else {
                    run_task_b_staged<T, VEC, TY, false, D, true>(d, tk, k, (T)alpha, ring, yb, wb, lane,
                                                                  val);
                }
            } else
                run_task_b<T, VEC, false>(d, tk, k, (T)alpha, yb, wb, ab, lane, val);
        }
        publish_task<2>(val, m.partials, t, lane);
        double tot[2];
        if (group_complete<2>(m, g, t, lane, tot) && lane == 0 && !done)   // active all launch
            finish_b<false>(d.sc, tot[0], tot[1], k, d.eps, d.max_iter, d.guard_limit);
    }
    if (!last_block(&m.msc->ticket[kTicketB])) return;
    // every group has been completed (and updated) by now
    int active = 0;
    for (int g = threadIdx.x; g < m.ngroups; g += blockDim.x) active |= !m.groups[g].sc->done;
    const int any = __syncthreads_or(active);
    if (threadIdx.x == 0) {
        m.msc->done = !any;                   // no group active any more
        m.msc->ticket[kTicketB] = 0u;
        m.msc->task_ctr[1] = 0u;
    }
}

}  // namespace gmaf
