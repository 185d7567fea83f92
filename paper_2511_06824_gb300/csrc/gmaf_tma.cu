// Phase B of the joint PCG as a block-marched strip with TMA tiles (FP32 inner
// solve of the mixed-precision mode).  A translation unit of its own (its kernels
// live in their own module), using the reductions, scalar update and mbarrier
// helpers of gmaf_pcg_kernels.cuh; the PCG driver (gmaf_pcg.cu) reaches it
// through gmaf_tma.h.
//
//   r -= alpha v;  y = omega D^-1 r;  w = y + omega D^-1 L y  (Eq. 3.5);
//   z = w + omega D^-1 L^T w  (Eq. 3.6, without its constant factor c1);
//   partial sums r.z and r.r  (Table 1, steps 5-8)
//
// The stored diagonal is omega/D for ASSOR-II and 1/D for Jacobi (then z = y).
// L is the strictly lower triangle in the joint index order (theta fastest):
// the lower neighbours of (i, j) are S, W for i > 0 and, across the periodic
// wrap, E when i = n_theta - 1; the upper ones mirror them.
//
// A task is one condition x one strip of 128 columns x TB rows (TB = d.ty_b).
// One block marches it in chunks of CR = 8 RPW staged rows; staged row
// s = 0 .. rows + 1 is grid row j0 - 1 + s (the task's rows and one halo row on
// each side).  The block has eight consumer warps, warp w owning staged rows
// CR k + RPW w .. + RPW - 1 of chunk k (lane l: columns i0 + 4 l .. + 3), and one
// producer warp.
//
// Loads.  The producer's lane 0 claims tasks and, for each chunk, issues one
// cp.async.bulk.tensor copy per input field (r, v, omega/D, aE, aN) of the 136 x
// CR box of columns i0 - 4 .. i0 + 131, completing on the chunk slot's "full"
// mbarrier.  Columns and rows outside the arrays come back as zeros, so y, w and
// their couplings vanish beyond n_z without tests; the two strips at the
// periodic seam take the four wrapped columns from a second, 4 x CR box.  The
// ring holds NS chunk slots; the consumers release a slot on its "empty" barrier
// once the passes that read it are done, so NS - 1 chunks are in flight while
// one is processed, across task boundaries.
//
// Passes over a chunk (block barriers among the consumer warps between them):
//   Y: r1 = r - alpha v, y = r1 omega/D; stores aN(j) y(j) for the row above and
//      the y of the four halo columns;
//   W: w(j) = y + omega/D [aN(j-1) y(j-1) + aW y_W (+ the wrap term)] for the
//      rows and the two halo columns the second pass needs;
//   Z: z of the warp's rows of the previous chunk, from the values it kept in
//      registers and w of the row above.
// The r and z rows are written from registers with 16-byte stores.
//
// Dot products: each lane adds its row sums (exact two-float form); the task's
// sums are reduced over the lanes and then the warps in a fixed order and handed
// to the producer warp, which publishes them per task, off the consumers' path;
// the launch's last block adds the task sums in task order (two levels from 4096
// tasks), so the totals do not depend on scheduling.
//
// Needs n_theta % 128 == 0 (whole strips, 16-byte aligned boxes) and 16-byte
// aligned fields.  Every mbarrier wait is bounded; a block whose wait gives up
// records GMAF_TIMEOUT, waits (bounded) for the copies it has in flight, and
// publishes zero sums for every task it claimed or still claims, so the launch's
// reductions complete and leave their counters at zero.
#include <cuda.h>

#include <atomic>
#include <cstring>

#include "gmaf_internal.cuh"
#include "gmaf_pcg_kernels.cuh"
#include "gmaf_tma.h"

namespace gmaf {

__device__ __forceinline__ void tma_load_3d(void *dst, const void *tmap, int x, int y, int z,
                                            unsigned long long *bar)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4}], [%5];\n" ::"r"(smem_u32(dst)),
        "l"(tmap), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void tmap_prefetch(const void *tmap)
{
    asm volatile("prefetch.tensormap [%0];\n" ::"l"(tmap) : "memory");
}

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;\n" : "=l"(t));
    return t;
}
// Bounded wait for the phase of `parity`, sleeping NS_SLEEP nanoseconds between
// polls so that a waiting lane takes few issue slots from the working warps:
// false after about two seconds (or 2^22 polls), or as soon as *stop is set,
// true once the phase completed.
template <unsigned NS_SLEEP>
__device__ __forceinline__ bool mbar_wait_nap(unsigned long long *bar, unsigned parity,
                                              const int *stop = nullptr)
{
    if (mbar_test(bar, parity)) return true;
    const unsigned long long t0 = global_ns();
    for (unsigned k = 0; k < kBarSpin; ++k) {
        __nanosleep(NS_SLEEP);
        if (mbar_test(bar, parity)) return true;
        if (stop && *(const volatile int *)stop) return false;
        if (global_ns() - t0 > 2000000000ull) return false;
    }
    return false;
}

__device__ __forceinline__ float4 lds4(const float *p) { return *reinterpret_cast<const float4 *>(p); }
__device__ __forceinline__ void sts4(float *p, const float (&v)[4])
{
    *reinterpret_cast<float4 *>(p) = make_float4(v[0], v[1], v[2], v[3]);
}
__device__ __forceinline__ void stg4(float *p, const float (&v)[4])
{
    *reinterpret_cast<float4 *>(p) = make_float4(v[0], v[1], v[2], v[3]);
}

// Named barrier 1 among the consumer warps (the producer warp never joins it).
__device__ __forceinline__ void consumers_sync()
{
    asm volatile("bar.sync 1, %0;\n" ::"n"(kTmaConsumers) : "memory");
}
// The same, returning whether p held in every consumer thread.
__device__ __forceinline__ bool consumers_sync_and(bool p)
{
    unsigned r;
    asm volatile(
        "{\n\t.reg .pred a, b;\n\tsetp.ne.u32 a, %1, 0;\n\t"
        "bar.red.and.pred b, 1, %2, a;\n\tselp.u32 %0, 1, 0, b;\n\t}\n"
        : "=r"(r)
        : "r"((unsigned)p), "n"(kTmaConsumers)
        : "memory");
    return r != 0;
}

// Task t of the TMA phase B: condition fastest, then strip, then row block (the
// numbering of task_of_rows, in 32-bit arithmetic).
__device__ __forceinline__ Task tma_task(unsigned t, int K, int tiles_x, int nz, int ty)
{
    Task r;
    const unsigned sp = t / (unsigned)K;
    r.cond = (int)(t - sp * (unsigned)K);
    const unsigned tyi = sp / (unsigned)tiles_x;
    r.i0 = (int)(sp - tyi * (unsigned)tiles_x) * kTmaW;
    r.j0 = (int)tyi * ty;
    r.jend = min(r.j0 + ty, nz);
    return r;
}

// Finished tasks' sums, handed by the consumers to the producer warp, which
// publishes them (fence, chunk counter) off the consumers' path.
struct TmaMail {
    int t[kTmaMail];
    double v[kTmaMail][2];
    unsigned tail, head;             // pushed by consumer thread 0, published by the producer
};

// Publish every task in the mailbox not yet published (producer warp); returns the
// new count.
__device__ __forceinline__ unsigned tma_publish_mail(TmaMail &mb, unsigned pubd, const PcgReduce &rd,
                                                     unsigned ntasks, int lane)
{
    unsigned tail = 0;
    if (lane == 0) tail = *(volatile unsigned *)&mb.tail;
    tail = __shfl_sync(0xffffffffu, tail, 0);
    __threadfence_block();
    for (; pubd < tail; ++pubd) {
        const int e = (int)(pubd % kTmaMail);
        const double val[2] = {lane == 0 ? mb.v[e][0] : 0.0, lane == 0 ? mb.v[e][1] : 0.0};
        publish_unit<2>(val, rd, ntasks, (unsigned)mb.t[e], lane);
    }
    __syncwarp();
    if (lane == 0) *(volatile unsigned *)&mb.head = pubd;
    return pubd;
}

// The producer's state (lane 0 of the producer warp): claims tasks and fills ring
// slots.  Chunk number g goes to slot g % NS; the slot's task and chunk index are
// written before its "full" barrier is armed, so a consumer whose wait completes
// reads them.  When no task is left the next slot gets an end marker (task -1)
// and a plain arrive, which completes its phase with nothing to copy.
template <bool INIT, int NS, int CR>
struct TmaIssuer {
    using C = TmaChunk<CR>;
    unsigned t = 0;                  // task being issued
    int kc = 0, nch = 0;             // its next chunk, its chunks
    int i0 = 0, j0 = 0, zc = 0, zs = 0;
    bool ew = false, ee = false;     // the strip touches column 0 / column n_theta - 1
    unsigned issued = 0;             // chunks issued, the end marker included
    unsigned claimed = 0;            // tasks claimed

    // Issue chunk number `issued`; false once the end marker has been issued.
    __device__ __forceinline__ bool issue(const PcgDesc<float> &d, const TmaParams &tp, int rsel,
                                          unsigned ntasks, float *ring, unsigned long long *full,
                                          int *s_task, int *s_chunk, int *s_cl, const int *s_cslot)
    {
        const int slot = (int)(issued % NS);
        if (kc == nch) {
            const unsigned c = atomicAdd(&d.sc->task_ctr[1], 1u);
            if (c >= ntasks) {
                s_task[slot] = -1;
                s_chunk[slot] = 0;
                mbar_arrive(&full[slot]);
                ++issued;
                return false;
            }
            t = ntasks - 1u - c;         // the reverse of phase A's order (L2 reuse)
            const Task tk = tma_task(t, d.K, d.tiles_x, d.nz, d.ty_b);
            i0 = tk.i0;
            j0 = tk.j0;
            nch = (tk.jend - tk.j0 + 2 + CR - 1) / CR;
            kc = 0;
            zc = tk.cond;
            zs = s_cslot[tk.cond];
            ew = i0 == 0;
            ee = i0 + kTmaW == d.nth;
            s_cl[claimed % kTmaMaxClaims] = (int)t;
            ++claimed;
        }
        s_task[slot] = (int)t;
        s_chunk[slot] = kc;
        float *dst = ring + (size_t)slot * 5 * C::kField;
        unsigned long long *b = &full[slot];
        const int y = j0 - 1 + CR * kc;
        const unsigned field_bytes =
            (unsigned)(CR * (kTmaRow + 4 * ((ew ? 1 : 0) + (ee ? 1 : 0))) * sizeof(float));
        fence_proxy_async_smem();        // the slot's last generic reads precede the copies
        mbar_arrive_tx(b, (INIT ? 4u : 5u) * field_bytes);
#pragma unroll
        for (int f = 0; f < 5; ++f) {
            if (INIT && f == 1) continue;
            const int m = f == 0 ? rsel : f == 1 ? kTmV : f == 2 ? kTmOd : f == 3 ? kTmAE : kTmAN;
            const int z = f < 2 ? zc : zs;
            float *fd = dst + f * C::kField;
            // columns i0 - 4 .. i0 + 131; outside 0 .. n_theta - 1 they come back as
            // zeros and the seam strips take the wrapped four columns from a second box
            tma_load_3d(fd, &tp.m[m], i0 - 4, y, z, b);
            if (ew) tma_load_3d(fd + C::kWrapW, &tp.m[m + 1], d.nth - 4, y, z, b);
            if (ee) tma_load_3d(fd + C::kWrapE, &tp.m[m + 1], 0, y, z, b);
        }
        ++kc;
        ++issued;
        return true;
    }
};

// A consumer warp's row kept from one chunk to the next for pass Z: r1, omega/D,
// aE, aN, w (y with Jacobi) and, in lane 0, aE of column i0 - 1.
struct TmaKept {
    float r[4], od[4], e[4], n[4], w[4], awrap;
};

template <bool INIT, int NS, int RPW>
__global__ void __maxnreg__(RPW == 1 ? 96 : 168) k_phase_b_tma(const PcgDesc<float> *__restrict__ dp,
                                                               const __grid_constant__ TmaParams tp)
{
    constexpr int CR = kTmaWarps * RPW;              // staged rows per chunk
    using C = TmaChunk<CR>;
    constexpr int RING = C::kRing;
    const PcgDesc<float> &d = *dp;
    Scalars *sc = d.sc;
    extern __shared__ __align__(128) unsigned char g_dyn_smem_tb[];
    __shared__ __align__(8) unsigned long long s_full[NS], s_empty[NS];
    __shared__ int s_task[NS], s_chunk[NS], s_cl[kTmaMaxClaims], s_cslot[kMaxCond];
    __shared__ double s_red[kTmaWarps][2];
    __shared__ TmaMail s_mb;
    __shared__ int s_done, s_k, s_abort;
    __shared__ unsigned s_consumed, s_issued, s_claimed;
    __shared__ double s_alpha;
    if (threadIdx.x == 0) {
        s_done = sc->done;
        s_k = sc->iter;
        s_alpha = sc->alpha;
        s_abort = 0;
        s_consumed = s_issued = s_claimed = 0u;
        s_mb.tail = s_mb.head = 0u;
        if (!s_done) {
            for (int q = 0; q < NS; ++q) {
                mbar_init(&s_full[q], 1);
                mbar_init(&s_empty[q], 1);
            }
            mbar_init_fence();
        }
    }
    __syncthreads();
    if (s_done) return;
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
    float *ring = reinterpret_cast<float *>(g_dyn_smem_tb);
    const int k = s_k;
    const unsigned ntasks = (unsigned)d.ntiles_b;
    const PcgReduce rd = reducer_of(d);
    unsigned pubd = 0;                   // producer warp: tasks published

    if (wp == kTmaWarps) {
        // ---------------- producer warp: lane 0 claims tasks and issues the copies;
        // the warp publishes the finished tasks' sums between the copies
        for (int q = lane; q < d.K; q += 32) s_cslot[q] = d.cslot[q];
        __syncwarp();
        if (lane == 0)
            for (int m = 0; m < kTmaMaps; ++m) tmap_prefetch(&tp.m[m]);
        const int rsel = (k & 1) ? kTmR1 : kTmR0;
        TmaIssuer<INIT, NS, CR> is;
        for (unsigned g = 0;; ++g) {
            int go = 1;
            if (lane == 0) {
                const int slot = (int)(g % NS);
                // the consumers release a slot once its chunk has been read
                if (g >= NS && !mbar_wait_nap<256>(&s_empty[slot], ((g / NS) - 1u) & 1u, &s_abort)) go = 0;
                if (go && *(volatile int *)&s_abort) go = 0;
                if (!go) {
                    if (atomicExch(&s_abort, 1) == 0) {
                        sc->status = GMAF_TIMEOUT;
                        __threadfence();
                    }
                } else if (!is.issue(d, tp, rsel, ntasks, ring, s_full, s_task, s_chunk, s_cl, s_cslot)) {
                    go = 2;
                }
            }
            go = __shfl_sync(0xffffffffu, go, 0);
            pubd = tma_publish_mail(s_mb, pubd, rd, ntasks, lane);
            if (go != 1) break;
        }
        if (lane == 0) {
            s_issued = is.issued;
            s_claimed = is.claimed;
        }
    } else {
        // ---------------- consumer warps
        float *ysr = ring + NS * 5 * C::kField;          // [RING][128] aN(j) y(j), own columns
        float *wr = ysr + RING * kTmaW;                  // [RING][128] w(j)
        float *ysh = wr + RING * kTmaW;                  // [RING][2]   aN y at i0 - 1, i0 + 128
        float *yh = ysh + RING * 2;                      // [RING][4]   y at i0 - 2, i0 - 1, i0 + 128, i0 + 129
        float *wh = yh + RING * 4;                       // [RING][2]   w at i0 - 1, i0 + 128
        const float alpha = (float)s_alpha;
        const bool assor = d.precond == 1;
        const int nth = d.nth, K = d.K, tiles_x = d.tiles_x, nz = d.nz, tyb = d.ty_b;
        const size_t n = (size_t)d.n;
        float *const rnext = d.r[(k + 1) & 1];
        float *const zout = d.z;

        // the task being processed
        int i0 = 0, j0 = 0, rows = 0, nch = 0;
        bool ew = false, ee = false;         // the strip touches column 0 / column n_theta - 1
        size_t base = 0;                     // cond * n + i0 + 4 lane
        bool at_w = false, at_e = false;     // the lane holds column 0 / column n_theta - 1
        RowAcc<float> arz, arr;
        bool lost = false;                   // thread 0: a task's sums could not be handed over
        TmaKept kept[RPW];
#pragma unroll
        for (int i = 0; i < RPW; ++i) {
#pragma unroll
            for (int q = 0; q < 4; ++q) kept[i].r[q] = kept[i].od[q] = kept[i].e[q] = kept[i].n[q] = kept[i].w[q] = 0.0f;
            kept[i].awrap = 0.0f;
        }

        // z of staged row sz from its kept values and w of the row above
        auto pass_z = [&](const TmaKept &kp, int sz) {
            if (sz < 1 || sz > rows) return;
            float z[4];
            if (assor) {
                const int rz = sz & (RING - 1), rn = (sz + 1) & (RING - 1);
                const float4 wn4 = lds4(wr + rn * kTmaW + 4 * lane);
                const float wn[4] = {wn4.x, wn4.y, wn4.z, wn4.w};
                float wE = __shfl_down_sync(0xffffffffu, kp.w[0], 1);
                if (lane == 31) wE = wh[rz * 2 + 1];
                const float wW = wh[rz * 2 + 0];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    float sum = kp.n[q] * wn[q];
                    const float we = q < 3 ? kp.w[q + 1] : wE;
                    if (q < 3 || !at_e) sum += kp.e[q] * we;
                    if (q == 0 && at_w) sum += kp.awrap * wW;
                    z[q] = kp.w[q] + kp.od[q] * sum;    // Eq. 3.6 without its factor c1
                }
            } else {
#pragma unroll
                for (int q = 0; q < 4; ++q) z[q] = kp.w[q];
            }
            float rzs = 0.0f, rrs = 0.0f;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                rzs += kp.r[q] * z[q];
                rrs += kp.r[q] * kp.r[q];
            }
            arz.add_row(rzs);
            arr.add_row(rrs);
            stg4(zout + base + (size_t)(j0 - 1 + sz) * nth, z);
        };

        for (unsigned g = 0;; ++g) {
            const int slot = (int)(g % NS);
            const unsigned par = (g / NS) & 1u;
            // lane 0 waits for the chunk (bounded); then every lane observes the
            // completed phase itself, which orders its reads after the copies
            int ok = 1;
            if (lane == 0) ok = mbar_wait_nap<32>(&s_full[slot], par) ? 1 : 0;
            ok = __shfl_sync(0xffffffffu, ok, 0);
            if (ok) mbar_test(&s_full[slot], par);
            const int t = s_task[slot], kc = s_chunk[slot];
            if (t >= 0 && kc == 0) {
                const Task tk = tma_task((unsigned)t, K, tiles_x, nz, tyb);
                i0 = tk.i0;
                j0 = tk.j0;
                rows = tk.jend - tk.j0;
                nch = (rows + 2 + CR - 1) / CR;
                base = (size_t)tk.cond * n + (size_t)(i0 + 4 * lane);
                at_w = i0 + 4 * lane == 0;
                at_e = i0 + 4 * lane + 4 == nth;
                ew = i0 == 0;
                ee = i0 + kTmaW == nth;
                arz = RowAcc<float>{};
                arr = RowAcc<float>{};
            }
            const float *Fr = ring + (size_t)slot * 5 * C::kField;
            const float *Fv = Fr + C::kField, *Fo = Fr + 2 * C::kField;
            const float *Fe = Fr + 3 * C::kField, *Fn = Fr + 4 * C::kField;

            // ---- pass Y: r1 = r - alpha v, y = omega/D r1 (shared-memory writes only
            // until every consumer's wait is known to have completed)
            float r1[RPW][4], y[RPW][4], od[RPW][4], an[RPW][4];
#pragma unroll
            for (int i = 0; i < RPW; ++i) {
                const int rr = RPW * wp + i;                 // the row in the chunk
                const int s = CR * kc + rr;                  // its staged row
                const int rs = s & (RING - 1);
                if (t >= 0 && s < rows + 2) {
                    const int co = rr * kTmaRow + 4 + 4 * lane;
                    const int offw = ew ? C::kWrapW + rr * 4 : rr * kTmaRow;
                    const int offe = ee ? C::kWrapE + rr * 4 : rr * kTmaRow + kTmaW + 4;
                    const float4 r4 = lds4(Fr + co);
                    const float4 v4 = INIT ? make_float4(0.f, 0.f, 0.f, 0.f) : lds4(Fv + co);
                    const float4 o4 = lds4(Fo + co);
                    const float4 n4 = lds4(Fn + co);
                    const float rv[4] = {r4.x, r4.y, r4.z, r4.w}, vv[4] = {v4.x, v4.y, v4.z, v4.w};
                    const float ov[4] = {o4.x, o4.y, o4.z, o4.w}, nv[4] = {n4.x, n4.y, n4.z, n4.w};
                    float ys[4];
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        r1[i][q] = INIT ? rv[q] : rv[q] - alpha * vv[q];
                        y[i][q] = r1[i][q] * ov[q];
                        od[i][q] = ov[q];
                        an[i][q] = nv[q];
                        ys[q] = nv[q] * y[i][q];
                    }
                    sts4(ysr + rs * kTmaW + 4 * lane, ys);
                    // halo columns: lane & 3 -> i0 - 2, i0 - 1, i0 + 128, i0 + 129
                    const int h = lane & 3;
                    const int ho = h < 2 ? offw + 2 + h : offe + (h - 2);
                    const float hr = INIT ? Fr[ho] : Fr[ho] - alpha * Fv[ho];
                    const float hy = hr * Fo[ho];
                    if (lane < 4) yh[rs * 4 + h] = hy;
                    if (lane == 1 || lane == 2) ysh[rs * 2 + (h - 1)] = Fn[ho] * hy;
                } else {
#pragma unroll
                    for (int q = 0; q < 4; ++q) r1[i][q] = y[i][q] = od[i][q] = an[i][q] = 0.0f;
                }
            }
            if (!consumers_sync_and(ok != 0 && !lost)) {
                // a wait gave up: the producer warp drains and publishes after the loop
                if (threadIdx.x == 0) {
                    s_consumed = g;
                    if (atomicExch(&s_abort, 1) == 0) {
                        sc->status = GMAF_TIMEOUT;
                        __threadfence();
                    }
                }
                break;
            }
            if (t < 0) break;
#pragma unroll
            for (int i = 0; i < RPW; ++i) {
                const int s = CR * kc + RPW * wp + i;
                if (!INIT && s >= 1 && s <= rows) stg4(rnext + base + (size_t)(j0 - 1 + s) * nth, r1[i]);
            }

            // ---- pass W: first ASSOR pass (Eq. 3.5) for the rows and two halo columns
            float w[RPW][4], ev[RPW][4], awrap[RPW];
#pragma unroll
            for (int i = 0; i < RPW; ++i) {
                const int rr = RPW * wp + i;
                const int s = CR * kc + rr;
                const int rs = s & (RING - 1), rsm = (s - 1) & (RING - 1);
#pragma unroll
                for (int q = 0; q < 4; ++q) w[i][q] = ev[i][q] = 0.0f;
                awrap[i] = 0.0f;
                if (s < rows + 2 && s >= 1 && assor) {
                    const int co = rr * kTmaRow + 4 + 4 * lane;
                    const int offw = ew ? C::kWrapW + rr * 4 : rr * kTmaRow;
                    const int offe = ee ? C::kWrapE + rr * 4 : rr * kTmaRow + kTmaW + 4;
                    const float4 e4 = lds4(Fe + co);
                    const float4 s4 = lds4(ysr + rsm * kTmaW + 4 * lane);
                    ev[i][0] = e4.x;
                    ev[i][1] = e4.y;
                    ev[i][2] = e4.z;
                    ev[i][3] = e4.w;
                    const float ss[4] = {s4.x, s4.y, s4.z, s4.w};
                    float yW = __shfl_up_sync(0xffffffffu, y[i][3], 1);
                    float aW = __shfl_up_sync(0xffffffffu, ev[i][3], 1);
                    float yE = __shfl_down_sync(0xffffffffu, y[i][0], 1);
                    if (lane == 0) {
                        yW = yh[rs * 4 + 1];
                        aW = Fe[offw + 3];
                    }
                    if (lane == 31) yE = yh[rs * 4 + 2];
                    awrap[i] = aW;
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        float sum = ss[q];                           // aN(j - 1) y(j - 1)
                        const float aw = q > 0 ? ev[i][q - 1] : aW;
                        const float yw = q > 0 ? y[i][q - 1] : yW;
                        if (q > 0 || !at_w) sum += aw * yw;
                        if (q == 3 && at_e) sum += ev[i][3] * yE;    // E across the wrap is lower
                        w[i][q] = y[i][q] + od[i][q] * sum;
                    }
                    sts4(wr + rs * kTmaW + 4 * lane, w[i]);
                    // halo w: lane 0 -> column i0 - 1, lane 31 -> column i0 + 128
                    if (lane == 0 || lane == 31) {
                        const bool west = lane == 0;
                        const int gc = west ? wrap_col(i0 - 1, nth) : wrap_col(i0 + kTmaW, nth);
                        const float yc = yh[rs * 4 + (west ? 1 : 2)];
                        const float odc = Fo[west ? offw + 3 : offe];
                        float sum = ysh[rsm * 2 + (west ? 0 : 1)];
                        const float awc = west ? Fe[offw + 2] : ev[i][3];
                        const float ywc = west ? yh[rs * 4 + 0] : y[i][3];
                        if (gc > 0) sum += awc * ywc;
                        if (gc == nth - 1)
                            sum += (west ? Fe[offw + 3] : Fe[offe]) * (west ? y[i][0] : yh[rs * 4 + 3]);
                        wh[rs * 2 + (west ? 0 : 1)] = yc + odc * sum;
                    }
                }
            }
            consumers_sync();
            // every consumer has read the slot: the producer may refill it
            if (threadIdx.x == 0) mbar_arrive(&s_empty[slot]);

            // ---- pass Z: second ASSOR pass (Eq. 3.6) of the warp's previous rows
#pragma unroll
            for (int i = 0; i < RPW; ++i) {
                const int s = CR * kc + RPW * wp + i;
                if (kc >= 1) pass_z(kept[i], s - CR);
                if (s < rows + 2) {
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        kept[i].r[q] = r1[i][q];
                        kept[i].od[q] = od[i][q];
                        kept[i].e[q] = ev[i][q];
                        kept[i].n[q] = an[i][q];
                        kept[i].w[q] = assor ? w[i][q] : y[i][q];
                    }
                    kept[i].awrap = awrap[i];
                }
            }
            if (kc == nch - 1) {
                // the task's last chunk: its own rows' z, then the task's sums to the
                // producer warp's mailbox (warps added in order)
#pragma unroll
                for (int i = 0; i < RPW; ++i) pass_z(kept[i], CR * kc + RPW * wp + i);
                const double a = warp_sum_d(arz.value()), b = warp_sum_d(arr.value());
                if (lane == 0) {
                    s_red[wp][0] = a;
                    s_red[wp][1] = b;
                }
                consumers_sync();
                if (threadIdx.x == 0) {
                    double sa = 0.0, sb = 0.0;
                    for (int w2 = 0; w2 < kTmaWarps; ++w2) {
                        sa += s_red[w2][0];
                        sb += s_red[w2][1];
                    }
                    const unsigned tail = s_mb.tail;
                    // a free entry: at most NS + 1 tasks wait in the mailbox (the producer
                    // publishes after every copy it issues and the consumers cannot run
                    // more than NS chunks ahead of it), so one is free unless the producer
                    // stopped; the wait is bounded all the same
                    unsigned spin = 0;
                    while (tail - *(volatile unsigned *)&s_mb.head >= (unsigned)kTmaMail && spin < kBarSpin) {
                        __nanosleep(64);
                        ++spin;
                    }
                    if (spin < kBarSpin) {
                        const int e = (int)(tail % kTmaMail);
                        s_mb.t[e] = t;
                        s_mb.v[e][0] = sa;
                        s_mb.v[e][1] = sb;
                        __threadfence_block();
                        *(volatile unsigned *)&s_mb.tail = tail + 1u;
                    } else {
                        // not handed over: the consumers stop at the next chunk, before
                        // any later task, so the cleanup below finds this one among the
                        // claimed tasks not published and publishes zero sums for it
                        lost = true;
                        if (atomicExch(&s_abort, 1) == 0) {
                            sc->status = GMAF_TIMEOUT;
                            __threadfence();
                        }
                    }
                }
            }
        }
    }
    __syncthreads();
    if (wp == kTmaWarps) {
        // the sums still in the mailbox
        pubd = tma_publish_mail(s_mb, pubd, rd, ntasks, lane);
        if (s_abort) {
            // a wait gave up: wait (bounded) for the copies still in flight, then
            // publish zero sums for every task claimed and not finished and for every
            // task still unclaimed, so the launch's reductions complete and rearm
            if (lane == 0)
                for (unsigned q = s_consumed; q < s_issued; ++q) mbar_wait_nap<256>(&s_full[q % NS], (q / NS) & 1u);
            __syncwarp();
            const double zero[2] = {0.0, 0.0};
            for (unsigned p = pubd; p < s_claimed; ++p)
                publish_unit<2>(zero, rd, ntasks, (unsigned)s_cl[p % kTmaMaxClaims], lane);
            for (unsigned c = next_task(&sc->task_ctr[1], lane); c < ntasks; c = next_task(&sc->task_ctr[1], lane))
                publish_unit<2>(zero, rd, ntasks, ntasks - 1u - c, lane);
        }
    }
    double tot[2];
    if (reduce_units<2>(rd, ntasks, &sc->ticket[kTicketB], &sc->task_ctr[1], tot) && threadIdx.x == 0) {
        int done = finish_b<INIT>(sc, tot[0], tot[1], k, d.eps, d.max_iter, d.guard_limit);
        if (sc->status == GMAF_TIMEOUT) {
            sc->done = 1;
            done = 1;
        }
        if (d.use_cond) cudaGraphSetConditional(d.cond, done ? 0u : 1u);
    }
}


// ------------------------------------------------------------------ host side

TmaKernels tma_kernels(int ns, int rpw)
{
    TmaKernels k{nullptr, nullptr, 0};
    if (ns == 4 && rpw == 1) {
        k = {(const void *)k_phase_b_tma<false, 4, 1>, (const void *)k_phase_b_tma<true, 4, 1>, 0};
    } else if (ns == 3 && rpw == 2) {
        k = {(const void *)k_phase_b_tma<false, 3, 2>, (const void *)k_phase_b_tma<true, 3, 2>, 0};
    } else if (ns == 4 && rpw == 2) {
        k = {(const void *)k_phase_b_tma<false, 4, 2>, (const void *)k_phase_b_tma<true, 4, 2>, 0};
    } else {
        return k;
    }
    k.smem = (size_t)tma_b_smem_floats(ns, rpw) * sizeof(float);
    // one opt-in mask per kernel (index: the pair above, then the initial pass)
    static std::atomic<unsigned long long> done[6];
    const int idx = ns == 4 && rpw == 1 ? 0 : ns == 3 ? 1 : 2;
    smem_optin(done[2 * idx], k.b, k.smem, true);
    smem_optin(done[2 * idx + 1], k.b_init, k.smem, true);
    return k;
}

using EncodeTiledFn = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                   const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                   const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                   CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// The driver's tensor-map encoder, looked up once through the runtime (no link
// against the driver library); null if it is not available.
static EncodeTiledFn encode_tiled()
{
    static const EncodeTiledFn fn = []() -> EncodeTiledFn {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q{};
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        return reinterpret_cast<EncodeTiledFn>(p);
    }();
    return fn;
}

static_assert(sizeof(TmaMapBytes) == sizeof(CUtensorMap), "tensor map size");

// The row box (136 x rows) and the wrap box (4 x rows) of r[0], r[1], v
// ([K][n_z][n_theta]) and omega/D, aE, aN ([slots][n_z][n_theta]), FP32, zero fill
// outside the arrays.
bool tma_encode_maps(const PcgDesc<float> &h, TmaParams &tp, int rows)
{
    if (h.nth % kTmaW != 0 || h.nslots < 1) return false;
    const EncodeTiledFn enc = encode_tiled();
    if (!enc) return false;
    const void *base[6] = {h.r[0], h.r[1], h.v, h.invD, h.aE, h.aN};
    for (int f = 0; f < 6; ++f) {
        const cuuint64_t dims[3] = {(cuuint64_t)h.nth, (cuuint64_t)h.nz,
                                    (cuuint64_t)(f < 3 ? h.K : h.nslots)};
        const cuuint64_t strides[2] = {(cuuint64_t)h.nth * sizeof(float),
                                       (cuuint64_t)h.nth * h.nz * sizeof(float)};
        const cuuint32_t estr[3] = {1, 1, 1};
        for (int b = 0; b < 2; ++b) {
            const cuuint32_t box[3] = {b == 0 ? (cuuint32_t)kTmaRow : 4u, (cuuint32_t)rows, 1u};
            CUtensorMap m;
            if (enc(&m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<void *>(base[f]), dims, strides,
                    box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                    CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
                return false;
            std::memcpy(&tp.m[2 * f + b], &m, sizeof(m));
        }
    }
    return true;
}

}  // namespace gmaf
