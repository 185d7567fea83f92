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
#include <algorithm>
#include <cstddef>
#include <cmath>
#include <cstring>
#include <vector>

#include "gmaf_internal.cuh"
#include "gmaf_pcg_kernels.cuh"
#include "gmaf_pcg_host.cuh"
#include "gmaf_mphase_kernels.cuh"
#include "gmaf_tma.h"
#include "gmaf_drec.h"

namespace gmaf {

// ------------------------------------------------------------------ host driver

// Phase B staged through shared memory D rows ahead (cp.async); id + 100000 D.
template <typename T, int VEC, int TY, int MINB, int D>
static KernelSet<T> ks_staged()
{
    const size_t smem = (size_t)kWarps * RingB<T, VEC>::per_warp(D) * sizeof(T);
    const void *b = (const void *)k_phase_b_staged<T, VEC, TY, MINB, false, D>;
    const void *bi = (const void *)k_phase_b_staged<T, VEC, TY, MINB, true, D>;
    static std::atomic<unsigned long long> done_b{0}, done_bi{0};
    smem_optin(done_b, b, smem);
    smem_optin(done_bi, bi, smem);
    return {(const void *)k_phase_a<T, VEC, TY, MINB, 0>, b, bi, 32 * VEC, TY,
            100000 * D + 1000 * VEC + 10 * TY + MINB, smem, 0};
}

// Phase A staged DA rows ahead and phase B DB rows ahead; id + 200000 DA + 100000 DB.
template <typename T, int VEC, int TY, int MINB, int DA, int DB = DA>
static KernelSet<T> ks_staged_ab()
{
    KernelSet<T> ks = ks_staged<T, VEC, TY, MINB, DB>();
    const size_t smem = (size_t)kWarps * RingA<T, VEC, sizeof(T) == 4>::per_warp(DA) * sizeof(T);
    const void *a = (const void *)k_phase_a_staged<T, VEC, TY, MINB, DA>;
    static std::atomic<unsigned long long> done_a{0};
    smem_optin(done_a, a, smem);
    ks.a = a;
    ks.smem_a = smem;
    ks.id += 200000 * DA;
    ks.p_period = sizeof(T) == 4 ? 2 : 1;      // the staged FP32 phase A pairs the p updates
    return ks;
}

// Phase A staged DA rows ahead (cp.async) and phase B filled by one lane's bulk
// copies of whole row segments DB rows ahead (cp.async.bulk + mbarrier);
// id 2000000 + 200000 DA + 100000 DB + 1000 VEC + 10 TY + MINB.
template <typename T, int VEC, int TY, int MINB, int DA, int DB = DA>
static KernelSet<T> ks_bulk_ab()
{
    KernelSet<T> ks = ks_staged_ab<T, VEC, TY, MINB, DA, DB>();
    const size_t smem = (size_t)kWarps * RingB<T, VEC>::per_warp(DB) * sizeof(T);
    const void *b = (const void *)k_phase_b_bulk<T, VEC, TY, MINB, false, DB>;
    const void *bi = (const void *)k_phase_b_bulk<T, VEC, TY, MINB, true, DB>;
    static std::atomic<unsigned long long> done_b{0}, done_bi{0};
    smem_optin(done_b, b, smem);
    smem_optin(done_bi, bi, smem);
    ks.b = b;
    ks.b_init = bi;
    ks.smem_b = smem;
    ks.id += 2000000;
    return ks;
}

// Both phases staged as ks_staged_ab, in blocks of NT threads (MINB blocks per SM);
// id + 100000000 * (NT / 32).
template <typename T, int VEC, int TY, int MINB, int DA, int NT>
static KernelSet<T> ks_staged_ab_nt(int rows = TY)
{
    KernelSet<T> ks{};
    constexpr int warps = NT / 32;
    ks.smem_b = (size_t)warps * RingB<T, VEC>::per_warp(DA) * sizeof(T);
    ks.smem_a = (size_t)warps * RingA<T, VEC, sizeof(T) == 4>::per_warp(DA) * sizeof(T);
    ks.a = (const void *)k_phase_a_staged<T, VEC, TY, MINB, DA, NT>;
    ks.b = (const void *)k_phase_b_staged<T, VEC, TY, MINB, false, DA, NT>;
    ks.b_init = (const void *)k_phase_b_staged<T, VEC, TY, MINB, true, DA, NT>;
    static std::atomic<unsigned long long> done_a{0}, done_b{0}, done_bi{0};
    smem_optin(done_a, ks.a, ks.smem_a);
    smem_optin(done_b, ks.b, ks.smem_b);
    smem_optin(done_bi, ks.b_init, ks.smem_b);
    ks.W = 32 * VEC;
    ks.TY = rows;           // rows per task, taken by the staged kernels from the descriptor
    ks.id = 100000000 * warps + 200000 * DA + 100000 * DA + 1000 * VEC + 10 * rows + MINB;
    ks.sched = 0;
    ks.p_period = sizeof(T) == 4 ? 2 : 1;
    ks.threads = NT;
    return ks;
}

// Phase A staged two rows ahead (as ks_staged_ab, p updates paired) and the
// block-marched TMA phase B with NS chunk slots, RPW rows per consumer warp
// (chunks of 8 RPW rows; RPW 1: two blocks per SM, RPW 2: one) and tasks of
// ty_b rows; id 3000000 + 10000 RPW + 1000 NS + ty_b.
template <int NS, int RPW>
static KernelSet<float> ks_tma(int ty_b)
{
    KernelSet<float> ks = ks_staged_ab<float, 4, 32, 2, 2>();
    const TmaKernels tk = tma_kernels(NS, RPW);
    ks.b = tk.b;
    ks.b_init = tk.b_init;
    ks.smem_b = tk.smem;
    ks.tma = RPW;
    ks.ty_b = ty_b;
    ks.threads_b = kTmaThreads;
    ks.id = 3000000 + 10000 * RPW + 1000 * NS + ty_b;
    return ks;
}

// ks_staged_ab<float, 4, 32, 2, 2> with phase A rebuilding the diagonal from the
// couplings (gmaf_drec.cu); id + 10000000.
static KernelSet<float> ks_drec()
{
    KernelSet<float> ks = ks_staged_ab<float, 4, 32, 2, 2>();
    const DrecKernel dk = drec_phase_a();
    ks.a = dk.a;
    ks.smem_a = dk.smem;
    ks.id += 10000000;
    return ks;
}

constexpr int kMaxVariants = 28;

// Candidate variants; the vector ones need n_theta % VEC == 0 and aligned fields.
static int variants(KernelSet<float> *out, bool vec_ok, bool vec8_ok = false, bool bulk_ok = false,
                    bool tma_ok = false, bool drec_ok = false)
{
    int n = 0;
    if (vec_ok) {
        // 32-row tasks suit the largest grids; 16 and 8 rows and the static
        // schedule keep every warp busy on smaller ones (1024 x 512 x 9 has only
        // 1152 tasks of 32 rows for 2432 resident warps)
        out[n++] = ks_staged_ab<float, 4, 32, 2, 2>();
        if (drec_ok) out[n++] = ks_drec();
        // 3 blocks of 6 warps per SM (18 warps, 94 registers); the task height is a
        // run-time choice: with equal tasks the phase lasts whole waves of tasks, and
        // on 2048 x 1024 x 9 18-row tasks fill exactly 3 waves of the 2736 warps
        for (int rows : {32, 24, 20, 18, 16}) out[n++] = ks_staged_ab_nt<float, 4, 32, 3, 2, 192>(rows);
        if (bulk_ok) out[n++] = ks_bulk_ab<float, 4, 32, 2, 2>();
        out[n++] = ks_staged_ab<float, 4, 16, 2, 2>();
        out[n++] = ks_of<float, 4, 32, 2>(0);
        out[n++] = ks_staged<float, 4, 32, 2, 2>();
        out[n++] = ks_staged<float, 4, 16, 2, 2>();
        out[n++] = ks_of<float, 4, 16, 2>(0);
        out[n++] = ks_of<float, 4, 8, 2>(0);
        out[n++] = ks_of<float, 2, 32, 4>(2);
        out[n++] = ks_of<float, 4, 32, 2, 1>(0);
    }
    if (vec8_ok) out[n++] = ks_staged<float, 8, 32, 2, 1>();
    out[n++] = ks_of<float, 1, 32, 4>(4);
    out[n++] = ks_of<float, 1, 16, 4>(5);
    out[n++] = ks_of<float, 1, 32, 4, 1>(0);
    if (tma_ok) {
        // block-marched TMA phase B; tasks of CR m - 2 rows fill whole chunks
        out[n++] = ks_tma<4, 1>(62);
        out[n++] = ks_tma<3, 2>(62);
        out[n++] = ks_tma<4, 2>(62);
        out[n++] = ks_tma<3, 2>(30);
    }
    return n;
}

static int variants(KernelSet<double> *out, bool vec_ok, bool = false, bool = false, bool = false,
                    bool = false)
{
    int n = 0;
    if (vec_ok) {
        out[n++] = ks_of<double, 2, 32, 2>(0);
        out[n++] = ks_staged<double, 2, 32, 2, 2>();
        out[n++] = ks_of<double, 2, 16, 2>(0);
        out[n++] = ks_of<double, 2, 32, 2, 1>(0);
    }
    out[n++] = ks_of<double, 1, 32, 3>(4);
    out[n++] = ks_of<double, 1, 16, 3>(5);
    out[n++] = ks_of<double, 1, 32, 3, 1>(0);
    return n;
}

// VEC = 8 float kernels: two 16-byte chunks per lane, n_theta % 8 == 0.
template <typename T>
static bool vec8_ok(const PcgDesc<T> &h)
{
    return sizeof(T) == 4 && vec_ok(h) && (h.nth % 8) == 0;
}

// Bulk-copied phase B (float, 4 columns a lane): 16-byte row pieces and at most
// one wrap per row segment of 136 columns.
template <typename T>
static bool bulk_ok(const PcgDesc<T> &h)
{
    return sizeof(T) == 4 && vec_ok(h) && h.nth >= 32 * 4 + 8;
}

template <typename T>
struct PcgRun {
    PcgDesc<T> *d_desc;     // device copy of h
    PcgDesc<T> h;
    KernelSet<T> ks;
    int grid_a, grid_b, grid_s;
    TmaParams tma[2];       // tensor maps of the TMA phase B (FP32), chunks of 8 and 16 rows
    bool tma_ready;         //   encoded for this run's arrays
    bool drec_ready;        // h.dbnd holds the boundary term of the rebuilt diagonal (FP32)
};

// The tensor maps a kernel set's TMA phase B takes (chunks of 8 ks.tma rows).
template <typename T>
static const TmaParams *tma_params(const PcgRun<T> &run)
{
    return &run.tma[run.ks.tma > 1 ? 1 : 0];
}

// Launch a phase-B kernel of the run (the TMA kernels also take their maps).
template <typename T>
static cudaError_t launch_b(const PcgRun<T> &run, const void *fn, cudaStream_t s)
{
    const PcgDesc<T> *dd = run.d_desc;
    void *args[] = {(void *)&dd, (void *)tma_params(run)};
    return cudaLaunchKernel(fn, dim3(run.grid_b), dim3(b_threads(run.ks)), args, run.ks.smem_b, s);
}

// The phase-B nodes of a TMA kernel set carry the run's tensor maps; other sets none.
template <typename T>
static const void *graph_tma(const PcgRun<T> &run)
{
    static const unsigned long long none[12 * 16] = {};
    return run.ks.tma ? (const void *)tma_params(run) : (const void *)none;
}

static bool graph_matches(const GraphCache &gc, int ga, int gb, int gs, const void *desc,
                          const void *ka, const void *kb, int pairs, const void *tma)
{
    return gc.exec && gc.grid_a == ga && gc.grid_b == gb && gc.grid_s == gs && gc.desc == desc &&
           gc.ka == ka && gc.kb == kb && gc.pairs == pairs &&
           std::memcmp(gc.tma, tma, sizeof(gc.tma)) == 0;
}

// Build and instantiate  [init B] -> WHILE{A -> B} -> [finalize]  for a launch
// shape.  The kernels read everything through the device descriptor, so one
// instantiated graph serves every problem of that shape.
template <typename T>
static int build_graph(PcgRun<T> &run, GraphCache &gc, cudaStream_t s, int pairs)
{
    if (gc.exec) {
        cudaGraphExecDestroy(gc.exec);
        gc.exec = nullptr;
    }
    cudaGraph_t g = nullptr;
    GMAF_CUDA(cudaGraphCreate(&g, 0));
    cudaGraphConditionalHandle h;
    cudaError_t e = cudaGraphConditionalHandleCreate(&h, g, 0u, cudaGraphCondAssignDefault);
    const PcgDesc<T> *dd = run.d_desc;
    void *args[] = {(void *)&dd};
    void *args_b[] = {(void *)&dd, (void *)tma_params(run)};   // the TMA kernels also take their maps
    cudaGraphNode_t n_init, n_while, n_fin, n_a, n_b;
    cudaKernelNodeParams kp{};
    kp.blockDim = dim3(kThreads);
    kp.kernelParams = args;
    if (e == cudaSuccess) {
        kp.blockDim = dim3(b_threads(run.ks));
        kp.func = (void *)run.ks.b_init;
        kp.gridDim = dim3(run.grid_b);
        kp.sharedMemBytes = (unsigned)run.ks.smem_b;
        kp.kernelParams = run.ks.tma ? args_b : args;
        e = cudaGraphAddKernelNode(&n_init, g, nullptr, 0, &kp);
    }
    cudaGraphNodeParams cp{};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = h;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    if (e == cudaSuccess) e = cudaGraphAddNode(&n_while, g, &n_init, nullptr, 1, &cp);
    if (e == cudaSuccess) {
        // the body runs `pairs` iterations per evaluation of the condition; once the
        // run is done, the remaining phases of the trip return at once (phase A also
        // writes "stop" to the condition before it looks at done)
        cudaGraph_t body = cp.conditional.phGraph_out[0];
        cudaGraphNode_t prev = nullptr;
        for (int q = 0; q < pairs && e == cudaSuccess; ++q) {
            kp.func = (void *)run.ks.a;
            kp.blockDim = dim3(run.ks.threads);
            kp.gridDim = dim3(run.grid_a);
            kp.sharedMemBytes = (unsigned)run.ks.smem_a;
            kp.kernelParams = args;
            e = cudaGraphAddKernelNode(&n_a, body, prev ? &prev : nullptr, prev ? 1 : 0, &kp);
            if (e == cudaSuccess) {
                kp.func = (void *)run.ks.b;
                kp.blockDim = dim3(b_threads(run.ks));
                kp.gridDim = dim3(run.grid_b);
                kp.sharedMemBytes = (unsigned)run.ks.smem_b;
                kp.kernelParams = run.ks.tma ? args_b : args;
                e = cudaGraphAddKernelNode(&n_b, body, &n_a, 1, &kp);
            }
            prev = n_b;
        }
    }
    if (e == cudaSuccess) {
        kp.blockDim = dim3(kThreads);
        kp.kernelParams = args;
        kp.func = (void *)k_finalize<T>;
        kp.gridDim = dim3(run.grid_s);
        kp.sharedMemBytes = 0;
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
    gc.ka = run.ks.a;
    gc.kb = run.ks.b;
    gc.pairs = pairs;
    std::memcpy(gc.tma, graph_tma(run), sizeof(gc.tma));
    (void)s;
    return GMAF_OK;
}

template <typename T>
static void shape_run(gmaf_ctx *ctx, PcgRun<T> &run, const KernelSet<T> &ks)
{
    PcgDesc<T> &h = run.h;
    run.ks = ks;
    h.ty = ks.TY;        // the staged kernels' task height (the others use their template's)
    h.tiles_x = (h.nth + ks.W - 1) / ks.W;
    h.tiles_y = (h.nz + ks.TY - 1) / ks.TY;
    h.ntiles = (long long)h.tiles_x * h.tiles_y * h.K;
    h.sgroups = 1;
    if (ks.sched) {
        // static schedule: both phases get the same warps, so that phase A walks
        // exactly phase B's ranges backward; groups of >= 4 rows on average
        int occ_a = 0, occ_b = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_a, ks.a, kThreads, ks.smem_a) !=
            cudaSuccess)
            occ_a = 1;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_b, ks.b, kThreads, ks.smem_b) !=
            cudaSuccess)
            occ_b = 1;
        const long long occ = std::max(1, std::min(occ_a, occ_b));
        const long long resident = occ * ctx->num_sms * kWarps;
        const long long L = (long long)h.tiles_x * h.nz;
        const long long G = std::max(1LL, std::min(resident / h.K, L / 4));
        const long long warps = std::min(resident, G * h.K);
        h.sgroups = G;
        run.grid_a = run.grid_b = (int)((warps + kWarps - 1) / kWarps);
    } else {
        run.grid_a = phase_grid(ks.a, h.ntiles, ctx->num_sms, ks.smem_a, ks.threads);
        run.grid_b = phase_grid(ks.b, h.ntiles, ctx->num_sms, ks.smem_b, ks.threads);
    }
    h.ty_b = 0;
    h.ntiles_b = 0;
    if (ks.tma) {
        // one block per task, tasks of ty_b rows
        h.ty_b = ks.ty_b;
        h.ntiles_b = (long long)h.tiles_x * ((h.nz + ks.ty_b - 1) / ks.ty_b) * h.K;
        run.grid_b = grid_for(ks.b, h.ntiles_b, ctx->num_sms, ks.smem_b, b_threads(ks));
    }
    run.grid_s = stream_grid(h.n * h.K, ctx->num_sms);
}

template <typename T>
static size_t partial_doubles(const PcgRun<T> &run)
{
    long long m = 2 * run.h.ntiles;
    if (2LL * run.h.ntiles_b > m) m = 2LL * run.h.ntiles_b;
    if (2LL * run.grid_s > m) m = 2LL * run.grid_s;
    // the static schedule publishes one partial pair per warp
    if (2LL * kWarps * run.grid_a > m) m = 2LL * kWarps * run.grid_a;
    if (2LL * kWarps * run.grid_b > m) m = 2LL * kWarps * run.grid_b;
    return (size_t)m;
}

// Buffers of the two-level reduction of the phase kernels: one chunk of 32
// publishing units (tasks, or warps under the static schedule).  The counters
// are zero when allocated and each launch leaves them zero.  Used from 4096
// units: below that the one-level sum is short, and the per-unit fence and
// counter cost more than they save (2048x1024x9, 4608 tasks: 0.2214 -> 0.2145 ms
// per iteration; 512x256x9, 1152 tasks: 0.0311 -> 0.0341 ms).
template <typename T>
static int attach_chunks(gmaf_ctx *ctx, PcgRun<T> &run)
{
    long long units = run.ks.sched ? (long long)run.grid_a * kWarps : run.h.ntiles;
    if (run.h.ntiles_b > units) units = run.h.ntiles_b;
    run.h.chunk_sum = nullptr;
    run.h.chunk_ctr = nullptr;
    if (units < ctx->chunked_from) return GMAF_OK;
    const long long chunks = (units + 31) / 32;
    GMAF_TRY(ensure(ctx, B_CHUNK, (size_t)chunks * 2 * sizeof(double)));
    GMAF_TRY(ensure(ctx, B_CHUNKCTR, (size_t)chunks * sizeof(unsigned)));
    run.h.chunk_sum = (double *)ctx->buf[B_CHUNK];
    run.h.chunk_ctr = (unsigned *)ctx->buf[B_CHUNKCTR];
    return GMAF_OK;
}

// Autotuner: time one iteration (phase A + phase B) of every candidate on the
// run's own data and keep the fastest for this shape.  The tuning iterate
// lives in run.h.p, which the real solve zero-initialises afterwards.
template <typename T>
static int autotune(gmaf_ctx *ctx, PcgRun<T> &run, KernelSet<T> *cand, int ncand, int *best_out)
{
    cudaStream_t s = ctx->stream;
    if (!ctx->ev_ready) {
        for (auto &ev : ctx->ev) GMAF_CUDA(cudaEventCreate(&ev));
        ctx->ev_ready = 1;
    }
    PcgRun<T> tr = run;
    tr.h.zero_init = 1;
    tr.h.eps = 1e-300;          // never converges during tuning
    tr.h.max_iter = 1 << 30;
    tr.h.use_cond = 0;
    // two round-robin passes, best time per candidate: the first pass also
    // brings the clocks up and loads every kernel
    float best_t[kMaxVariants];
    for (int c = 0; c < ncand; ++c) best_t[c] = 3.0e38f;
    for (int round = 0; round < 2; ++round) {
        for (int c = 0; c < ncand; ++c) {
            shape_run<T>(ctx, tr, cand[c]);
            GMAF_TRY(ensure(ctx, B_PART, partial_doubles(tr) * sizeof(double)));
            tr.h.partials = (double *)ctx->buf[B_PART];
            GMAF_TRY(attach_chunks<T>(ctx, tr));
            GMAF_CUDA(cudaMemcpyAsync(tr.d_desc, &tr.h, sizeof(PcgDesc<T>), cudaMemcpyHostToDevice, s));
            k_reset<<<1, 32, 0, s>>>(tr.h.sc, 0);
            k_init_r<T><<<tr.grid_s, kThreads, 0, s>>>(tr.d_desc);
            GMAF_CUDA(launch_b<T>(tr, tr.ks.b_init, s));
            const int warm = 3, reps = 10;
            for (int q = 0; q < warm + reps; ++q) {
                if (q == warm) GMAF_CUDA(cudaEventRecord(ctx->ev[0], s));
                GMAF_CUDA(launch<T>(tr.ks.a, tr.grid_a, tr.d_desc, s, tr.ks.smem_a, tr.ks.threads));
                GMAF_CUDA(launch_b<T>(tr, tr.ks.b, s));
            }
            GMAF_CUDA(cudaEventRecord(ctx->ev[1], s));
            GMAF_CUDA(cudaEventSynchronize(ctx->ev[1]));
            float ms = 0.0f;
            GMAF_CUDA(cudaEventElapsedTime(&ms, ctx->ev[0], ctx->ev[1]));
            if (ms < best_t[c]) best_t[c] = ms;
        }
    }
    // a later candidate replaces the pick only when it is more than 1% faster, so
    // that near-ties (within the timing noise) resolve to the earlier, preferred one
    int best_i = 0;
    for (int c = 1; c < ncand; ++c)
        if (best_t[c] < 0.99f * best_t[best_i]) best_i = c;
    *best_out = best_i;
    return GMAF_OK;
}

// Kernel set (tuned per shape), launch shape, partial-sum buffer and
// descriptor slot of a run.
template <typename T>
static int setup_run(gmaf_ctx *ctx, PcgRun<T> &run, PcgDesc<T> *desc_slot)
{
    PcgDesc<T> &h = run.h;
    run.d_desc = desc_slot;
    KernelSet<T> cand[kMaxVariants];
    const bool vo = vec_ok(h);
    run.tma_ready = false;
    if constexpr (sizeof(T) == 4)
        run.tma_ready = vo && tma_encode_maps(h, run.tma[0], 8) && tma_encode_maps(h, run.tma[1], 16);
    const int ncand = variants(cand, vo, vec8_ok(h), bulk_ok(h), run.tma_ready, run.drec_ready);
    int pick = 0;
    TuneEntry key{};
    key.tsize = (int)sizeof(T);
    key.nth = h.nth;
    key.nz = h.nz;
    key.K = h.K;
    key.precond = h.precond;
    key.vec_ok = vo ? 1 : 0;
    int found = -1;
    for (int q = 0; q < ctx->ntune; ++q) {
        const TuneEntry &e = ctx->tune[q];
        if (e.tsize == key.tsize && e.nth == key.nth && e.nz == key.nz && e.K == key.K &&
            e.precond == key.precond && e.vec_ok == key.vec_ok)
            found = q;
    }
    int forced = -1;
    for (int q = 0; q < ncand; ++q)
        if (cand[q].id == ctx->force_variant) forced = q;
    if (forced >= 0) {
        pick = forced;
    } else if (found >= 0) {
        pick = ctx->tune[found].choice;
    } else if (!ctx->no_tune && ncand > 1 && h.zero_init) {
        GMAF_TRY(autotune<T>(ctx, run, cand, ncand, &pick));
        key.choice = pick;
        const int slot = ctx->ntune < kTuneEntries ? ctx->ntune++ : (ctx->tune_next++ % kTuneEntries);
        ctx->tune[slot] = key;
    }
    if (pick < 0 || pick >= ncand) pick = 0;
    shape_run<T>(ctx, run, cand[pick]);
    GMAF_TRY(ensure(ctx, B_PART, partial_doubles(run) * sizeof(double)));
    h.partials = (double *)ctx->buf[B_PART];
    GMAF_TRY(attach_chunks<T>(ctx, run));
    return GMAF_OK;
}

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
        if (!graph_matches(gc, run.grid_a, run.grid_b, run.grid_s, run.d_desc, run.ks.a, run.ks.b,
                           ctx->graph_pairs, graph_tma(run)))
            GMAF_TRY(build_graph<T>(run, gc, ctx->stream, ctx->graph_pairs));
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
    // After the stream has been synchronised.  Only the first `real_pairs` phase A
    // and phase B launches of the chunk ran an iteration; the ones issued after the
    // run was done returned at once and are not counted.
    void collect(long long real_pairs)
    {
        long long seen[2] = {0, 0};
        for (int q = 0; q < used; ++q) {
            const int k = kinds[q];
            if (k < 2 && seen[k]++ >= real_pairs) continue;
            float ms = 0.0f;
            if (cudaEventElapsedTime(&ms, ctx->ev[2 * q], ctx->ev[2 * q + 1]) == cudaSuccess) {
                ctx->phase_ms[k] += ms;
                ctx->phase_count[k] += 1;
            }
        }
        used = 0;
    }
};

static_assert(offsetof(Scalars, done) == offsetof(Scalars, iter) + 2 * sizeof(int),
              "iter, first and done are read back together");

// [reset] [init_r] [init B] WHILE{A, B} [finalize], all on the stream.
template <typename T>
static int pcg_once(gmaf_ctx *ctx, PcgRun<T> &run, GraphCache &gc, bool keep_iter, bool do_init_r,
                    double cont_scale = 0.0)
{
    cudaStream_t s = ctx->stream;
    if (cont_scale > 0.0)
        k_continue<<<1, 32, 0, s>>>(run.h.sc, cont_scale);
    else
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
    const PcgDesc<T> *dd = run.d_desc;
    int *it_h = (int *)ctx->pinned;        // iter, first, done of the scalars
    PhaseClock clk{ctx};
    clk.begin(s);
    GMAF_CUDA(launch_b<T>(run, run.ks.b_init, s));
    clk.end(s, 2);
    const int chunk = 16;
    int prev_iter = -1;
    for (int it = 0; it <= run.h.max_iter + chunk; it += chunk) {
        GMAF_CUDA(cudaMemcpyAsync(it_h, &run.h.sc->iter, 3 * sizeof(int), cudaMemcpyDeviceToHost, s));
        GMAF_CUDA(cudaStreamSynchronize(s));
        // every iteration that ran advanced iter by one (phase B's last block)
        clk.collect(prev_iter < 0 ? 0 : it_h[0] - prev_iter);
        prev_iter = it_h[0];
        if (it_h[2]) break;
        for (int q = 0; q < chunk; ++q) {
            clk.begin(s);
            GMAF_CUDA(launch<T>(run.ks.a, run.grid_a, dd, s, run.ks.smem_a, run.ks.threads));
            clk.end(s, 0);
            clk.begin(s);
            GMAF_CUDA(launch_b<T>(run, run.ks.b, s));
            clk.end(s, 1);
        }
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


// ---------------------------------------------------------------- asynchronized criterion
//
// Eq. 3.10: condition k is its own PCG (own alpha, beta, d, Table 1) and stops
// when ||A_k p_k - S_k|| / ||S_k|| <= eps.  All conditions run in one
// persistent launch per CG phase (k_mphase_a/b over one-condition groups); a
// condition that has converged drops out through the done flag of its
// scalars, on the device, with no relaunch or resizing from the host.  The
// host reads the "every condition done" flag once per kAsyncChunk iterations.
// After the loop each condition gets the FP64 true-residual check of the
// synchronized path (one restart from the true residual if it fails).  FP64.
constexpr int kAsyncChunk = 32;

static size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

// DB > 0: phase B staged DB rows ahead (VEC = 2).
template <int VEC, int TY, int MINB, int DB>
static int solve_async64(gmaf_ctx *ctx, int nth, int nz, int K, const int *cslot_host,
                         const double *D, const double *invD, const double *aE, const double *aN,
                         const double *S, double *p, const gmaf_solver_opts *opts,
                         gmaf_solve_info *info)
{
    cudaStream_t s = ctx->stream;
    constexpr int W = 32 * VEC;
    const long long n = (long long)nth * nz;
    Scalars *scal = (Scalars *)ctx->buf[B_SCAL];
    Scalars *msc = scal + 2;                   // tickets and task counters of the batched launches
    Scalars *gsc = scal + 3;                   // [K] per-condition PCG scalars
    Scalars *rsc = scal + 3 + kMaxCond;        // [K] per-condition true residuals
    // device descriptors: MultiDesc, PcgDesc[K], ResidDesc[K], the one-slot table {0}
    const size_t o_groups = align256(sizeof(MultiDesc<double>));
    const size_t o_resid = o_groups + align256((size_t)kMaxCond * sizeof(PcgDesc<double>));
    const size_t o_slot = o_resid + align256((size_t)kMaxCond * sizeof(ResidDesc));
    GMAF_TRY(ensure(ctx, B_ASYNC, o_slot + 256));
    char *abase = (char *)ctx->buf[B_ASYNC];
    MultiDesc<double> *d_m = (MultiDesc<double> *)abase;
    PcgDesc<double> *d_groups = (PcgDesc<double> *)(abase + o_groups);
    ResidDesc *d_rd = (ResidDesc *)(abase + o_resid);
    int *d_slot0 = (int *)(abase + o_slot);

    const int tiles_x = (nth + W - 1) / W, tiles_y = (nz + TY - 1) / TY;
    const long long ntiles = (long long)tiles_x * tiles_y;
    const long long total = ntiles * K;
    const int gs = stream_grid(n, ctx->num_sms);
    long long np = 2 * total;
    if (2LL * gs > np) np = 2LL * gs;
    GMAF_TRY(ensure(ctx, B_PART, (size_t)np * sizeof(double)));
    double *partials = (double *)ctx->buf[B_PART];

    std::vector<PcgDesc<double>> g(K);
    std::vector<ResidDesc> rd(K);
    double *z = (double *)ctx->buf[B_Z], *v = (double *)ctx->buf[B_V];
    double *u0 = (double *)ctx->buf[B_U0], *u1 = (double *)ctx->buf[B_U1];
    double *r0 = (double *)ctx->buf[B_R0], *r1 = (double *)ctx->buf[B_R1];
    for (int k = 0; k < K; ++k) {
        const long long o = (long long)k * n, c = (long long)cslot_host[k] * n;
        PcgDesc<double> &h = g[k];
        h = PcgDesc<double>{};
        h.nth = nth;
        h.nz = nz;
        h.K = 1;
        h.tiles_x = tiles_x;
        h.tiles_y = tiles_y;
        h.precond = kernel_precond(opts);
        h.zero_init = opts->zero_init;
        h.use_cond = 0;
        h.n = n;
        h.ntiles = ntiles;
        h.sgroups = 1;
        h.D = D + c;
        h.invD = invD + c;
        h.aE = aE + c;
        h.aN = aN + c;
        h.cslot = d_slot0;
        h.b = S + o;
        h.p = p + o;
        h.z = z + o;
        h.v = v + o;
        h.u[0] = u0 + o;
        h.u[1] = u1 + o;
        h.r[0] = r0 + o;
        h.r[1] = r1 + o;
        h.omega = opts->omega;
        h.eps = opts->eps;
        h.max_iter = opts->max_iter;
        h.sc = gsc + k;
        h.guard_limit = ctx->loop_guard;
        h.partials = partials;
        ResidDesc &q = rd[k];
        q = ResidDesc{};
        q.nth = nth;
        q.nz = nz;
        q.K = 1;
        q.n = n;
        q.D = D + c;
        q.aE = aE + c;
        q.aN = aN + c;
        q.cslot = d_slot0;
        q.S = S + o;
        q.p = p + o;
        q.sc = rsc + k;
        q.partials = partials;
    }
    MultiDesc<double> hm{};
    hm.ngroups = K;
    hm.total_tasks = (unsigned)total;
    for (int k = 0; k <= K; ++k) hm.task_off[k] = (unsigned)(ntiles * k);
    hm.groups = d_groups;
    hm.msc = msc;
    hm.partials = partials;
    // two-level reduction per condition: chunks of kChunk tasks; the counters
    // ([kMaxGroups] group counters, then the chunk counters) are zero between launches
    const long long nch = (ntiles + kChunk - 1) / kChunk;
    for (int k = 0; k <= K; ++k) hm.chunk_off[k] = (unsigned)(nch * k);
    GMAF_TRY(ensure(ctx, B_CHUNK, (size_t)2 * nch * K * sizeof(double)));
    GMAF_TRY(ensure(ctx, B_CHUNKCTR, (size_t)(kMaxGroups + nch * K) * sizeof(unsigned)));
    hm.chunk_sum = (double *)ctx->buf[B_CHUNK];
    hm.group_ctr = (unsigned *)ctx->buf[B_CHUNKCTR];
    hm.chunk_ctr = hm.group_ctr + kMaxGroups;
    const int zero = 0;
    // pageable sources: each copy has consumed its source when it returns
    GMAF_CUDA(cudaMemcpyAsync(d_slot0, &zero, sizeof(int), cudaMemcpyHostToDevice, s));
    GMAF_CUDA(cudaMemcpyAsync(d_groups, g.data(), (size_t)K * sizeof(PcgDesc<double>),
                              cudaMemcpyHostToDevice, s));
    GMAF_CUDA(cudaMemcpyAsync(d_m, &hm, sizeof(hm), cudaMemcpyHostToDevice, s));

    const void *kb_init = (const void *)k_phase_b<double, VEC, TY, MINB, true, 0>;
    const int grid_b = phase_grid(kb_init, ntiles, ctx->num_sms);
    const void *kma = (const void *)k_mphase_a<double, VEC, TY, MINB, 0>;
    const void *kmb = (const void *)k_mphase_b<double, VEC, TY, MINB, DB>;
    const size_t smem_b = DB > 0 ? (size_t)kWarps * RingB<double, VEC>::per_warp(DB) * sizeof(double) : 0;
    if (DB > 0) {
        static std::atomic<unsigned long long> done_mb{0};
        smem_optin(done_mb, kmb, smem_b);
    }
    const int grid_m = std::min(phase_grid(kma, total, ctx->num_sms),
                                phase_grid(kmb, total, ctx->num_sms, smem_b));
    void *margs[] = {(void *)&d_m};
    GMAF_CUDA(cudaMemsetAsync(rsc, 0, (size_t)K * sizeof(Scalars), s));   // clean residual records
    // start: r0 = S_k - A_k p0, z0, d0 and the first criterion test, per condition
    for (int k = 0; k < K; ++k) {
        k_reset<<<1, 32, 0, s>>>(gsc + k, 0);
        k_init_r<double><<<gs, kThreads, 0, s>>>(d_groups + k);
        GMAF_CUDA(launch<double>(kb_init, grid_b, d_groups + k, s));
    }
    GMAF_CUDA(cudaGetLastError());
    std::vector<Scalars> hg(K), hr(K);
    std::vector<int> ran(K, 1), restarted(K, 0), final_ok(K, 0);
    std::vector<double> true_rel(K, 0.0);
    int *done_h = (int *)ctx->pinned;
    for (;;) {
        GMAF_CUDA(cudaMemsetAsync(msc, 0, sizeof(Scalars), s));
        for (long long it = 0; it <= (long long)opts->max_iter + 2 * kAsyncChunk; it += kAsyncChunk) {
            for (int q = 0; q < kAsyncChunk; ++q) {
                GMAF_CUDA(cudaLaunchKernel(kma, dim3(grid_m), dim3(kThreads), margs, 0, s));
                GMAF_CUDA(cudaLaunchKernel(kmb, dim3(grid_m), dim3(kThreads), margs, smem_b, s));
            }
            GMAF_CUDA(cudaGetLastError());
            GMAF_CUDA(cudaMemcpyAsync(done_h, &msc->done, sizeof(int), cudaMemcpyDeviceToHost, s));
            GMAF_CUDA(cudaStreamSynchronize(s));
            if (*done_h) break;
        }
        // the deferred p += alpha u of each condition that ran, then its true residual
        GMAF_CUDA(cudaMemcpyAsync(hg.data(), gsc, (size_t)K * sizeof(Scalars), cudaMemcpyDeviceToHost, s));
        GMAF_CUDA(cudaStreamSynchronize(s));
        for (int k = 0; k < K; ++k) {
            if (!ran[k]) continue;
            k_finalize<double><<<gs, kThreads, 0, s>>>(d_groups + k);
            rd[k].r = g[k].r[hg[k].iter & 1];        // where a restart reads it
            GMAF_CUDA(cudaMemcpyAsync(d_rd + k, &rd[k], sizeof(ResidDesc), cudaMemcpyHostToDevice, s));
            k_resid64<<<gs, kThreads, 0, s>>>(d_rd + k);
        }
        GMAF_CUDA(cudaGetLastError());
        GMAF_CUDA(cudaMemcpyAsync(hr.data(), rsc, (size_t)K * sizeof(Scalars), cudaMemcpyDeviceToHost, s));
        GMAF_CUDA(cudaStreamSynchronize(s));
        bool again = false;
        for (int k = 0; k < K; ++k) {
            if (!ran[k]) continue;
            ran[k] = 0;
            true_rel[k] = hr[k].true_rel;
            if (hg[k].zero_rhs) {
                GMAF_CUDA(cudaMemsetAsync(p + (long long)k * n, 0, (size_t)n * sizeof(double), s));
                true_rel[k] = 0.0;
            }
            if (hg[k].status != 0 || hr[k].status != 0) continue;
            if ((hg[k].converged || hg[k].zero_rhs) && true_rel[k] <= 10.0 * opts->eps) {
                final_ok[k] = 1;
                continue;
            }
            if (restarted[k] || hg[k].iter >= opts->max_iter) continue;
            // restart condition k from its true residual (already in r[iter & 1])
            restarted[k] = 1;
            ran[k] = 1;
            again = true;
            k_reset<<<1, 32, 0, s>>>(gsc + k, 1);
            GMAF_CUDA(launch<double>(kb_init, grid_b, d_groups + k, s));
        }
        GMAF_CUDA(cudaGetLastError());
        if (!again) break;
    }
    GMAF_CUDA(cudaStreamSynchronize(s));
    gmaf_solve_info inf{};
    int status = GMAF_OK;
    for (int k = 0; k < K; ++k) {
        inf.iterations = std::max(inf.iterations, hg[k].iter);
        inf.iterations_sum += hg[k].iter;
        inf.rel_residual = std::max(inf.rel_residual, hg[k].rel);
        inf.true_rel_residual = std::max(inf.true_rel_residual, true_rel[k]);
        inf.restarts += restarted[k];
        const int st = hg[k].status != 0 ? hg[k].status : hr[k].status;
        if (st != 0 && status == GMAF_OK) status = st;
        if (!final_ok[k] && st == 0 && status == GMAF_OK) status = GMAF_NOT_CONVERGED;
    }
    inf.status = status;
    inf.outer_iterations = 1;
    inf.kernel_variant = 1000 * VEC + 10 * TY + MINB;
    inf.tasks = (int)total;
    inf.p_update_period = 1;
    *info = inf;
    return status;
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
    // [0] PCG run, [1] outer / true residual, [2] batched-launch tickets, then the
    // per-condition scalars of the asynchronized criterion ([kMaxCond] PCG, [kMaxCond] residual)
    GMAF_TRY(ensure(ctx, B_SCAL, (3 + 2 * kMaxCond) * sizeof(Scalars)));
    Scalars *dsc = (Scalars *)ctx->buf[B_SCAL];        // PCG run (FP64, or FP32 inner)
    Scalars *dsc_outer = dsc + 1;                       // FP64 residual of the outer loop
    // the residual kernel only ever raises its status: start every solve from a
    // clean record, so that a non-finite earlier solve does not leak into this one
    GMAF_CUDA(cudaMemsetAsync(dsc_outer, 0, sizeof(Scalars), s));
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
        diag_inverse64(opts, D, aE, aN, nth, nz, m, (double *)ctx->buf[B_INVD], ctx->num_sms, s);
        GMAF_CUDA(cudaGetLastError());
        if (opts->criterion == 1) {
            const bool vec = (nth % 2) == 0;     // 16-byte rows of doubles in every condition
            const double *iv = (const double *)ctx->buf[B_INVD];
            return vec ? solve_async64<2, 32, 2, 2>(ctx, nth, nz, K, cslot_host, D, iv, aE, aN, S, p, opts, info)
                       : solve_async64<1, 32, 3, 0>(ctx, nth, nz, K, cslot_host, D, iv, aE, aN, S, p, opts, info);
        }
        PcgRun<double> run{};
        PcgDesc<double> &h = run.h;
        h.nth = nth;
        h.nz = nz;
        h.K = K;
        h.n = n;
        h.precond = kernel_precond(opts);
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
        h.eps = opts->eps;
        h.max_iter = opts->max_iter;
        h.sc = dsc;
        h.guard_limit = ctx->loop_guard;
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
                clk.collect(0);
            }
            double true_rel = ho->true_rel;
            if (hsc->zero_rhs) {
                GMAF_CUDA(cudaMemsetAsync(p, 0, (size_t)N * sizeof(double), s));
                GMAF_CUDA(cudaStreamSynchronize(s));
                true_rel = 0.0;
            }
            inf.iterations = hsc->iter;
            inf.iterations_sum = hsc->iter * K;
            inf.rel_residual = hsc->rel;
            inf.true_rel_residual = true_rel;
            inf.restarts = restarted;
            inf.outer_iterations = 1;
            inf.kernel_variant = run.ks.id;
            inf.tasks = (int)run.h.ntiles;
            inf.p_update_period = std::max(1, run.ks.p_period);
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
        (float *)ctx->buf[B_AN32], m, dsc_outer, opts->precond == 1 ? opts->omega : 1.0);
    if (opts->precond == 2)
        k_assor1_diag<float><<<stream_grid(m, ctx->num_sms), kThreads, 0, s>>>(
            D, aE, aN, nth, nz, m, opts->omega, dsc_outer, (float *)ctx->buf[B_INVD32]);
    GMAF_CUDA(cudaGetLastError());
    if (opts->zero_init) GMAF_CUDA(cudaMemsetAsync(p, 0, (size_t)N * sizeof(double), s));

    PcgRun<float> run{};
    PcgDesc<float> &h = run.h;
    h.nth = nth;
    h.nz = nz;
    h.K = K;
    h.n = n;
    h.precond = kernel_precond(opts);
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
    h.sc = dsc;
    h.nslots = nslots;
    if (nth % 4 == 0) {
        // the boundary term of the diagonal for the phase A variant that rebuilds it
        GMAF_TRY(ensure(ctx, B_DBND32, (size_t)nslots * 2 * nth * sizeof(float)));
        GMAF_TRY(launch_dbnd32(h.D, h.aE, h.aN, (float *)ctx->buf[B_DBND32], nth, nz, nslots,
                               ctx->num_sms, s));
        h.dbnd = (const float *)ctx->buf[B_DBND32];
        run.drec_ready = true;
    }
    // The first outer residual and the inner right-hand side are formed before the
    // kernel set is chosen, so that the autotuner times iterations on real data.
    GMAF_TRY(ensure(ctx, B_PART, (size_t)2 * gs * sizeof(double)));
    rd.partials = (double *)ctx->buf[B_PART];
    rd.sc = dsc_outer;
    rd.r = (double *)ctx->buf[B_R64];
    GMAF_CUDA(cudaMemcpyAsync(d_rdesc, &rd, sizeof(ResidDesc), cudaMemcpyHostToDevice, s));

    // Refinement: p64 += the inner FP32 solution, r64 = S - A p64 in FP64, repeated
    // until the FP64 residual meets eps.  By default the inner PCG is not
    // restarted at a refinement: its residual is replaced by the FP64 one (a
    // reliable update) and the recurrence continues with its direction u, so the
    // Krylov information gathered so far is kept.  The residual is refreshed
    // after every reduction by reliable_delta (GMAF_RELIABLE_DELTA, 0.1), before
    // the FP32 recurrence drifts far from the true residual.  GMAF_MIXED_RESTART=1
    // restarts the inner solve from each new residual instead, solving it down to
    // the inner floor (GMAF_INNER_EPS) each time.
    const bool continued = !ctx->mixed_restart;
    const double inner_floor = continued ? ctx->reliable_delta : ctx->inner_floor;
    const int max_outer = continued ? 200 : 12;
    int total_inner = 0, outer = 0, longest = 0;
    int last_iter = 0;          // the inner iteration counter at the end of the last solve
    bool tuned = false, stalled = false;
    double rnorm_prev = 0.0;
    inf.status = GMAF_NOT_CONVERGED;
    for (;;) {
        {
            PhaseClock clk{ctx};
            clk.begin(s);
            k_resid64<<<gs, kThreads, 0, s>>>(d_rdesc);
            clk.end(s, 3);
            GMAF_CUDA(cudaGetLastError());
            GMAF_TRY(read_scalars(ctx, dsc_outer, ho));
            clk.collect(0);
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
        k_make_b32<<<gs, kThreads, 0, s>>>((const double *)ctx->buf[B_R64], (float *)ctx->buf[B_B32],
                                           N, dsc_outer);
        GMAF_CUDA(cudaGetLastError());
        if (!tuned) {
            GMAF_TRY(setup_run<float>(ctx, run, (PcgDesc<float> *)(dbase + 1024)));
            rd.partials = h.partials;
            GMAF_CUDA(cudaMemcpyAsync(d_rdesc, &rd, sizeof(ResidDesc), cudaMemcpyHostToDevice, s));
            tuned = true;
        }
        // inner tolerance: a fixed reduction, but no further than the outer target needs
        double eps_in = 0.5 * opts->eps / ho->true_rel;
        if (eps_in < inner_floor) eps_in = inner_floor;
        if (eps_in > 0.5) eps_in = 0.5;
        h.eps = eps_in;
        const bool cont = outer > 0 && continued && rnorm_prev > 0.0 && !stalled;
        // a continued recurrence keeps counting from where the last solve stopped;
        // one that needs more than max(1000, 4 x the longest solve so far) for its
        // reduction is cut off, and the next solve restarts from its residual
        const int left = opts->max_iter - total_inner;
        const int cap = std::max(1000, 4 * longest);
        h.max_iter = cont ? last_iter + std::min(left, cap) : left;
        h.guard_limit = ctx->loop_guard;
        GMAF_TRY(prepare<float>(ctx, run, ctx->graph32));
        GMAF_TRY(pcg_once<float>(ctx, run, ctx->graph32, cont, true, cont ? rnorm_prev / ho->rnorm : 0.0));
        rnorm_prev = ho->rnorm;
        k_update_p64<<<gs, kThreads, 0, s>>>(p, (const float *)ctx->buf[B_X32], N, dsc_outer);
        GMAF_CUDA(cudaGetLastError());
        GMAF_TRY(read_scalars(ctx, dsc, hsc));
        const int seg = cont ? hsc->iter - last_iter : hsc->iter;     // iterations of this solve
        last_iter = hsc->iter;
        total_inner += seg;
        longest = std::max(longest, seg);
        stalled = continued && !hsc->converged;
        ++outer;
        if (hsc->status != 0) {
            inf.status = hsc->status;
            break;
        }
        if (seg == 0) break;     // no progress possible
    }
    inf.iterations = total_inner;
    inf.iterations_sum = total_inner * K;
    inf.outer_iterations = outer;
    inf.kernel_variant = run.ks.id;
    inf.tasks = (int)run.h.ntiles;
    inf.p_update_period = std::max(1, run.ks.p_period);
    *info = inf;
    return inf.status;
}

}  // namespace gmaf
