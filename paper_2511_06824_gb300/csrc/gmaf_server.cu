// Continuous-batching server for Picard-step requests (mixed precision).
//
// A request is one general Picard iteration (Eq. 2.12-2.19) of a 9-condition
// joint system on its own grid.  Requests are admitted first-come first-served
// while their device footprint fits in the server's arena (a sub-allocator over
// one allocation of the HBM budget), each becomes a group of the batched
// persistent PCG kernels (k_mphase_a/b), and the host advances the whole set in
// rounds of a fixed number of iterations.  Between rounds, groups whose inner
// FP32 solve finished take their FP64 refinement step (update, FP64 residual)
// and either start the next inner solve or retire (loads, Jacobian, update,
// result copied to the host), which frees their arena block for queued
// requests.  Each group keeps its own scalars and buffers and the kernels reduce
// each group over its own tasks in task order, so a request's result is the
// same whether it runs alone or among others.
#include <algorithm>
#include <cstdlib>
#include <cmath>
#include <cstring>
#include <deque>
#include <mutex>
#include <new>
#include <vector>

#include "gmaf_internal.cuh"
#include "gmaf_pcg_kernels.cuh"
#include "gmaf_mphase_kernels.cuh"

namespace gmaf {

// Kernel variant of the served requests (n_theta % 4 == 0): 128-column tasks.
// The batched kernels are one instantiation shared by every group (one
// persistent kernel per CG phase), so columns per lane and staging are fixed;
// the task height is per group (PcgDesc::ty), chosen per grid by the tuner
// below.  A request's task decomposition depends only on its grid, never on
// what else is running.
constexpr int kSvVec = 4, kSvTY = 32, kSvMinB = 2;
constexpr int kSvW = 32 * kSvVec;
constexpr int kSvStage = 2;            // rows staged ahead by cp.async (0: register prefetch)
constexpr int kSvTyCand[] = {32, 16, 64};   // tuner candidates, the default first
constexpr int kSvTyMin = 16;                // smallest candidate (sizes the partial sums)

// Tuner decisions, shared by every server of the process: the first request of
// a grid on a device fixes the task height of that grid (for the kernel form
// the server uses), so the same grid is always decomposed the same way.
struct SvTuneEntry {
    int dev, nth, nz, staged, ty;
};
static std::mutex g_sv_tune_mutex;
static std::vector<SvTuneEntry> g_sv_tune;

static int sv_tuned_rows(int dev, int nth, int nz, int staged)
{
    std::lock_guard<std::mutex> lock(g_sv_tune_mutex);
    for (const auto &e : g_sv_tune)
        if (e.dev == dev && e.nth == nth && e.nz == nz && e.staged == staged) return e.ty;
    return 0;
}

static int sv_record_rows(int dev, int nth, int nz, int staged, int ty)
{
    std::lock_guard<std::mutex> lock(g_sv_tune_mutex);
    for (const auto &e : g_sv_tune)     // another server may have decided first: keep its pick
        if (e.dev == dev && e.nth == nth && e.nz == nz && e.staged == staged) return e.ty;
    g_sv_tune.push_back({dev, nth, nz, staged, ty});
    return ty;
}

static long long sv_tasks(int nth, int nz, int ty)
{
    return (long long)((nth + kSvW - 1) / kSvW) * ((nz + ty - 1) / ty) * 9;
}

// The two batched phase kernels of the server and their dynamic shared memory.
struct SvKernels {
    const void *a, *b;
    size_t smem_a, smem_b;
};

static SvKernels sv_kernels(bool staged)
{
    if (!staged)
        return {(const void *)k_mphase_a<float, kSvVec, kSvTY, kSvMinB, 0>,
                (const void *)k_mphase_b<float, kSvVec, kSvTY, kSvMinB, 0>, 0, 0};
    SvKernels k{(const void *)k_mphase_a<float, kSvVec, kSvTY, kSvMinB, kSvStage>,
                (const void *)k_mphase_b<float, kSvVec, kSvTY, kSvMinB, kSvStage>,
                (size_t)kWarps * RingA<float, kSvVec, true>::per_warp(kSvStage) * sizeof(float),
                (size_t)kWarps * RingB<float, kSvVec>::per_warp(kSvStage) * sizeof(float)};
    static std::atomic<unsigned long long> done_a{0}, done_b{0};
    smem_optin(done_a, k.a, k.smem_a);
    smem_optin(done_b, k.b, k.smem_b);
    return k;
}

// ------------------------------------------------------------------ arena

// First-fit sub-allocator with coalescing over [0, size), 256-byte granules.
class Arena {
public:
    void reset(size_t size)
    {
        size_ = size;
        free_.clear();
        free_.push_back({0, size});
    }
    bool alloc(size_t bytes, size_t *off)
    {
        bytes = round_up(bytes);
        for (size_t i = 0; i < free_.size(); ++i) {
            if (free_[i].size >= bytes) {
                *off = free_[i].off;
                free_[i].off += bytes;
                free_[i].size -= bytes;
                if (free_[i].size == 0) free_.erase(free_.begin() + (long)i);
                return true;
            }
        }
        return false;
    }
    void release(size_t off, size_t bytes)
    {
        bytes = round_up(bytes);
        size_t i = 0;
        while (i < free_.size() && free_[i].off < off) ++i;
        free_.insert(free_.begin() + (long)i, {off, bytes});
        if (i + 1 < free_.size() && free_[i].off + free_[i].size == free_[i + 1].off) {
            free_[i].size += free_[i + 1].size;
            free_.erase(free_.begin() + (long)i + 1);
        }
        if (i > 0 && free_[i - 1].off + free_[i - 1].size == free_[i].off) {
            free_[i - 1].size += free_[i].size;
            free_.erase(free_.begin() + (long)i);
        }
    }
    size_t free_bytes() const
    {
        size_t s = 0;
        for (const auto &b : free_) s += b.size;
        return s;
    }
    static size_t round_up(size_t b) { return (b + 255) & ~size_t(255); }

private:
    struct Blk {
        size_t off, size;
    };
    std::vector<Blk> free_;
    size_t size_ = 0;
};

// ------------------------------------------------------------------ requests

struct Request {
    int64_t id;
    gmaf_request in;
    Geom g;
    long long n, N, ntasks;
    int ty;                       // rows per task (kSvTY until tuned)
    size_t off, bytes;
    // fields carved from the arena block
    double *D, *aE, *aN, *S, *p, *r64, *trig, *conds, *loads, *result, *part;
    float *D32, *invD32, *aE32, *aN32, *b32, *x32, *r32[2], *u32[2], *z32, *v32;
    int *cslot_w, *cslot, *flags;
    unsigned *tickets;
    Scalars *sc_in, *sc_out;
    PcgDesc<float> *d_desc;
    ResidDesc *d_rdesc;
    PcgDesc<float> h;
    ResidDesc rd;
    int outer, total_inner, grid_s;
    // continued inner recurrence (reliable updates, as in the joint solve)
    double rnorm_prev;            // norm of the FP64 residual the last inner solve started from
    int last_iter, longest;       // inner iteration counter after the last solve; longest solve
    bool cont_run, stalled;       // the last solve continued the recurrence; it stalled
    bool no_progress;             // the last solve made no iteration
    double rel0, rnorm0;          // FP64 residual at admission (p = 0)
};

constexpr size_t kHdrBytes = 8192;   // scalars, descriptors, conditions, flags, loads, result

static size_t loads_part_doubles(int num_sms) { return (size_t)9 * num_sms * 2 * 12; }

static size_t partial_doubles_for(long long ntasks, int grid_s, int num_sms)
{
    size_t m = (size_t)(2 * ntasks);
    if ((size_t)2 * grid_s > m) m = (size_t)2 * grid_s;
    const size_t lp = loads_part_doubles(num_sms);
    return m > lp ? m : lp;
}

static int stream_grid_s(long long N, int num_sms)
{
    long long g = (N + kThreads - 1) / kThreads;
    const long long cap = (long long)num_sms * 8;
    if (g > cap) g = cap;
    if (g < 1) g = 1;
    return (int)g;
}

// Device bytes of one request of this grid (what admission checks against the arena).
static size_t footprint(int nth, int nz, int num_sms)
{
    const long long n = (long long)nth * nz, N = 9 * n, m = 5 * n;
    const long long ntasks = sv_tasks(nth, nz, kSvTyMin);   // the most tasks any tiling has
    size_t b = kHdrBytes;
    b += Arena::round_up((size_t)4 * nth * sizeof(double));                          // trig
    b += Arena::round_up(partial_doubles_for(ntasks, stream_grid_s(N, num_sms), num_sms) *
                         sizeof(double));                                            // partials
    b += 3 * Arena::round_up((size_t)m * sizeof(double));                            // D aE aN
    b += 3 * Arena::round_up((size_t)N * sizeof(double));                            // S p r64
    b += 4 * Arena::round_up((size_t)m * sizeof(float));                             // FP32 slots
    b += 8 * Arena::round_up((size_t)N * sizeof(float));                             // FP32 vectors
    return b;
}

}  // namespace gmaf

using namespace gmaf;

struct gmaf_server {
    gmaf_ctx *ctx;
    cudaStream_t stream;
    int num_sms;
    char *base;
    size_t budget;
    Arena arena;
    std::deque<Request *> queue;
    std::vector<Request *> active;
    std::vector<gmaf_result> finished;
    int64_t next_id;
    // batched launches
    MultiDesc<float> *d_mdesc;
    PcgDesc<float> *d_groups;
    Scalars *msc;
    double *mpart;
    size_t mpart_cap;
    double *mchunk;                // chunk sums of the batched reduction
    size_t mchunk_cap;
    unsigned *mctr;                // [kMaxGroups] group counters, then the chunk counters
    size_t mctr_cap;
    bool dirty;
    MultiDesc<float> hm;
    int grid_m;
    SvKernels kern;
    int device;
    int staged;                    // kernel form: rows staged by cp.async (1) or not (0)
    int tune;                      // tune the task height per grid (GMAF_SV_TUNE, default 1)
    int use_graph;                 // rounds as CUDA graphs (GMAF_SV_GRAPH, default 1)
    // tuner: a one-group batched table and two events
    PcgDesc<float> *d_tune_group;
    MultiDesc<float> *d_tune_mdesc;
    cudaEvent_t ev[2];
    // the round graph: `iters` phase pairs on the batched table, launch grid `grid`
    cudaGraph_t graph;
    cudaGraphExec_t graph_exec;
    std::vector<cudaGraphNode_t> graph_nodes;
    int graph_grid, graph_iters;
    const void *graph_a, *graph_b;
};

namespace gmaf {

static void carve(gmaf_server *sv, Request *r)
{
    char *b = sv->base + r->off;
    const long long n = r->n, N = r->N, m = 5 * n;
    // header
    r->sc_in = (Scalars *)(b + 0);
    r->sc_out = (Scalars *)(b + 256);
    r->d_desc = (PcgDesc<float> *)(b + 512);
    r->d_rdesc = (ResidDesc *)(b + 1536);
    r->conds = (double *)(b + 2048);           // 9 x 8 doubles
    r->cslot_w = (int *)(b + 2816);            // 9 ints
    r->cslot = (int *)(b + 2880);              // 9 ints
    r->flags = (int *)(b + 2944);
    r->tickets = (unsigned *)(b + 3072);       // 64
    r->loads = (double *)(b + 3584);           // 9 x 12
    r->result = (double *)(b + 4608);          // kResultDoubles
    size_t o = kHdrBytes;
    auto take = [&](size_t bytes) {
        char *q = b + o;
        o += Arena::round_up(bytes);
        return q;
    };
    r->trig = (double *)take((size_t)4 * r->g.nth * sizeof(double));
    r->part = (double *)take(partial_doubles_for(sv_tasks(r->g.nth, r->g.nz, kSvTyMin), r->grid_s,
                                                 sv->num_sms) * sizeof(double));
    r->D = (double *)take((size_t)m * 8);
    r->aE = (double *)take((size_t)m * 8);
    r->aN = (double *)take((size_t)m * 8);
    r->S = (double *)take((size_t)N * 8);
    r->p = (double *)take((size_t)N * 8);
    r->r64 = (double *)take((size_t)N * 8);
    r->D32 = (float *)take((size_t)m * 4);
    r->invD32 = (float *)take((size_t)m * 4);
    r->aE32 = (float *)take((size_t)m * 4);
    r->aN32 = (float *)take((size_t)m * 4);
    r->b32 = (float *)take((size_t)N * 4);
    r->x32 = (float *)take((size_t)N * 4);
    r->r32[0] = (float *)take((size_t)N * 4);
    r->r32[1] = (float *)take((size_t)N * 4);
    r->u32[0] = (float *)take((size_t)N * 4);
    r->u32[1] = (float *)take((size_t)N * 4);
    r->z32 = (float *)take((size_t)N * 4);
    r->v32 = (float *)take((size_t)N * 4);
}

static constexpr double kInnerFloor = 5e-7;
static constexpr int kMaxOuter = 12;            // refinements when each restarts the inner solve
static constexpr int kMaxOuterContinued = 200;  // refinements of a continued inner recurrence

// Start (or restart) the inner FP32 solve of a request from its current r64.
// Next inner solve of a request from its FP64 residual (norm rnorm, relative
// true_rel).  As in the joint solve, the inner recurrence continues across
// refinements (its residual replaced by the FP64 one after every reduction by
// the context's reliable_delta) unless the context asks for restarts or the last
// continued solve stalled.
static int start_inner(gmaf_server *sv, Request *r, double true_rel, double rnorm)
{
    cudaStream_t s = sv->stream;
    const bool continued = !sv->ctx->mixed_restart;
    double eps_in = 0.5 * r->in.eps / true_rel;
    const double floor_in = continued ? sv->ctx->reliable_delta : kInnerFloor;
    if (eps_in < floor_in) eps_in = floor_in;
    if (eps_in > 0.5) eps_in = 0.5;
    r->h.eps = eps_in;
    const bool cont = continued && r->outer > 0 && !r->stalled && r->rnorm_prev > 0.0;
    const int left = r->in.max_iter - r->total_inner;
    r->h.max_iter = cont ? r->last_iter + std::min(left, std::max(1000, 4 * r->longest)) : left;
    r->h.guard_limit = sv->ctx->loop_guard;
    cudaError_t e = cudaMemcpyAsync(r->d_desc, &r->h, sizeof(PcgDesc<float>), cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return cuda_status(e);
    k_make_b32<<<r->grid_s, kThreads, 0, s>>>(r->r64, r->b32, r->N, r->sc_out);
    if (cont)
        k_continue<<<1, 32, 0, s>>>(r->sc_in, r->rnorm_prev / rnorm);
    else
        k_reset<<<1, 32, 0, s>>>(r->sc_in, 0);
    r->cont_run = cont;
    r->rnorm_prev = rnorm;
    k_init_r<float><<<r->grid_s, kThreads, 0, s>>>(r->d_desc);
    const int gb = (int)std::min<long long>((r->ntasks + kWarps - 1) / kWarps, (long long)sv->num_sms * kSvMinB);
    k_phase_b<float, kSvVec, kSvTY, kSvMinB, true, 0><<<gb, kThreads, 0, s>>>(r->d_desc);
    r->outer += 1;
    sv->dirty = true;
    return cuda_status(cudaGetLastError());
}

// Admission work: fan-out, assembly, FP32 copies, FP64 residual of p = 0, and
// the first inner solve's initial pass.  Synchronises to read the residual.
static int admit(gmaf_server *sv, Request *r)
{
    cudaStream_t s = sv->stream;
    carve(sv, r);
    const int cslot[9] = {0, 1, 2, 3, 4, 0, 0, 0, 0};
    double base[8];
    std::memcpy(base, r->in.state.e, 4 * sizeof(double));
    std::memcpy(base + 4, r->in.state.edot, 4 * sizeof(double));
    char *hdr = sv->base + r->off;
    cudaError_t e = cudaMemsetAsync(hdr, 0, kHdrBytes, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(r->cslot, cslot, sizeof cslot, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(r->p, 0, (size_t)r->N * sizeof(double), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(r->x32, 0, (size_t)r->N * sizeof(float), s);
    if (e != cudaSuccess) return cuda_status(e);
    int st;
    if ((st = launch_fanout(base, r->in.d_e, r->in.d_edot, r->conds, r->cslot_w, s))) return st;
    if ((st = launch_trig(r->g, r->trig, s))) return st;
    if ((st = launch_assemble(r->g, 9, r->conds, r->cslot_w, r->D, r->aE, r->aN, r->S, r->trig,
                              r->flags, 5, s)))
        return st;
    const long long m = 5 * r->n;
    k_to_f32<<<stream_grid_s(m, sv->num_sms), kThreads, 0, s>>>(r->D, r->aE, r->aN, r->D32, r->invD32,
                                                               r->aE32, r->aN32, m, r->sc_out,
                                                               r->in.omega);
    // inner solve descriptor
    PcgDesc<float> &h = r->h;
    h = PcgDesc<float>{};
    h.nth = r->g.nth;
    h.nz = r->g.nz;
    h.K = 9;
    h.n = r->n;
    h.tiles_x = (r->g.nth + kSvW - 1) / kSvW;
    h.tiles_y = (r->g.nz + r->ty - 1) / r->ty;
    h.ntiles = r->ntasks;
    h.ty = r->ty;
    h.precond = 1;
    h.zero_init = 1;
    h.use_cond = 0;
    h.D = r->D32;
    h.invD = r->invD32;
    h.aE = r->aE32;
    h.aN = r->aN32;
    h.cslot = r->cslot;
    h.b = r->b32;
    h.p = r->x32;
    h.z = r->z32;
    h.v = r->v32;
    h.u[0] = r->u32[0];
    h.u[1] = r->u32[1];
    h.r[0] = r->r32[0];
    h.r[1] = r->r32[1];
    h.omega = (float)r->in.omega;
    h.sc = r->sc_in;
    h.partials = r->part;
    // FP64 residual descriptor
    ResidDesc &rd = r->rd;
    rd = ResidDesc{};
    rd.nth = r->g.nth;
    rd.nz = r->g.nz;
    rd.K = 9;
    rd.n = r->n;
    rd.D = r->D;
    rd.aE = r->aE;
    rd.aN = r->aN;
    rd.cslot = r->cslot;
    rd.S = r->S;
    rd.p = r->p;
    rd.r = r->r64;
    rd.sc = r->sc_out;
    rd.partials = r->part;
    e = cudaMemcpyAsync(r->d_rdesc, &rd, sizeof(ResidDesc), cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return cuda_status(e);
    k_resid64<<<r->grid_s, kThreads, 0, s>>>(r->d_rdesc);
    Scalars ho;
    e = cudaMemcpyAsync(&ho, r->sc_out, sizeof(Scalars), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_status(e);
    r->outer = 0;
    r->total_inner = 0;
    r->rnorm_prev = 0.0;
    r->last_iter = r->longest = 0;
    r->cont_run = r->stalled = r->no_progress = false;
    r->rel0 = ho.true_rel;
    r->rnorm0 = ho.rnorm;
    if (ho.normS == 0.0 || !std::isfinite(ho.true_rel) || ho.true_rel <= r->in.eps) return 1;
    return start_inner(sv, r, ho.true_rel, ho.rnorm);
}

// Loads of the 9 conditions, Jacobian and update; result to the host.
static int retire(gmaf_server *sv, Request *r, int status, double true_rel)
{
    cudaStream_t s = sv->stream;
    int st;
    if ((st = launch_loads(r->g, 9, r->conds, r->p, r->trig, r->part, r->tickets, r->loads, r->flags,
                           sv->num_sms, s)))
        return st;
    PicardIn in{};
    std::memcpy(in.base, r->in.state.e, 4 * sizeof(double));
    std::memcpy(in.base + 4, r->in.state.edot, 4 * sizeof(double));
    std::memcpy(in.e_prev, r->in.e_prev, 4 * sizeof(double));
    std::memcpy(in.F_ext, r->in.F_ext, 4 * sizeof(double));
    if ((st = launch_picard_update(r->loads, in, r->in.dt, r->in.d_e, r->in.d_edot, r->g.L, r->result, s)))
        return st;
    double res[kResultDoubles];
    int flag = 0;
    cudaError_t e = cudaMemcpyAsync(res, r->result, sizeof res, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&flag, r->flags, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_status(e);
    gmaf_result out{};
    out.id = r->id;
    out.iterations = r->total_inner;
    out.outer_iterations = r->outer;
    out.true_rel_residual = true_rel;
    out.tile_rows = r->ty;
    std::memcpy(out.loads, res, 12 * sizeof(double));
    std::memcpy(out.J, res + 12, 48 * sizeof(double));
    std::memcpy(out.G, res + 60, 4 * sizeof(double));
    out.state = r->in.state;
    if (flag & 1) {
        out.status = GMAF_CONTACT;
    } else if (status != GMAF_OK) {
        out.status = status;
    } else if (res[72] != 0.0) {
        out.status = GMAF_NONFINITE;
    } else {
        out.status = GMAF_OK;
        std::memcpy(out.state.e, res + 64, 4 * sizeof(double));
        std::memcpy(out.state.edot, res + 68, 4 * sizeof(double));
    }
    sv->finished.push_back(out);
    sv->arena.release(r->off, r->bytes);
    delete r;
    return GMAF_OK;
}

// Rebuild the batched-launch table after the active set or a descriptor changed.
// Grow a device buffer to at least `need` bytes, zero-filled when (re)allocated;
// the stream is synchronised before the old buffer is freed.
static int grow_zeroed(gmaf_server *sv, void **buf, size_t *cap, size_t need)
{
    if (need <= *cap) return GMAF_OK;
    cudaError_t e = cudaStreamSynchronize(sv->stream);
    if (e != cudaSuccess) return cuda_status(e);
    if (*buf) cudaFree(*buf);
    *buf = nullptr;
    *cap = 0;
    if (cudaMalloc(buf, need) != cudaSuccess) {
        cudaGetLastError();
        *buf = nullptr;
        return GMAF_OUT_OF_MEMORY;
    }
    e = cudaMemsetAsync(*buf, 0, need, sv->stream);
    if (e != cudaSuccess) return cuda_status(e);
    *cap = need;
    return GMAF_OK;
}

// Grow the partial-sum buffer of the batched launches (no zeroing needed: every
// task writes its own entries before they are read).
static int grow_partials(gmaf_server *sv, size_t need)
{
    if (need <= sv->mpart_cap) return GMAF_OK;
    cudaError_t e = cudaStreamSynchronize(sv->stream);
    if (e != cudaSuccess) return cuda_status(e);
    if (sv->mpart) cudaFree(sv->mpart);
    sv->mpart = nullptr;
    sv->mpart_cap = 0;
    if (cudaMalloc(&sv->mpart, need) != cudaSuccess) {
        cudaGetLastError();
        sv->mpart = nullptr;
        return GMAF_OUT_OF_MEMORY;
    }
    sv->mpart_cap = need;
    return GMAF_OK;
}

static int batched_grid(gmaf_server *sv, long long tasks)
{
    int per_sm = 0, per_sm_a = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, sv->kern.b, kThreads, sv->kern.smem_b) !=
            cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_a, sv->kern.a, kThreads, sv->kern.smem_a) !=
            cudaSuccess) {
        cudaGetLastError();
        per_sm = per_sm_a = 1;
    }
    per_sm = std::max(1, std::min(per_sm, per_sm_a));
    long long gm = (tasks + kWarps - 1) / kWarps;
    if (gm > (long long)per_sm * sv->num_sms) gm = (long long)per_sm * sv->num_sms;
    if (gm < 1) gm = 1;
    return (int)gm;
}

static int rebuild_table(gmaf_server *sv)
{
    MultiDesc<float> &hm = sv->hm;
    hm.ngroups = (int)sv->active.size();
    unsigned acc = 0;
    std::vector<PcgDesc<float>> groups(sv->active.size());
    for (size_t g = 0; g < sv->active.size(); ++g) {
        hm.task_off[g] = acc;
        acc += (unsigned)sv->active[g]->ntasks;
        groups[g] = sv->active[g]->h;
    }
    hm.task_off[hm.ngroups] = acc;
    hm.total_tasks = acc;
    hm.groups = sv->d_groups;
    hm.msc = sv->msc;
    int pst = grow_partials(sv, (size_t)2 * (acc ? acc : 1) * sizeof(double));
    if (pst != GMAF_OK) return pst;
    hm.partials = sv->mpart;
    // two-level reduction: chunks of kChunk tasks, counted per group
    unsigned cacc = 0;
    for (size_t g = 0; g < sv->active.size(); ++g) {
        hm.chunk_off[g] = cacc;
        cacc += (unsigned)((sv->active[g]->ntasks + kChunk - 1) / kChunk);
    }
    hm.chunk_off[hm.ngroups] = cacc;
    int gst = grow_zeroed(sv, (void **)&sv->mchunk, &sv->mchunk_cap,
                          (size_t)2 * (cacc ? cacc : 1) * sizeof(double));
    if (gst == GMAF_OK)
        gst = grow_zeroed(sv, (void **)&sv->mctr, &sv->mctr_cap, (size_t)(kMaxGroups + cacc) * sizeof(unsigned));
    if (gst != GMAF_OK) return gst;
    hm.chunk_sum = sv->mchunk;
    hm.group_ctr = sv->mctr;
    hm.chunk_ctr = sv->mctr + kMaxGroups;
    cudaError_t e = cudaSuccess;
    if (!groups.empty())
        e = cudaMemcpyAsync(sv->d_groups, groups.data(), groups.size() * sizeof(PcgDesc<float>),
                            cudaMemcpyHostToDevice, sv->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(sv->d_mdesc, &hm, sizeof(MultiDesc<float>), cudaMemcpyHostToDevice, sv->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(&sv->msc->done, 0, sizeof(int), sv->stream);
    if (e != cudaSuccess) return cuda_status(e);
    sv->grid_m = batched_grid(sv, acc);
    sv->dirty = false;
    return GMAF_OK;
}

// Tuner: the time of `reps` batched iterations (phase A + phase B) of request r
// alone, decomposed into tasks of `ty` rows, on its own data (its inner solve
// has just been started).  The timed copy of its descriptor never converges;
// the caller restarts the inner solve afterwards.
static int time_alone(gmaf_server *sv, Request *r, int ty, int reps, float *ms_out)
{
    cudaStream_t s = sv->stream;
    PcgDesc<float> hh = r->h;
    hh.ty = ty;
    hh.tiles_y = (r->g.nz + ty - 1) / ty;
    hh.ntiles = sv_tasks(r->g.nth, r->g.nz, ty);
    hh.eps = 1e-300;
    hh.max_iter = 1 << 30;
    hh.guard_limit = 0;
    const unsigned nt = (unsigned)hh.ntiles;
    const unsigned nch = (nt + kChunk - 1) / kChunk;
    int st = grow_partials(sv, (size_t)2 * nt * sizeof(double));
    if (st == GMAF_OK)
        st = grow_zeroed(sv, (void **)&sv->mchunk, &sv->mchunk_cap, (size_t)2 * nch * sizeof(double));
    if (st == GMAF_OK)
        st = grow_zeroed(sv, (void **)&sv->mctr, &sv->mctr_cap, (size_t)(kMaxGroups + nch) * sizeof(unsigned));
    if (st != GMAF_OK) return st;
    sv->dirty = true;                 // the batched table must pick up regrown buffers
    MultiDesc<float> tm{};
    tm.ngroups = 1;
    tm.total_tasks = nt;
    tm.task_off[0] = 0;
    tm.task_off[1] = nt;
    tm.groups = sv->d_tune_group;
    tm.msc = sv->msc;
    tm.partials = sv->mpart;
    tm.chunk_off[0] = 0;
    tm.chunk_off[1] = nch;
    tm.chunk_sum = sv->mchunk;
    tm.group_ctr = sv->mctr;
    tm.chunk_ctr = sv->mctr + kMaxGroups;
    cudaError_t e = cudaMemcpyAsync(sv->d_tune_group, &hh, sizeof hh, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(sv->d_tune_mdesc, &tm, sizeof tm, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(&sv->msc->done, 0, sizeof(int), s);
    if (e != cudaSuccess) return cuda_status(e);
    const int grid = batched_grid(sv, nt);
    void *args[] = {(void *)&sv->d_tune_mdesc};
    const int warm = 2;
    for (int q = 0; q < warm + reps && e == cudaSuccess; ++q) {
        if (q == warm) e = cudaEventRecord(sv->ev[0], s);
        if (e == cudaSuccess)
            e = cudaLaunchKernel(sv->kern.a, dim3(grid), dim3(kThreads), args, sv->kern.smem_a, s);
        if (e == cudaSuccess)
            e = cudaLaunchKernel(sv->kern.b, dim3(grid), dim3(kThreads), args, sv->kern.smem_b, s);
    }
    if (e == cudaSuccess) e = cudaEventRecord(sv->ev[1], s);
    if (e == cudaSuccess) e = cudaEventSynchronize(sv->ev[1]);
    if (e == cudaSuccess) e = cudaEventElapsedTime(ms_out, sv->ev[0], sv->ev[1]);
    return cuda_status(e);
}

// Task height of r's grid: the process-wide decision for the grid, or (the first
// request of the grid) the fastest candidate timed on r alone, in two
// round-robin passes taking the best time of each; a later candidate replaces
// the default only when it is more than 3% faster.  r's inner solve is
// restarted when the tuner ran.
static int tune_request(gmaf_server *sv, Request *r)
{
    int ty = sv_tuned_rows(sv->device, r->g.nth, r->g.nz, sv->staged);
    if (ty == 0) {
        float best[3] = {3e38f, 3e38f, 3e38f};
        int tiles[3];
        const int nc = (int)(sizeof kSvTyCand / sizeof kSvTyCand[0]);
        for (int round = 0; round < 2; ++round) {
            for (int c = 0; c < nc; ++c) {
                tiles[c] = (r->g.nz + kSvTyCand[c] - 1) / kSvTyCand[c];
                bool dup = false;                      // same decomposition as an earlier one
                for (int q = 0; q < c; ++q) dup = dup || tiles[q] == tiles[c];
                if (dup) continue;
                float ms = 0.0f;
                const int st = time_alone(sv, r, kSvTyCand[c], 5, &ms);
                if (st != GMAF_OK) return st;
                best[c] = std::min(best[c], ms);
            }
        }
        int pick = 0;
        for (int c = 1; c < nc; ++c)
            if (best[c] < 0.97f * best[pick]) pick = c;
        ty = sv_record_rows(sv->device, r->g.nth, r->g.nz, sv->staged, kSvTyCand[pick]);
        // restart the inner solve that the timing runs advanced
        r->ty = ty;
        r->ntasks = sv_tasks(r->g.nth, r->g.nz, ty);
        r->h.ty = ty;
        r->h.tiles_y = (r->g.nz + ty - 1) / ty;
        r->h.ntiles = r->ntasks;
        r->outer = 0;
        r->rnorm_prev = 0.0;
        return start_inner(sv, r, r->rel0, r->rnorm0);
    }
    return GMAF_OK;
}

// The round graph: `iterations` phase pairs on the batched table.  Rebuilt when
// the round length or the kernels change; when only the launch grid changed
// (the active set grew or shrank) its kernel nodes are updated in place.
static void destroy_round_graph(gmaf_server *sv)
{
    if (sv->graph_exec) cudaGraphExecDestroy(sv->graph_exec);
    if (sv->graph) cudaGraphDestroy(sv->graph);
    sv->graph_exec = nullptr;
    sv->graph = nullptr;
    sv->graph_nodes.clear();
    sv->graph_iters = 0;
}

static int round_graph(gmaf_server *sv, int iterations)
{
    void *args[] = {(void *)&sv->d_mdesc};
    cudaKernelNodeParams kp{};
    kp.blockDim = dim3(kThreads);
    kp.gridDim = dim3(sv->grid_m);
    kp.kernelParams = args;
    if (sv->graph_exec && sv->graph_iters == iterations && sv->graph_a == sv->kern.a &&
        sv->graph_b == sv->kern.b) {
        if (sv->graph_grid == sv->grid_m) return GMAF_OK;
        cudaError_t e = cudaSuccess;
        for (size_t q = 0; q < sv->graph_nodes.size() && e == cudaSuccess; ++q) {
            const bool a = (q & 1) == 0;
            kp.func = (void *)(a ? sv->kern.a : sv->kern.b);
            kp.sharedMemBytes = (unsigned)(a ? sv->kern.smem_a : sv->kern.smem_b);
            e = cudaGraphExecKernelNodeSetParams(sv->graph_exec, sv->graph_nodes[q], &kp);
        }
        if (e == cudaSuccess) {
            sv->graph_grid = sv->grid_m;
            return GMAF_OK;
        }
        cudaGetLastError();               // fall through: rebuild
    }
    destroy_round_graph(sv);
    cudaError_t e = cudaGraphCreate(&sv->graph, 0);
    cudaGraphNode_t prev = nullptr;
    for (int q = 0; q < 2 * iterations && e == cudaSuccess; ++q) {
        const bool a = (q & 1) == 0;
        kp.func = (void *)(a ? sv->kern.a : sv->kern.b);
        kp.sharedMemBytes = (unsigned)(a ? sv->kern.smem_a : sv->kern.smem_b);
        cudaGraphNode_t node = nullptr;
        e = cudaGraphAddKernelNode(&node, sv->graph, prev ? &prev : nullptr, prev ? 1 : 0, &kp);
        if (e == cudaSuccess) sv->graph_nodes.push_back(node);
        prev = node;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&sv->graph_exec, sv->graph, 0);
    if (e != cudaSuccess) {
        destroy_round_graph(sv);
        return cuda_status(e);
    }
    sv->graph_iters = iterations;
    sv->graph_grid = sv->grid_m;
    sv->graph_a = sv->kern.a;
    sv->graph_b = sv->kern.b;
    return GMAF_OK;
}

// Groups whose inner run ended: refinement step, then restart or retire.
static int harvest(gmaf_server *sv)
{
    cudaStream_t s = sv->stream;
    const size_t na = sv->active.size();
    if (na == 0) return GMAF_OK;
    std::vector<Scalars> hs(na);
    for (size_t g = 0; g < na; ++g) {
        cudaError_t e = cudaMemcpyAsync(&hs[g], sv->active[g]->sc_in, sizeof(Scalars),
                                        cudaMemcpyDeviceToHost, s);
        if (e != cudaSuccess) return cuda_status(e);
    }
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_status(e);
    std::vector<size_t> ended;
    for (size_t g = 0; g < na; ++g) {
        if (!hs[g].done) continue;
        Request *r = sv->active[g];
        k_finalize<float><<<r->grid_s, kThreads, 0, s>>>(r->d_desc);
        k_update_p64<<<r->grid_s, kThreads, 0, s>>>(r->p, r->x32, r->N, r->sc_out);
        k_resid64<<<r->grid_s, kThreads, 0, s>>>(r->d_rdesc);
        const int seg = r->cont_run ? hs[g].iter - r->last_iter : hs[g].iter;
        r->last_iter = hs[g].iter;
        r->total_inner += seg;
        r->longest = std::max(r->longest, seg);
        r->stalled = !sv->ctx->mixed_restart && !hs[g].converged;
        r->no_progress = seg == 0;
        ended.push_back(g);
    }
    if (ended.empty()) return GMAF_OK;
    std::vector<Scalars> ho(ended.size());
    for (size_t q = 0; q < ended.size(); ++q) {
        e = cudaMemcpyAsync(&ho[q], sv->active[ended[q]]->sc_out, sizeof(Scalars),
                            cudaMemcpyDeviceToHost, s);
        if (e != cudaSuccess) return cuda_status(e);
    }
    e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_status(e);
    std::vector<Request *> keep;
    size_t q = 0;
    for (size_t g = 0; g < na; ++g) {
        Request *r = sv->active[g];
        if (q < ended.size() && ended[q] == g) {
            const Scalars &o = ho[q];
            const Scalars &in = hs[g];
            ++q;
            int status = GMAF_OK;
            bool finish = false;
            if (in.status != 0 || o.status != 0 || !std::isfinite(o.true_rel)) {
                status = in.status != 0 ? in.status : GMAF_NONFINITE;
                finish = true;
            } else if (o.normS == 0.0 || o.true_rel <= r->in.eps) {
                finish = true;
            } else if (r->outer >= (sv->ctx->mixed_restart ? kMaxOuter : kMaxOuterContinued) ||
                       r->total_inner >= r->in.max_iter || r->no_progress) {
                status = GMAF_NOT_CONVERGED;
                finish = true;
            }
            if (finish) {
                int st = retire(sv, r, status, o.true_rel);
                if (st != GMAF_OK) return st;
                sv->dirty = true;
                continue;
            }
            int st = start_inner(sv, r, o.true_rel, o.rnorm);
            if (st != GMAF_OK) return st;
        }
        keep.push_back(r);
    }
    sv->active.swap(keep);
    return GMAF_OK;
}

}  // namespace gmaf

extern "C" {

int gmaf_request_footprint(const gmaf_grid *grid, size_t *bytes_out)
{
    if (!grid || !bytes_out || grid->n_theta < 3 || grid->n_z < 2) return GMAF_INVALID_ARG;
    int dev = 0, sms = 152;
    if (cudaGetDevice(&dev) == cudaSuccess)
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    else
        cudaGetLastError();
    *bytes_out = footprint(grid->n_theta, grid->n_z, sms);
    return GMAF_OK;
}

int gmaf_server_create(gmaf_ctx *ctx, size_t hbm_budget_bytes, gmaf_server **out)
{
    if (!ctx || !out || hbm_budget_bytes < (1u << 20)) return GMAF_INVALID_ARG;
    *out = nullptr;
    gmaf_server *sv = new (std::nothrow) gmaf_server();
    if (!sv) return GMAF_OUT_OF_MEMORY;
    sv->ctx = ctx;
    sv->stream = ctx->stream;
    sv->num_sms = ctx->num_sms;
    sv->budget = Arena::round_up(hbm_budget_bytes) - 256;
    sv->next_id = 1;
    sv->base = nullptr;
    sv->d_mdesc = nullptr;
    sv->d_groups = nullptr;
    sv->msc = nullptr;
    sv->mpart = nullptr;
    sv->mpart_cap = 0;
    sv->mchunk = nullptr;
    sv->mchunk_cap = 0;
    sv->mctr = nullptr;
    sv->mctr_cap = 0;
    sv->dirty = true;
    sv->hm = MultiDesc<float>{};
    sv->grid_m = 1;
    sv->device = ctx->device;
    const char *stg = std::getenv("GMAF_SV_STAGED");
    sv->staged = (stg && std::atoi(stg) == 0) ? 0 : 1;
    sv->kern = sv_kernels(sv->staged != 0);
    const char *tn = std::getenv("GMAF_SV_TUNE");
    sv->tune = (tn && std::atoi(tn) == 0) ? 0 : 1;
    const char *gr = std::getenv("GMAF_SV_GRAPH");
    sv->use_graph = (gr && std::atoi(gr) == 0) ? 0 : 1;
    sv->d_tune_group = nullptr;
    sv->d_tune_mdesc = nullptr;
    sv->ev[0] = sv->ev[1] = nullptr;
    sv->graph = nullptr;
    sv->graph_exec = nullptr;
    sv->graph_grid = sv->graph_iters = 0;
    sv->graph_a = sv->graph_b = nullptr;
    cudaError_t e = cudaMalloc(&sv->base, sv->budget);
    if (e == cudaSuccess) e = cudaMalloc(&sv->d_mdesc, sizeof(MultiDesc<float>));
    if (e == cudaSuccess) e = cudaMalloc(&sv->d_groups, kMaxGroups * sizeof(PcgDesc<float>));
    if (e == cudaSuccess) e = cudaMalloc(&sv->msc, sizeof(Scalars));
    if (e == cudaSuccess) e = cudaMalloc(&sv->d_tune_group, sizeof(PcgDesc<float>));
    if (e == cudaSuccess) e = cudaMalloc(&sv->d_tune_mdesc, sizeof(MultiDesc<float>));
    if (e == cudaSuccess) e = cudaEventCreate(&sv->ev[0]);
    if (e == cudaSuccess) e = cudaEventCreate(&sv->ev[1]);
    if (e == cudaSuccess) e = cudaMemsetAsync(sv->msc, 0, sizeof(Scalars), sv->stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        if (sv->base) cudaFree(sv->base);
        if (sv->d_mdesc) cudaFree(sv->d_mdesc);
        if (sv->d_groups) cudaFree(sv->d_groups);
        if (sv->msc) cudaFree(sv->msc);
        if (sv->d_tune_group) cudaFree(sv->d_tune_group);
        if (sv->d_tune_mdesc) cudaFree(sv->d_tune_mdesc);
        for (cudaEvent_t ev : sv->ev)
            if (ev) cudaEventDestroy(ev);
        delete sv;
        return GMAF_OUT_OF_MEMORY;
    }
    sv->arena.reset(sv->budget);
    *out = sv;
    return GMAF_OK;
}

int gmaf_server_destroy(gmaf_server *sv)
{
    if (!sv) return GMAF_INVALID_ARG;
    cudaError_t e = cudaStreamSynchronize(sv->stream);
    for (Request *r : sv->active) delete r;
    for (Request *r : sv->queue) delete r;
    cudaFree(sv->base);
    cudaFree(sv->d_mdesc);
    cudaFree(sv->d_groups);
    cudaFree(sv->msc);
    cudaFree(sv->d_tune_group);
    cudaFree(sv->d_tune_mdesc);
    for (cudaEvent_t ev : sv->ev) cudaEventDestroy(ev);
    destroy_round_graph(sv);
    if (sv->mpart) cudaFree(sv->mpart);
    if (sv->mchunk) cudaFree(sv->mchunk);
    if (sv->mctr) cudaFree(sv->mctr);
    delete sv;
    return e == cudaSuccess ? GMAF_OK : GMAF_CUDA_ERROR;
}

int gmaf_server_submit(gmaf_server *sv, const gmaf_request *req, int64_t *id_out)
{
    if (!sv || !req) return GMAF_INVALID_ARG;
    if (!geom_valid(&req->grid, &req->phys, &req->tex)) return GMAF_INVALID_ARG;
    if (req->grid.n_theta % kSvVec != 0) return GMAF_INVALID_ARG;
    if (!(req->omega > 0.0 && req->omega < 2.0) || !(req->eps > 0.0) || req->max_iter < 1 ||
        req->d_e == 0.0 || req->d_edot == 0.0 || !std::isfinite(req->dt))
        return GMAF_INVALID_ARG;
    const size_t bytes = footprint(req->grid.n_theta, req->grid.n_z, sv->num_sms);
    if (bytes > sv->budget) return GMAF_OUT_OF_MEMORY;
    Request *r = new (std::nothrow) Request();
    if (!r) return GMAF_OUT_OF_MEMORY;
    r->id = sv->next_id++;
    r->in = *req;
    r->g = make_geom(&req->grid, &req->phys, &req->tex);
    r->n = (long long)req->grid.n_theta * req->grid.n_z;
    r->N = 9 * r->n;
    r->ty = kSvTY;                     // the tuned height is looked up at admission
    r->ntasks = sv_tasks(req->grid.n_theta, req->grid.n_z, r->ty);
    r->grid_s = stream_grid_s(r->N, sv->num_sms);
    r->bytes = bytes;
    sv->queue.push_back(r);
    if (id_out) *id_out = r->id;
    return GMAF_OK;
}

int gmaf_server_run(gmaf_server *sv, int32_t iterations, int32_t *active_out, int32_t *queued_out)
{
    if (!sv || iterations < 0) return GMAF_INVALID_ARG;
    int st;
    // admission, first-come first-served while the footprint fits
    while (!sv->queue.empty() && sv->active.size() < (size_t)kMaxGroups) {
        Request *r = sv->queue.front();
        size_t off = 0;
        if (!sv->arena.alloc(r->bytes, &off)) break;
        sv->queue.pop_front();
        r->off = off;
        // the grid's tuned task height, when decided; else the default until tuned
        const int known = sv_tuned_rows(sv->device, r->g.nth, r->g.nz, sv->staged);
        r->ty = known ? known : kSvTY;
        r->ntasks = sv_tasks(r->g.nth, r->g.nz, r->ty);
        st = admit(sv, r);
        if (st == GMAF_OK && sv->tune && !known) st = tune_request(sv, r);
        if (st == 1) {                        // nothing to solve: retire at once
            st = retire(sv, r, GMAF_OK, 0.0);
            if (st != GMAF_OK) return st;
            continue;
        }
        if (st != GMAF_OK) {
            sv->arena.release(r->off, r->bytes);
            delete r;
            return st;
        }
        sv->active.push_back(r);
        sv->dirty = true;
    }
    if (!sv->active.empty() && iterations > 0) {
        if (sv->dirty && (st = rebuild_table(sv))) return st;
        cudaError_t e0 = cudaMemsetAsync(&sv->msc->done, 0, sizeof(int), sv->stream);
        if (e0 != cudaSuccess) return cuda_status(e0);
        cudaError_t e = cudaSuccess;
        if (sv->use_graph) {
            if ((st = round_graph(sv, iterations))) return st;
            e = cudaGraphLaunch(sv->graph_exec, sv->stream);
        } else {
            void *args[] = {(void *)&sv->d_mdesc};
            for (int it = 0; it < iterations && e == cudaSuccess; ++it) {
                e = cudaLaunchKernel(sv->kern.a, dim3(sv->grid_m), dim3(kThreads), args, sv->kern.smem_a,
                                     sv->stream);
                if (e == cudaSuccess)
                    e = cudaLaunchKernel(sv->kern.b, dim3(sv->grid_m), dim3(kThreads), args,
                                         sv->kern.smem_b, sv->stream);
            }
        }
        if (e == cudaSuccess) e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_status(e);
    }
    if ((st = harvest(sv))) return st;
    if (active_out) *active_out = (int32_t)sv->active.size();
    if (queued_out) *queued_out = (int32_t)sv->queue.size();
    return GMAF_OK;
}

int gmaf_server_poll(gmaf_server *sv, gmaf_result *out, int32_t max_results, int32_t *n_out)
{
    if (!sv || !n_out || max_results < 0 || (max_results > 0 && !out)) return GMAF_INVALID_ARG;
    const int32_t n = (int32_t)std::min<size_t>((size_t)max_results, sv->finished.size());
    for (int32_t i = 0; i < n; ++i) out[i] = sv->finished[i];
    sv->finished.erase(sv->finished.begin(), sv->finished.begin() + n);
    *n_out = n;
    return GMAF_OK;
}

int gmaf_server_free_bytes(const gmaf_server *sv, size_t *bytes_out)
{
    if (!sv || !bytes_out) return GMAF_INVALID_ARG;
    *bytes_out = sv->arena.free_bytes();
    return GMAF_OK;
}

int gmaf_server_cancel(gmaf_server *sv, int64_t id)
{
    if (!sv) return GMAF_INVALID_ARG;
    Request *r = nullptr;
    for (auto it = sv->queue.begin(); it != sv->queue.end(); ++it) {
        if ((*it)->id == id) {
            r = *it;
            sv->queue.erase(it);
            break;
        }
    }
    if (!r) {
        for (auto it = sv->active.begin(); it != sv->active.end(); ++it) {
            if ((*it)->id == id) {
                r = *it;
                // work already issued for it (the next inner solve's set-up) may still
                // be running on its block: let it finish before the block is reused
                cudaError_t e = cudaStreamSynchronize(sv->stream);
                if (e != cudaSuccess) return cuda_status(e);
                sv->active.erase(it);
                sv->arena.release(r->off, r->bytes);
                sv->dirty = true;
                break;
            }
        }
    }
    if (!r) return GMAF_INVALID_ARG;
    gmaf_result out{};
    out.id = r->id;
    out.status = GMAF_CANCELLED;
    out.tile_rows = r->ty;
    out.iterations = r->total_inner;
    out.outer_iterations = r->outer;
    out.state = r->in.state;
    sv->finished.push_back(out);
    delete r;
    return GMAF_OK;
}

}  // extern "C"
