// Internal declarations of the GB300 piston-gap library (not part of the ABI).
#pragma once

#include <cuda_runtime.h>

#include <atomic>
#include <cstddef>
#include <cstdint>

#include "gmaf.h"

namespace gmaf {

constexpr double kPi = 3.14159265358979323846;
constexpr int kMaxCond = 64;       // conditions in one joint system
constexpr int kThreads = 256;      // threads per block of the stencil kernels

// ---------------------------------------------------------------- geometry

// Hexagonal lattice of flat-bottom circular dimples (h_Text of Eq. 2.3).
struct Lattice {
    int on;
    double r, depth, oth, oz;
    double ath, az;   // column pitch around the piston, row pitch along z
};

struct Geom {
    int nth, nz;
    double Rk, L, c, mu, v, pch, pcase;
    double dth, dx, dz, invL;
    Lattice lt;
};

Lattice make_lattice(const gmaf_texture *tex, double Rk);
Geom make_geom(const gmaf_grid *g, const gmaf_physics *ph, const gmaf_texture *tex);

// ---------------------------------------------------------------- solver state

// Scalars of one joint PCG run, resident on the device.
struct Scalars {
    double alpha, beta, d;
    double normS, rel, true_rel;
    double scale;           // mixed precision: FP32 matrix = scale * A
    double rnorm;           // mixed precision: norm of the FP64 outer residual
    int iter, first, done, converged, status, guard, zero_rhs;
    int pending;            // alpha u terms not yet added to p (0, 1 or 2)
    int max_iter;
    int cont;               // mixed precision: the next initial pass continues the recurrence
    double cscale;          //   (reliable update) with the old direction rescaled by cscale
    double alpha_pp;        // alpha of the older of two pending p updates (pending == 2)
    unsigned int ticket[6];
    unsigned int task_ctr[2];   // next task of phase A / phase B
};

enum Ticket { kTicketA = 0, kTicketB = 1, kTicketInit = 2, kTicketResid = 3, kTicketMisc = 4 };

template <typename T>
struct PcgDesc {
    int nth, nz, K, tiles_x, tiles_y, precond, zero_init, use_cond;
    long long n, ntiles;
    long long sgroups;             // row groups of the static schedule
    const T *D, *invD, *aE, *aN;   // coefficient slots, [slot][n]; invD holds omega / D for
                                   // ASSOR-II, 1 / D for Jacobi, the ASSOR-I diagonal for it
    const int *cslot;              // coefficient slot of each condition, [K]
    const T *b;                    // right-hand side, [K][n]
    T *p, *z, *v;
    T *u[2], *r[2];
    T omega;                       // ASSOR relaxation factor
    double eps;
    int max_iter;
    int guard_limit;               // phase-A bodies allowed before GMAF_TIMEOUT (0: max_iter + 4)
    int ty;                        // rows per task of the batched kernels (0: their template TY)
    cudaGraphConditionalHandle cond;
    Scalars *sc;
    double *partials;              // per-task (or per-warp) sums [ntiles][2], or per-block [2][grid]
    double *chunk_sum;             // two-level reduction: chunk sums [chunks][2] (nullptr: one level)
    unsigned *chunk_ctr;           // per-chunk counters, zero between launches
    // block-marched phase B with TMA tiles (FP32): coefficient slots, task height and tasks
    int nslots;                    // coefficient slots (planes of the coefficient maps)
    const T *dbnd;                 // phase A with the rebuilt diagonal: the Dirichlet term of
                                   // the first and last rows, [slots][2][n_theta] (or null)
    int ty_b;                      // rows per task of that phase B
    long long ntiles_b;            // its tasks
};

// FP64 residual r = S - A p over all conditions, with ||r||^2 and ||S||^2.
struct ResidDesc {
    int nth, nz, K;
    long long n;
    const double *D, *aE, *aN;
    const int *cslot;
    const double *S, *p;
    double *r;                     // written (may be null)
    Scalars *sc;
    double *partials;
};

// ---------------------------------------------------------------- context

enum BufId {
    B_TRIG, B_FLAGS, B_CONDS, B_CSLOT, B_SCAL, B_PART, B_DESC, B_LOADPART, B_LOADS, B_RESULT,
    // FP64 coefficient slots / fields owned by the Picard step
    B_PD, B_PAE, B_PAN, B_PS, B_PP,
    // FP64 PCG workspace
    B_INVD, B_R0, B_R1, B_U0, B_U1, B_Z, B_V,
    // mixed-precision workspace
    B_D32, B_INVD32, B_AE32, B_AN32, B_B32, B_X32, B_R032, B_R132, B_U032, B_U132, B_Z32, B_V32,
    B_R64,
    // asynchronized criterion: per-condition descriptors
    B_ASYNC,
    // two-level reduction of the phase kernels: chunk sums, chunk counters
    B_CHUNK, B_CHUNKCTR,
    // boundary rows' Dirichlet term of the FP32 diagonal (phase A with the rebuilt diagonal)
    B_DBND32,
    B_COUNT
};

struct GraphCache {
    cudaGraphExec_t exec = nullptr;
    cudaGraphConditionalHandle handle = 0;
    int grid_a = 0, grid_b = 0, grid_s = 0;
    const void *desc = nullptr;
    const void *ka = nullptr;      // phase kernels the graph was built with
    const void *kb = nullptr;
    int pairs = 0;                 // A -> B pairs per trip of the WHILE body
    unsigned long long tma[12 * 16];   // tensor maps the phase-B nodes were given (or zero)
};

// Autotuner decision for one solve shape.
struct TuneEntry {
    int tsize, nth, nz, K, precond, vec_ok;
    int choice;
};
constexpr int kTuneEntries = 32;

}  // namespace gmaf

struct gmaf_ctx {
    int device;
    cudaStream_t stream;
    size_t budget;
    size_t held;
    void *buf[gmaf::B_COUNT];
    size_t bytes[gmaf::B_COUNT];
    void *pinned;                  // pinned host staging, kPinnedBytes
    gmaf_solve_info info;
    gmaf::GraphCache graph64, graph32;
    int num_sms;
    int no_graph;                  // loop control by host chunks instead of a graph
    int graph_pairs;               // PCG iterations per trip of the graph's WHILE body
    long long chunked_from;        // two-level reduction from this many publishing units
    int phase_timing;              // events around each phase launch (host chunks)
    double phase_ms[4];
    long long phase_count[4];
    cudaEvent_t ev[2 * 2 * 16 + 2];
    int ev_ready;
    int no_tune;                   // GMAF_NO_TUNE=1: first candidate kernels, no tuning
    int force_variant;             // GMAF_VARIANT=<id>: use that kernel variant when eligible
    gmaf::TuneEntry tune[gmaf::kTuneEntries];
    int ntune, tune_next;
    int pp_nth, pp_nz, pp_K;       // shape of the Picard-step fields held in B_PP
    double inner_floor;            // smallest relative residual asked of an inner FP32 solve
    int mixed_restart;             // restart the inner FP32 PCG at each refinement (else continue it)
    double reliable_delta;         // continued recurrence: residual reduction between two refinements
    int loop_guard;                // GMAF_LOOP_GUARD: fixed loop-guard limit (0: max_iter + 4)
};

namespace gmaf {

constexpr size_t kPinnedBytes = 64 * 1024;

// Opt a kernel in to `bytes` of dynamic shared memory on the current device
// (and, if asked, to the largest shared-memory carve-out).
// The attribute is per device, so each call site keeps a mask of the device
// ordinals it has set (ordinals from 64 on are set on every call).
inline void smem_optin(std::atomic<unsigned long long> &done, const void *fn, size_t bytes,
                       bool max_carveout = false)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return;
    }
    const unsigned long long bit = dev < 64 ? 1ull << dev : 0ull;
    if (bit && (done.load() & bit)) return;
    bool ok = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes) ==
              cudaSuccess;
    // the largest shared-memory carve-out, so that several blocks of a kernel with
    // a large ring fit on one SM
    if (ok && max_carveout)
        ok = cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout,
                                  (int)cudaSharedmemCarveoutMaxShared) == cudaSuccess;
    if (ok)
        done.fetch_or(bit);
    else
        cudaGetLastError();
}

int ensure(gmaf_ctx *ctx, int id, size_t bytes);
int cuda_status(cudaError_t e);
bool geom_valid(const gmaf_grid *g, const gmaf_physics *ph, const gmaf_texture *tex);
bool opts_valid(const gmaf_solver_opts *o);

// geometry / assembly / loads / Picard kernels (gmaf_assemble.cu)
int launch_trig(const Geom &g, double *trig, cudaStream_t s);
// simplified = 0: the 9 conditions of the general scheme (base, e_j + d_e, edot_j + d_edot)
// in 5 coefficient slots; 1: the 5 of the simplified scheme (base, edot_j + d_edot) in 1 slot.
int launch_fanout(const double *base, double d_e, double d_edot, double *conds, int *cslot_write,
                  cudaStream_t s, int simplified = 0);
int launch_assemble(const Geom &g, int ncond, const double *conds, const int *coef_slot,
                    double *D, double *aE, double *aN, double *S, const double *trig, int *flags,
                    int nslots, cudaStream_t s);
int launch_loads(const Geom &g, int ncond, const double *conds, const double *p,
                 const double *trig, double *partials, unsigned int *tickets, double *loads,
                 int *flags, int num_sms, cudaStream_t s);
struct PicardIn {
    double base[8], e_prev[4], F_ext[4];
    int simplified;                // Eq. 2.20-2.22 on the 5-condition batch
};
constexpr int kResultDoubles = 73;
int launch_picard_update(const double *loads, const PicardIn &in, double dt, double d_e,
                         double d_edot, double L, double *result, cudaStream_t s);
size_t loads_partials_bytes(int ncond, int num_sms);

// joint PCG (gmaf_pcg.cu).  Coefficient slots in device memory, FP64.
int solve_joint_device(gmaf_ctx *ctx, int nth, int nz, int K, int nslots, const int *cslot_host,
                       const double *D, const double *aE, const double *aN, const double *S,
                       double *p, const gmaf_solver_opts *opts, gmaf_solve_info *info);

}  // namespace gmaf
