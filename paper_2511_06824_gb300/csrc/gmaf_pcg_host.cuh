// Host-side helpers of the PCG drivers (launch shapes, kernel sets, the stored
// diagonal), shared by the joint solver (gmaf_pcg.cu) and the allocation-free
// joint solve (gmaf_noalloc.cu).  Internal; not part of the ABI.
#pragma once

#include <cstdint>

#include "gmaf_internal.cuh"
#include "gmaf_pcg_kernels.cuh"

namespace gmaf {

static int grid_for(const void *kernel, long long work_items, int num_sms, size_t smem = 0,
                    int threads = kThreads)
{
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem) != cudaSuccess ||
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

// The phase kernels of one run: strip width W = 32 * VEC, TY rows per task,
// MINB blocks per SM requested from the register allocator, and the schedule
// (0: dynamic tasks; 1: static ranges, phase A marching against phase B).
template <typename T>
struct KernelSet {
    const void *a, *b, *b_init;
    int W, TY, id;
    size_t smem_b;             // dynamic shared memory of the phase-B kernels
    int sched;
    size_t smem_a;             // dynamic shared memory of the phase-A kernel
    int p_period;              // iterations between two p updates of phase A (1 or 2)
    int threads = kThreads;    // threads per block of both phase kernels
    int tma = 0;               // phase B is the block-marched TMA kernel (tasks per block)
    int ty_b = 0;              //   its rows per task
    int threads_b = 0;         // threads per block of the phase-B kernels (0: threads)
};

// Threads per block of a kernel set's phase-B kernels.
template <typename T>
static int b_threads(const KernelSet<T> &ks)
{
    return ks.threads_b ? ks.threads_b : ks.threads;
}

// id = 1000 VEC + 10 TY + MINB (dynamic), 1000000 + 1000 VEC + MINB (static).
template <typename T, int VEC, int TY, int MINB, int SCHED = 0>
static KernelSet<T> ks_of(int)
{
    return {(const void *)k_phase_a<T, VEC, TY, MINB, SCHED>,
            (const void *)k_phase_b<T, VEC, TY, MINB, false, SCHED>,
            (const void *)k_phase_b<T, VEC, TY, MINB, true, SCHED>, 32 * VEC, TY,
            SCHED ? 1000000 + 1000 * VEC + MINB : 1000 * VEC + 10 * TY + MINB, 0, SCHED};
}


static bool aligned16(const void *p) { return ((uintptr_t)p & 15u) == 0; }

template <typename T>
static bool vec_ok(const PcgDesc<T> &h)
{
    constexpr int V = sizeof(T) == 4 ? 4 : 2;
    bool ok = (h.nth % V) == 0;
    const void *ptrs[] = {h.D, h.invD, h.aE, h.aN, h.p, h.z, h.v, h.u[0], h.u[1], h.r[0], h.r[1]};
    for (const void *q : ptrs) ok = ok && aligned16(q);
    return ok;
}

template <typename T>
static cudaError_t launch(const void *fn, int grid, const PcgDesc<T> *dd, cudaStream_t s,
                         size_t smem = 0, int threads = kThreads)
{
    void *args[] = {(void *)&dd};
    return cudaLaunchKernel(fn, dim3(grid), dim3(threads), args, smem, s);
}

// Blocks for a persistent phase kernel: enough to hold every task's warp, at
// most what stays resident.
static int phase_grid(const void *kernel, long long ntasks, int num_sms, size_t smem = 0,
                      int threads = kThreads)
{
    const int warps = threads / 32;
    return grid_for(kernel, (ntasks + warps - 1) / warps, num_sms, smem, threads);
}

// ---------------------------------------------------------------- ASSOR-I
//
// Eq. 3.2: {M^-1}_ii = w (2 - w) / {(D + w L) D^-1 (D + w L)^T}_ii
//                    = w (2 - w) / (D_i + w^2 sum_{k in low(i)} a_ik^2 / D_k),
// low(i) = {S; W if i > 0; E across the wrap if i = n_theta - 1}, the strictly
// lower couplings in the joint index order.  The PCG phases apply it as a
// diagonal, through the Jacobi path.  With outer given the result is for the
// FP32 matrix scale * A (outer->scale, set by k_to_f32), i.e. divided by scale.
template <typename T>
static __global__ void __launch_bounds__(kThreads)
k_assor1_diag(const double *__restrict__ D, const double *__restrict__ aE,
              const double *__restrict__ aN, int nth, int nz, long long m, double omega,
              const Scalars *__restrict__ outer, T *__restrict__ out)
{
    const long long n = (long long)nth * nz;
    const double scale = outer ? outer->scale : 1.0;
    const double c1 = omega * (2.0 - omega), w2 = omega * omega;
    for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < m;
         q += (long long)gridDim.x * blockDim.x) {
        const long long P = q % n;
        const int j = (int)(P / nth), i = (int)(P - (long long)j * nth);
        double s = 0.0;
        if (j > 0) {
            const double a = aN[q - nth];
            s += a * a / D[q - nth];
        }
        if (i > 0) {
            const double a = aE[q - 1];
            s += a * a / D[q - 1];
        }
        if (i == nth - 1) {
            const double a = aE[q];
            s += a * a / D[q - (nth - 1)];
        }
        out[q] = (T)(c1 / (D[q] + w2 * s) / scale);
    }
}

// The diagonal the PCG phases divide by: 1/D (Jacobi, ASSOR-II) or ASSOR-I's.
static void diag_inverse64(const gmaf_solver_opts *opts, const double *D, const double *aE,
                           const double *aN, int nth, int nz, long long m, double *out, int num_sms,
                           cudaStream_t s)
{
    if (opts->precond == 2)
        k_assor1_diag<double><<<stream_grid(m, num_sms), kThreads, 0, s>>>(D, aE, aN, nth, nz, m,
                                                                          opts->omega, nullptr, out);
    else
        k_invd64<<<stream_grid(m, num_sms), kThreads, 0, s>>>(D, out, m,
                                                               opts->precond == 1 ? opts->omega : 1.0);
}

// PCG-kernel preconditioner: ASSOR-II runs its two passes, Jacobi and ASSOR-I
// divide by the stored diagonal.
static int kernel_precond(const gmaf_solver_opts *opts) { return opts->precond == 1 ? 1 : 0; }

}  // namespace gmaf
