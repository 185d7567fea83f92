// Staged FP32 phase A with the rebuilt diagonal, in a translation unit of its own.
//
// The assembly forms the diagonal of the Reynolds matrix as the sum of the four
// couplings of a cell plus, in the first and last rows, the conductance of the
// Dirichlet face (Eq. 2.1-2.7), so phase A, which holds the couplings of the row
// it multiplies anyway, rebuilds it in FP32 and reads only that boundary term:
// 4 bytes fewer per unknown and coefficient slot than reading the diagonal.  The
// FP32 sum differs from the rounded FP32 diagonal by a few units in the last place,
// an operator of the inner solve still symmetric and positive definite; the FP64
// refinement measures the residual with the exact matrix.
//
// The kernel lives here rather than in gmaf_pcg.cu because the staged phase A
// there is sensitive to where its code lies in its module.
#include "gmaf_internal.cuh"
#include "gmaf_pcg_kernels.cuh"
#include "gmaf_pcg_host.cuh"
#include "gmaf_drec.h"

#include <atomic>

namespace gmaf {

DrecKernel drec_phase_a()
{
    using R = RingA<float, 4, true>;
    const void *a = (const void *)k_phase_a_staged<float, 4, 32, 2, 2, kThreads, true>;
    const size_t smem = (size_t)kWarps * R::per_warp(2) * sizeof(float);
    static std::atomic<unsigned long long> done{0};
    smem_optin(done, a, smem);
    return {a, smem};
}

static __global__ void __launch_bounds__(kThreads) k_dbnd32(const float *__restrict__ D32,
                                                            const float *__restrict__ aE32,
                                                            const float *__restrict__ aN32,
                                                            float *__restrict__ dbnd, int nth, int nz,
                                                            int nslots)
{
    const long long n = (long long)nth * nz;
    const long long total = (long long)nslots * 2 * nth;
    for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < total;
         q += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(q % nth);
        const long long sj = q / nth;
        const int s = (int)(sj / 2), jb = (int)(sj % 2);
        const int j = jb ? nz - 1 : 0;
        const long long row = (long long)s * n + (long long)j * nth;
        const float aW = aE32[row + (i == 0 ? nth - 1 : i - 1)];
        const float aS = j > 0 ? aN32[row + i - nth] : 0.0f;
        const float sum = ((aE32[row + i] + aW) + aN32[row + i]) + aS;
        dbnd[q] = D32[row + i] - sum;
    }
}

int launch_dbnd32(const float *D32, const float *aE32, const float *aN32, float *dbnd, int nth,
                  int nz, int nslots, int num_sms, cudaStream_t s)
{
    const long long total = (long long)nslots * 2 * nth;
    k_dbnd32<<<stream_grid(total, num_sms), kThreads, 0, s>>>(D32, aE32, aN32, dbnd, nth, nz, nslots);
    return cuda_status(cudaGetLastError());
}

}  // namespace gmaf
