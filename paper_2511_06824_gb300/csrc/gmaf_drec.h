// Host-visible part of the staged FP32 phase A with the rebuilt diagonal
// (gmaf_drec.cu): its kernel and the boundary-term kernel the PCG driver
// (gmaf_pcg.cu) calls.  Internal; not part of the ABI.
#pragma once

#include <cstddef>

#include "gmaf_internal.cuh"

namespace gmaf {

// The staged FP32 phase A (4 columns a lane, 32-row tasks, 2 blocks per SM, rows
// two ahead, p updates paired) that rebuilds the diagonal from the couplings
// instead of reading it, opted in to its shared memory on the current device.
struct DrecKernel {
    const void *a;
    size_t smem;
};
DrecKernel drec_phase_a();

// The Dirichlet term of the first and last rows that the rebuilt diagonal needs:
// dbnd[slot][0 or 1][i] = D32 - (((aE + aW) + aN) + aS) in FP32 at rows 0 and
// n_z - 1 (the sum in the order the phase kernel forms it).
int launch_dbnd32(const float *D32, const float *aE32, const float *aN32, float *dbnd, int nth,
                  int nz, int nslots, int num_sms, cudaStream_t s);

}  // namespace gmaf
