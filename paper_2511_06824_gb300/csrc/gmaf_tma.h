// Host-visible part of the TMA phase B (gmaf_tma.cu): launch shape constants, the
// tensor-map parameter block, and the entry points the PCG driver (gmaf_pcg.cu)
// calls.  Internal; not part of the ABI.
#pragma once

#include <cstddef>

#include "gmaf_internal.cuh"

namespace gmaf {

constexpr int kTmaW = 128;                        // strip width (columns)
constexpr int kTmaRow = kTmaW + 8;                // a staged row: columns i0 - 4 .. i0 + 131
constexpr int kTmaWarps = 8;                      // consumer warps of a block
constexpr int kTmaConsumers = 32 * kTmaWarps;
constexpr int kTmaThreads = kTmaConsumers + 32;   // and the producer warp
constexpr int kTmaMaxClaims = 8;                  // tasks claimed and not yet finished
constexpr int kTmaMail = 16;                      // finished tasks waiting to be published

// Layout of one field's chunk (CR staged rows) in a ring slot: the rows, then the
// wrap boxes of columns n_theta - 4 .. n_theta - 1 and 0 .. 3.
template <int CR>
struct TmaChunk {
    static constexpr int kWrapW = CR * kTmaRow;
    static constexpr int kWrapE = kWrapW + CR * 4;
    static constexpr int kField = kWrapE + CR * 4;   // floats per field
    static constexpr int kRing = 2 * CR;              // rows of the y and w rings
};

// The kernel's tensor maps: {row box, wrap box} of r[0], r[1], v, omega/D, aE, aN.
enum TmaMap { kTmR0 = 0, kTmR1 = 2, kTmV = 4, kTmOd = 6, kTmAE = 8, kTmAN = 10, kTmaMaps = 12 };

// One encoded tensor map (the driver's 128-byte, 64-byte aligned object).
struct alignas(64) TmaMapBytes {
    unsigned long long w[16];
};
// The maps travel as a __grid_constant__ kernel parameter.
struct TmaParams {
    TmaMapBytes m[kTmaMaps];
};

// Dynamic shared memory of k_phase_b_tma<., NS, RPW>, in floats.
__host__ __device__ constexpr int tma_b_smem_floats(int NS, int RPW)
{
    return NS * 5 * (8 * RPW * (kTmaRow + 8)) + 2 * (8 * RPW) * (kTmaW * 2 + 2 + 4 + 2);
}

// The TMA phase-B kernels with NS chunk slots and RPW rows per consumer warp
// (NS in {3, 4}, RPW in {1, 2}), opted in to their shared memory on the current
// device; null kernels for another pair.
struct TmaKernels {
    const void *b, *b_init;
    size_t smem;
};
TmaKernels tma_kernels(int ns, int rpw);

// Encode the tensor maps of a run's FP32 arrays for chunks of `rows` rows (8 or
// 16); false when the shape does not suit them or the driver's encoder is missing.
bool tma_encode_maps(const PcgDesc<float> &h, TmaParams &tp, int rows);

}  // namespace gmaf
