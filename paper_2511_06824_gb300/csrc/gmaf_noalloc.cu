// Allocation-free joint solve (gmaf_solve_joint_noalloc).
//
// The FP64 joint solve for callers that may not allocate device memory while
// they run.  All of its scratch (descriptor, scalars, partial sums, the stored
// diagonal and the six PCG vectors) lives in one file-scope device array of
// GMAF_NOALLOC_SCRATCH_BYTES.  This file is a module of its own: the array is
// committed on a device when this module is first loaded there, i.e. at the
// first call of gmaf_solve_joint_noalloc on that device (under lazy module
// loading, the CUDA default; at context creation under CUDA_MODULE_LOADING=EAGER),
// and held until the process exits.  The other entry points never load it.
//
// Host code cannot use the array's name as a device address, so the address is
// looked up once per device with cudaGetSymbolAddress and passed to the kernels.
// The loop is driven from the host in chunks (no graph, no events, no pinned
// staging), so nothing here allocates.  The kernels are the untuned default
// variants of the joint solver (two columns per lane when n_theta is even and
// the arrays are 16-byte aligned, else one), with the one-level reduction of
// the phase sums.
#include <mutex>

#include "gmaf_internal.cuh"
#include "gmaf_pcg_kernels.cuh"
#include "gmaf_pcg_host.cuh"

namespace gmaf {

static __device__ __align__(256) unsigned char g_noalloc_scratch[GMAF_NOALLOC_SCRATCH_BYTES];

namespace {
constexpr size_t kNaDesc = 0;          // PcgDesc<double>
constexpr size_t kNaResid = 2048;      // ResidDesc
constexpr size_t kNaScal = 4096;       // Scalars of the run, Scalars of the residual
constexpr size_t kNaCslot = 8192;      // int[kMaxCond], identity coefficient map
constexpr size_t kNaPart = 16384;      // per-task / per-block partial sums
constexpr size_t kNaPartBytes = 524288;
constexpr size_t kNaVec = 1048576;     // 1/D, r0, r1, u0, u1, z, v: N doubles each
constexpr int kNaMaxDevices = 64;
static_assert(sizeof(PcgDesc<double>) <= kNaResid - kNaDesc, "descriptor slot");
static_assert(sizeof(ResidDesc) <= kNaScal - kNaResid, "residual descriptor slot");
static_assert(2 * sizeof(Scalars) <= kNaCslot - kNaScal, "scalar slot");
static_assert(kNaPart + kNaPartBytes <= kNaVec, "partials slot");

std::mutex g_na_mutex;
void *g_na_base[kNaMaxDevices];

size_t round256(size_t b) { return (b + 255) & ~size_t(255); }

// Device address of the scratch array on the current device (looked up once per device).
int noalloc_base(char **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_status(e);
    if (dev < 0 || dev >= kNaMaxDevices) return GMAF_CUDA_ERROR;
    std::lock_guard<std::mutex> lock(g_na_mutex);
    if (!g_na_base[dev]) {
        void *ptr = nullptr;
        e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
        if (e != cudaSuccess || ptr == nullptr) return cuda_status(e == cudaSuccess ? cudaErrorInvalidSymbol : e);
        g_na_base[dev] = ptr;
    }
    *out = (char *)g_na_base[dev];
    return GMAF_OK;
}
}  // namespace

}  // namespace gmaf

extern "C" int gmaf_solve_joint_noalloc(const gmaf_grid *grid, int32_t n_cond, const double *D,
                                        const double *aE, const double *aN, const double *S,
                                        double *p, const gmaf_solver_opts *opts,
                                        void *cuda_stream, int32_t *iters_out,
                                        double *rel_res_out)
{
    using namespace gmaf;
    if (!grid || !D || !aE || !aN || !S || !p) return GMAF_INVALID_ARG;
    if (grid->n_theta < 3 || grid->n_z < 2 || n_cond < 1 || n_cond > kMaxCond) return GMAF_INVALID_ARG;
    if (!opts_valid(opts) || opts->precision != 0 || opts->criterion != 0) return GMAF_INVALID_ARG;
    const int nth = grid->n_theta, nz = grid->n_z, K = n_cond;
    const long long n = (long long)nth * nz;
    const long long N = n * K;
    const size_t vec = round256((size_t)N * sizeof(double));
    if ((long long)nth * nz > (1LL << 31) - 1 || kNaVec + 7 * vec > (size_t)GMAF_NOALLOC_SCRATCH_BYTES)
        return GMAF_OUT_OF_MEMORY;
    char *base = nullptr;
    int st = noalloc_base(&base);
    if (st != GMAF_OK) return st;
    int dev = 0, num_sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return cuda_status(e);
    cudaStream_t s = (cudaStream_t)cuda_stream;
    // Once work is on the stream, an error return first waits for it, so that the
    // call leaves nothing running on the shared array (result ignored: the error
    // being returned is the one that counts).
    auto fail = [&](cudaError_t err) {
        cudaStreamSynchronize(s);
        cudaGetLastError();
        return cuda_status(err);
    };

    PcgDesc<double> h{};
    h.nth = nth;
    h.nz = nz;
    h.K = K;
    h.n = n;
    h.precond = kernel_precond(opts);
    h.zero_init = opts->zero_init;
    h.use_cond = 0;
    double *vbase = (double *)(base + kNaVec);
    double *invD = vbase;
    double *vecs[6];
    for (int q = 0; q < 6; ++q) vecs[q] = (double *)(base + kNaVec + (size_t)(q + 1) * vec);
    Scalars *dsc = (Scalars *)(base + kNaScal);
    Scalars *dsc_res = dsc + 1;
    int *cslot = (int *)(base + kNaCslot);
    h.D = D;
    h.invD = invD;
    h.aE = aE;
    h.aN = aN;
    h.cslot = cslot;
    h.b = S;
    h.p = p;
    h.r[0] = vecs[0];
    h.r[1] = vecs[1];
    h.u[0] = vecs[2];
    h.u[1] = vecs[3];
    h.z = vecs[4];
    h.v = vecs[5];
    h.omega = opts->omega;
    h.eps = opts->eps;
    h.max_iter = opts->max_iter;
    h.sc = dsc;
    h.partials = (double *)(base + kNaPart);
    const KernelSet<double> ks = vec_ok(h) ? ks_of<double, 2, 32, 2>(0) : ks_of<double, 1, 32, 3>(4);
    h.tiles_x = (nth + ks.W - 1) / ks.W;
    h.tiles_y = (nz + ks.TY - 1) / ks.TY;
    h.ntiles = (long long)h.tiles_x * h.tiles_y * K;
    const int grid_a = phase_grid(ks.a, h.ntiles, num_sms, ks.smem_a);
    const int grid_b = phase_grid(ks.b, h.ntiles, num_sms, ks.smem_b);
    const int grid_s = stream_grid(N, num_sms);
    long long np = 2 * h.ntiles;
    if (2LL * grid_s > np) np = 2LL * grid_s;
    if ((size_t)np * sizeof(double) > kNaPartBytes) return GMAF_OUT_OF_MEMORY;
    PcgDesc<double> *d_desc = (PcgDesc<double> *)(base + kNaDesc);
    ResidDesc *d_rdesc = (ResidDesc *)(base + kNaResid);
    ResidDesc rd{};
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
    rd.sc = dsc_res;
    rd.partials = h.partials;
    int slots[kMaxCond];
    for (int k = 0; k < K; ++k) slots[k] = k;

    // The array keeps the previous call's contents: clear the scalars and the
    // reduction tickets, which must start at zero.  The copies below come from
    // pageable (stack) memory and have consumed their sources when they return.
    e = cudaMemsetAsync(base + kNaScal, 0, kNaCslot - kNaScal, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(cslot, slots, (size_t)K * sizeof(int), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(d_desc, &h, sizeof(h), cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return fail(e);
    diag_inverse64(opts, D, aE, aN, nth, nz, N, invD, num_sms, s);

    Scalars hs{}, hr{};
    int restarted = 0;
    bool keep = false, init_r = true;
    int status = GMAF_NOT_CONVERGED;
    double true_rel = 0.0;
    for (;;) {
        k_reset<<<1, 32, 0, s>>>(dsc, keep ? 1 : 0);
        if (init_r) k_init_r<double><<<grid_s, kThreads, 0, s>>>(d_desc);
        e = launch<double>(ks.b_init, grid_b, d_desc, s, ks.smem_b);
        if (e == cudaSuccess) e = cudaGetLastError();
        if (e != cudaSuccess) return fail(e);
        const int chunk = 16;
        for (int it = 0; it <= opts->max_iter + chunk; it += chunk) {
            int done = 0;
            e = cudaMemcpyAsync(&done, &dsc->done, sizeof(int), cudaMemcpyDeviceToHost, s);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s);
            if (e != cudaSuccess) return fail(e);
            if (done) break;
            for (int q = 0; q < chunk && e == cudaSuccess; ++q) {
                e = launch<double>(ks.a, grid_a, d_desc, s, ks.smem_a);
                if (e == cudaSuccess) e = launch<double>(ks.b, grid_b, d_desc, s, ks.smem_b);
            }
            if (e != cudaSuccess) return fail(e);
        }
        k_finalize<double><<<grid_s, kThreads, 0, s>>>(d_desc);
        e = cudaMemcpyAsync(&hs, dsc, sizeof(Scalars), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return fail(e);
        // true residual S - A p into r[iter & 1], where a restart reads it
        rd.r = h.r[hs.iter & 1];
        e = cudaMemcpyAsync(d_rdesc, &rd, sizeof(rd), cudaMemcpyHostToDevice, s);
        if (e != cudaSuccess) return fail(e);
        k_resid64<<<grid_s, kThreads, 0, s>>>(d_rdesc);
        e = cudaMemcpyAsync(&hr, dsc_res, sizeof(Scalars), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return fail(e);
        true_rel = hr.true_rel;
        if (hs.zero_rhs) {
            e = cudaMemsetAsync(p, 0, (size_t)N * sizeof(double), s);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s);
            if (e != cudaSuccess) return fail(e);
            true_rel = 0.0;
        }
        if (hs.status != 0 || hr.status != 0) {
            status = hs.status != 0 ? hs.status : hr.status;
            break;
        }
        if ((hs.converged || hs.zero_rhs) && true_rel <= 10.0 * opts->eps) {
            status = GMAF_OK;
            break;
        }
        if (restarted || hs.iter >= opts->max_iter) {
            status = GMAF_NOT_CONVERGED;
            break;
        }
        restarted = 1;
        keep = true;
        init_r = false;
    }
    if (iters_out) *iters_out = hs.iter;
    if (rel_res_out) *rel_res_out = true_rel;
    return status;
}
