// C ABI of the piston-gap library: context, workspace, argument checks and the
// orchestration of one Picard iteration.  Kernels live in gmaf_assemble.cu and
// gmaf_pcg.cu.
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <new>

#include "gmaf_internal.cuh"

namespace gmaf {

int cuda_status(cudaError_t e)
{
    if (e == cudaSuccess) return GMAF_OK;
    if (e == cudaErrorMemoryAllocation) return GMAF_OUT_OF_MEMORY;
    return GMAF_CUDA_ERROR;
}

// Grow buffer `id` to at least `bytes` within the context's budget.  Contents
// are not preserved.
int ensure(gmaf_ctx *ctx, int id, size_t bytes)
{
    if (bytes == 0) bytes = 16;
    if (ctx->bytes[id] >= bytes) return GMAF_OK;
    const size_t grow = bytes - ctx->bytes[id];
    if (ctx->budget && ctx->held + grow > ctx->budget) return GMAF_OUT_OF_MEMORY;
    if (ctx->buf[id]) {
        cudaError_t e = cudaStreamSynchronize(ctx->stream);
        if (e != cudaSuccess) return cuda_status(e);
        cudaFree(ctx->buf[id]);
        ctx->held -= ctx->bytes[id];
        ctx->buf[id] = nullptr;
        ctx->bytes[id] = 0;
    }
    void *p = nullptr;
    cudaError_t e = cudaMalloc(&p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return GMAF_OUT_OF_MEMORY;
    }
    e = cudaMemsetAsync(p, 0, bytes, ctx->stream);
    if (e != cudaSuccess) {
        cudaFree(p);
        return cuda_status(e);
    }
    ctx->buf[id] = p;
    ctx->bytes[id] = bytes;
    ctx->held += bytes;
    return GMAF_OK;
}

static bool finite_pos(double x) { return std::isfinite(x) && x > 0.0; }

bool geom_valid(const gmaf_grid *g, const gmaf_physics *ph, const gmaf_texture *tex)
{
    if (!g || !ph) return false;
    if (g->n_theta < 3 || g->n_z < 2) return false;
    if ((long long)g->n_theta * g->n_z > (1LL << 31) - 1) return false;
    if (!finite_pos(ph->R_k) || !finite_pos(ph->L) || !finite_pos(ph->c) || !finite_pos(ph->mu))
        return false;
    if (!std::isfinite(ph->v_slide) || !std::isfinite(ph->p_chamber) || !std::isfinite(ph->p_case))
        return false;
    if (tex && tex->kind != 0) {
        if (tex->kind != 1) return false;
        if (!finite_pos(tex->radius) || !std::isfinite(tex->depth) || tex->depth < 0.0) return false;
        if (!(tex->area_density > 0.0 && tex->area_density < 0.9069)) return false;   // < hexagonal packing
        if (!std::isfinite(tex->offset_theta) || !std::isfinite(tex->offset_z)) return false;
    }
    return true;
}

bool opts_valid(const gmaf_solver_opts *o)
{
    if (!o) return false;
    if (o->precond != 0 && o->precond != 1 && o->precond != 2) return false;
    if (o->precond != 0 && !(o->omega > 0.0 && o->omega < 2.0)) return false;
    if (!(o->eps > 0.0) || !std::isfinite(o->eps)) return false;
    if (o->max_iter < 0) return false;
    if (o->precision != 0 && o->precision != 1) return false;
    if (o->criterion != 0 && o->criterion != 1) return false;
    if (o->criterion == 1 && o->precision != 0) return false;    // asynchronized: FP64 only
    return true;
}

static bool state_finite(const gmaf_state *s)
{
    for (int q = 0; q < 4; ++q)
        if (!std::isfinite(s->e[q]) || !std::isfinite(s->edot[q])) return false;
    return true;
}

}  // namespace gmaf

using namespace gmaf;

extern "C" {

const char *gmaf_status_string(int st)
{
    switch (st) {
    case GMAF_OK: return "ok";
    case GMAF_INVALID_ARG: return "invalid argument";
    case GMAF_CONTACT: return "film thickness <= 0 (contact)";
    case GMAF_NOT_CONVERGED: return "not converged within the iteration budget";
    case GMAF_NONFINITE: return "non-finite value in a reduction";
    case GMAF_OUT_OF_MEMORY: return "workspace exceeds the HBM budget";
    case GMAF_CUDA_ERROR: return "CUDA runtime error";
    case GMAF_TIMEOUT: return "device-side loop guard expired";
    case GMAF_CANCELLED: return "request cancelled";
    default: return "unknown status";
    }
}

int gmaf_create(gmaf_ctx **out, size_t hbm_budget_bytes, void *cuda_stream)
{
    if (!out) return GMAF_INVALID_ARG;
    *out = nullptr;
    gmaf_ctx *c = new (std::nothrow) gmaf_ctx();
    if (!c) return GMAF_OUT_OF_MEMORY;
    std::memset(c, 0, sizeof(*c));
    c->graph64 = GraphCache{};
    c->graph32 = GraphCache{};
    cudaError_t e = cudaGetDevice(&c->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device);
    if (e == cudaSuccess) e = cudaMallocHost(&c->pinned, kPinnedBytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        delete c;
        return GMAF_CUDA_ERROR;
    }
    std::memset(c->pinned, 0, kPinnedBytes);
    c->stream = (cudaStream_t)cuda_stream;
    c->budget = hbm_budget_bytes;
    const char *ng = std::getenv("GMAF_NO_GRAPH");
    c->no_graph = (ng && ng[0] == '1') ? 1 : 0;
    const char *gp = std::getenv("GMAF_GRAPH_UNROLL");
    // 8 PCG iterations per evaluation of the graph's loop condition: each evaluation
    // costs about 4 us on the 2048 x 1024 x 9 step (4 iterations: 0.2245 -> 0.2214 ms
    // per iteration; 8: the step 604.6 -> 602.4 ms)
    c->graph_pairs = gp ? std::atoi(gp) : 8;
    if (c->graph_pairs < 1 || c->graph_pairs > 16) c->graph_pairs = 8;
    const char *cf = std::getenv("GMAF_CHUNKED_FROM");
    c->chunked_from = cf ? std::atoll(cf) : 4096;
    if (c->chunked_from < 1) c->chunked_from = 4096;
    const char *nt = std::getenv("GMAF_NO_TUNE");
    c->no_tune = (nt && nt[0] == '1') ? 1 : 0;
    const char *fv = std::getenv("GMAF_VARIANT");
    c->force_variant = fv ? std::atoi(fv) : -1;
    const char *ie = std::getenv("GMAF_INNER_EPS");
    c->inner_floor = ie ? std::atof(ie) : 5e-7;
    if (!(c->inner_floor > 0.0 && c->inner_floor < 0.5)) c->inner_floor = 5e-7;
    const char *mr = std::getenv("GMAF_MIXED_RESTART");
    c->mixed_restart = (mr && std::atoi(mr) != 0) ? 1 : 0;
    const char *rdl = std::getenv("GMAF_RELIABLE_DELTA");
    c->reliable_delta = rdl ? std::atof(rdl) : 0.1;
    if (!(c->reliable_delta > 0.0 && c->reliable_delta < 0.5)) c->reliable_delta = 0.1;
    // fault injection from the host: a fixed, lower limit for the device loop guard,
    // so that a test can make it expire (GMAF_TIMEOUT) without any device fault
    const char *lg = std::getenv("GMAF_LOOP_GUARD");
    c->loop_guard = lg ? std::atoi(lg) : 0;
    if (c->loop_guard < 0) c->loop_guard = 0;
    *out = c;
    return GMAF_OK;
}

int gmaf_destroy(gmaf_ctx *c)
{
    if (!c) return GMAF_INVALID_ARG;
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (c->graph64.exec) cudaGraphExecDestroy(c->graph64.exec);
    if (c->graph32.exec) cudaGraphExecDestroy(c->graph32.exec);
    for (int i = 0; i < B_COUNT; ++i)
        if (c->buf[i]) cudaFree(c->buf[i]);
    if (c->pinned) cudaFreeHost(c->pinned);
    if (c->ev_ready)
        for (auto &ev : c->ev) cudaEventDestroy(ev);
    delete c;
    return e == cudaSuccess ? GMAF_OK : GMAF_CUDA_ERROR;
}

int gmaf_set_stream(gmaf_ctx *c, void *cuda_stream)
{
    if (!c) return GMAF_INVALID_ARG;
    cudaError_t e = cudaStreamSynchronize(c->stream);
    c->stream = (cudaStream_t)cuda_stream;
    return cuda_status(e);
}

int gmaf_set_phase_timing(gmaf_ctx *c, int on)
{
    if (!c) return GMAF_INVALID_ARG;
    if (on && !c->ev_ready) {
        for (auto &ev : c->ev) {
            cudaError_t e = cudaEventCreate(&ev);
            if (e != cudaSuccess) return cuda_status(e);
        }
        c->ev_ready = 1;
    }
    c->phase_timing = on ? 1 : 0;
    for (int q = 0; q < 4; ++q) {
        c->phase_ms[q] = 0.0;
        c->phase_count[q] = 0;
    }
    return GMAF_OK;
}

int gmaf_phase_timing(const gmaf_ctx *c, double ms_out[4], int64_t launches_out[4])
{
    if (!c || !ms_out || !launches_out) return GMAF_INVALID_ARG;
    for (int q = 0; q < 4; ++q) {
        ms_out[q] = c->phase_ms[q];
        launches_out[q] = c->phase_count[q];
    }
    return GMAF_OK;
}

int gmaf_last_fields(gmaf_ctx *c, const gmaf_grid *grid, double *p_out)
{
    if (!c || !grid || !p_out || !c->buf[B_PP]) return GMAF_INVALID_ARG;
    if (grid->n_theta != c->pp_nth || grid->n_z != c->pp_nz) return GMAF_INVALID_ARG;
    const size_t bytes = (size_t)c->pp_K * grid->n_theta * grid->n_z * sizeof(double);
    return cuda_status(cudaMemcpyAsync(p_out, c->buf[B_PP], bytes, cudaMemcpyDeviceToDevice, c->stream));
}

int gmaf_workspace_bytes(const gmaf_ctx *c, size_t *bytes_out)
{
    if (!c || !bytes_out) return GMAF_INVALID_ARG;
    *bytes_out = c->held;
    return GMAF_OK;
}

int gmaf_last_solve_info(const gmaf_ctx *c, gmaf_solve_info *info_out)
{
    if (!c || !info_out) return GMAF_INVALID_ARG;
    *info_out = c->info;
    return GMAF_OK;
}

int gmaf_assemble(gmaf_ctx *c, const gmaf_grid *grid, const gmaf_physics *phys,
                  const gmaf_texture *tex, const gmaf_state *conds, int32_t n_cond, double *D,
                  double *aE, double *aN, double *S)
{
    if (!c || !conds || !D || !aE || !aN || !S) return GMAF_INVALID_ARG;
    if (!geom_valid(grid, phys, tex) || n_cond < 1 || n_cond > kMaxCond) return GMAF_INVALID_ARG;
    for (int k = 0; k < n_cond; ++k)
        if (!state_finite(&conds[k])) return GMAF_INVALID_ARG;
    const Geom g = make_geom(grid, phys, tex);
    cudaStream_t s = c->stream;
    int st;
    if ((st = ensure(c, B_TRIG, (size_t)4 * g.nth * sizeof(double)))) return st;
    if ((st = ensure(c, B_FLAGS, 64))) return st;
    if ((st = ensure(c, B_CONDS, (size_t)kMaxCond * 8 * sizeof(double)))) return st;
    if ((st = ensure(c, B_CSLOT, (size_t)kMaxCond * 2 * sizeof(int)))) return st;
    // condition states (gmaf_state is 8 contiguous doubles) and the identity
    // coefficient map, copied from pageable memory so the copies consume the
    // sources before returning
    static_assert(sizeof(gmaf_state) == 8 * sizeof(double), "gmaf_state layout");
    int hs[kMaxCond];
    for (int k = 0; k < n_cond; ++k) hs[k] = k;
    int *slots = (int *)c->buf[B_CSLOT] + kMaxCond;
    cudaError_t e = cudaMemcpyAsync(c->buf[B_CONDS], conds, (size_t)n_cond * sizeof(gmaf_state),
                                    cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(slots, hs, (size_t)n_cond * sizeof(int), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->buf[B_FLAGS], 0, 64, s);
    if (e != cudaSuccess) return cuda_status(e);
    if ((st = launch_trig(g, (double *)c->buf[B_TRIG], s))) return st;
    if ((st = launch_assemble(g, n_cond, (const double *)c->buf[B_CONDS], slots, D, aE, aN, S,
                              (const double *)c->buf[B_TRIG], (int *)c->buf[B_FLAGS], n_cond, s)))
        return st;
    int *flag_h = (int *)((char *)c->pinned + 12288);
    e = cudaMemcpyAsync(flag_h, c->buf[B_FLAGS], sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_status(e);
    return (*flag_h & 1) ? GMAF_CONTACT : GMAF_OK;
}

int gmaf_solve_joint(gmaf_ctx *c, const gmaf_grid *grid, int32_t n_cond, const double *D,
                     const double *aE, const double *aN, const double *S, double *p,
                     const gmaf_solver_opts *opts, int32_t *iters_out, double *rel_res_out)
{
    if (!c || !grid || !D || !aE || !aN || !S || !p) return GMAF_INVALID_ARG;
    if (grid->n_theta < 3 || grid->n_z < 2 || n_cond < 1 || n_cond > kMaxCond) return GMAF_INVALID_ARG;
    if ((long long)grid->n_theta * grid->n_z > (1LL << 31) - 1) return GMAF_INVALID_ARG;
    if (!opts_valid(opts)) return GMAF_INVALID_ARG;
    int slots[kMaxCond];
    for (int k = 0; k < n_cond; ++k) slots[k] = k;
    gmaf_solve_info info{};
    int st = solve_joint_device(c, grid->n_theta, grid->n_z, n_cond, n_cond, slots, D, aE, aN, S, p,
                                opts, &info);
    c->info = info;
    if (iters_out) *iters_out = info.iterations;
    if (rel_res_out) *rel_res_out = info.true_rel_residual;
    return st;
}

int gmaf_integrate_loads(gmaf_ctx *c, const gmaf_grid *grid, const gmaf_physics *phys,
                         const gmaf_texture *tex, const gmaf_state *conds, int32_t n_cond,
                         const double *p, double *loads)
{
    if (!c || !conds || !p || !loads) return GMAF_INVALID_ARG;
    if (!geom_valid(grid, phys, tex) || n_cond < 1 || n_cond > kMaxCond) return GMAF_INVALID_ARG;
    for (int k = 0; k < n_cond; ++k)
        if (!state_finite(&conds[k])) return GMAF_INVALID_ARG;
    const Geom g = make_geom(grid, phys, tex);
    cudaStream_t s = c->stream;
    int st;
    if ((st = ensure(c, B_TRIG, (size_t)4 * g.nth * sizeof(double)))) return st;
    if ((st = ensure(c, B_FLAGS, 64))) return st;
    if ((st = ensure(c, B_CONDS, (size_t)kMaxCond * 8 * sizeof(double)))) return st;
    if ((st = ensure(c, B_LOADPART, loads_partials_bytes(kMaxCond, c->num_sms)))) return st;
    cudaError_t e = cudaMemcpyAsync(c->buf[B_CONDS], conds, (size_t)n_cond * sizeof(gmaf_state),
                                    cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return cuda_status(e);
    if ((st = launch_trig(g, (double *)c->buf[B_TRIG], s))) return st;
    unsigned *tickets = (unsigned *)c->buf[B_LOADPART];
    double *part = (double *)((char *)c->buf[B_LOADPART] + kMaxCond * sizeof(unsigned));
    return launch_loads(g, n_cond, (const double *)c->buf[B_CONDS], p, (const double *)c->buf[B_TRIG],
                        part, tickets, loads, (int *)c->buf[B_FLAGS], c->num_sms, s);
}

}  // extern "C"

// One Picard iteration on the device: the general double-Jacobian scheme (9
// conditions in 5 coefficient slots) or, with simplified, the conventional one
// of Eq. 2.20-2.22 (5 conditions in 1 slot, e_prev unused).
static int picard_impl(gmaf_ctx *c, const gmaf_grid *grid, const gmaf_physics *phys,
                       const gmaf_texture *tex, gmaf_state *state, const double e_prev[4], double dt,
                       const double F_ext[4], double d_e, double d_edot,
                       const gmaf_solver_opts *opts, double loads_out[12], double J_out[48],
                       double G_out[4], int32_t *iters_out, bool simplified)
{
    if (!c || !state || !e_prev || !F_ext) return GMAF_INVALID_ARG;
    if (!geom_valid(grid, phys, tex) || !opts_valid(opts)) return GMAF_INVALID_ARG;
    if (!state_finite(state) || !std::isfinite(dt) || !std::isfinite(d_e) || !std::isfinite(d_edot) ||
        d_e == 0.0 || d_edot == 0.0)
        return GMAF_INVALID_ARG;
    for (int q = 0; q < 4; ++q)
        if (!std::isfinite(e_prev[q]) || !std::isfinite(F_ext[q])) return GMAF_INVALID_ARG;
    const int K = simplified ? 5 : 9, NSLOT = simplified ? 1 : 5;
    const Geom g = make_geom(grid, phys, tex);
    const size_t n = (size_t)g.nth * g.nz;
    cudaStream_t s = c->stream;
    int st;
    if ((st = ensure(c, B_TRIG, (size_t)4 * g.nth * sizeof(double)))) return st;
    if ((st = ensure(c, B_FLAGS, 64))) return st;
    if ((st = ensure(c, B_CONDS, (size_t)kMaxCond * 8 * sizeof(double)))) return st;
    if ((st = ensure(c, B_CSLOT, (size_t)kMaxCond * 2 * sizeof(int)))) return st;
    if ((st = ensure(c, B_PD, NSLOT * n * sizeof(double)))) return st;
    if ((st = ensure(c, B_PAE, NSLOT * n * sizeof(double)))) return st;
    if ((st = ensure(c, B_PAN, NSLOT * n * sizeof(double)))) return st;
    if ((st = ensure(c, B_PS, K * n * sizeof(double)))) return st;
    if ((st = ensure(c, B_PP, K * n * sizeof(double)))) return st;
    if ((st = ensure(c, B_LOADPART, loads_partials_bytes(kMaxCond, c->num_sms)))) return st;
    if ((st = ensure(c, B_LOADS, (size_t)kMaxCond * 12 * sizeof(double)))) return st;
    if ((st = ensure(c, B_RESULT, 128 * sizeof(double)))) return st;

    double base[8];
    std::memcpy(base, state->e, 4 * sizeof(double));
    std::memcpy(base + 4, state->edot, 4 * sizeof(double));
    double *conds = (double *)c->buf[B_CONDS];
    int *cslot_write = (int *)c->buf[B_CSLOT] + kMaxCond;
    double *D = (double *)c->buf[B_PD], *aE = (double *)c->buf[B_PAE], *aN = (double *)c->buf[B_PAN];
    double *S = (double *)c->buf[B_PS], *p = (double *)c->buf[B_PP];
    cudaError_t e = cudaMemsetAsync(c->buf[B_FLAGS], 0, 64, s);
    if (e != cudaSuccess) return cuda_status(e);
    // (a1) fan-out, (a2) assembly of 5 coefficient sets and 9 sources
    if ((st = launch_fanout(base, d_e, d_edot, conds, cslot_write, s, simplified ? 1 : 0))) return st;
    if ((st = launch_trig(g, (double *)c->buf[B_TRIG], s))) return st;
    if ((st = launch_assemble(g, K, conds, cslot_write, D, aE, aN, S, (const double *)c->buf[B_TRIG],
                              (int *)c->buf[B_FLAGS], NSLOT, s)))
        return st;
    // (a3) joint solve; the edot-perturbed conditions use the coefficients of condition 0.
    // zero_init = 0 warm-starts from the fields the previous step of this shape and
    // scheme left in the context (the previous Picard iterate or time step); otherwise
    // from zero.
    const int cslot_general[9] = {0, 1, 2, 3, 4, 0, 0, 0, 0};
    const int cslot_simplified[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    const int *cslot = simplified ? cslot_simplified : cslot_general;
    gmaf_solver_opts o = *opts;
    const bool warm = !opts->zero_init && c->pp_nth == g.nth && c->pp_nz == g.nz && c->pp_K == K;
    o.zero_init = warm ? 0 : 1;
    c->pp_nth = g.nth;
    c->pp_nz = g.nz;
    c->pp_K = K;
    gmaf_solve_info info{};
    const int sst = solve_joint_device(c, g.nth, g.nz, K, NSLOT, cslot, D, aE, aN, S, p, &o, &info);
    c->info = info;
    if (iters_out) *iters_out = info.iterations;
    if (sst != GMAF_OK && sst != GMAF_NOT_CONVERGED) return sst;
    // (a4) loads of the 9 conditions, (a5) Jacobian and update
    unsigned *tickets = (unsigned *)c->buf[B_LOADPART];
    double *part = (double *)((char *)c->buf[B_LOADPART] + kMaxCond * sizeof(unsigned));
    if ((st = launch_loads(g, K, conds, p, (const double *)c->buf[B_TRIG], part, tickets,
                           (double *)c->buf[B_LOADS], (int *)c->buf[B_FLAGS], c->num_sms, s)))
        return st;
    PicardIn in{};
    std::memcpy(in.base, base, sizeof base);
    std::memcpy(in.e_prev, e_prev, 4 * sizeof(double));
    std::memcpy(in.F_ext, F_ext, 4 * sizeof(double));
    in.simplified = simplified ? 1 : 0;
    if ((st = launch_picard_update((const double *)c->buf[B_LOADS], in, dt, d_e, d_edot, g.L,
                                   (double *)c->buf[B_RESULT], s)))
        return st;
    double *res = (double *)((char *)c->pinned + 20480);
    int *flag_h = (int *)((char *)c->pinned + 12288);
    e = cudaMemcpyAsync(res, c->buf[B_RESULT], kResultDoubles * sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(flag_h, c->buf[B_FLAGS], sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_status(e);
    if (loads_out) std::memcpy(loads_out, res, 12 * sizeof(double));
    if (J_out) std::memcpy(J_out, res + 12, 48 * sizeof(double));
    if (G_out) std::memcpy(G_out, res + 60, 4 * sizeof(double));
    if (*flag_h & 1) return GMAF_CONTACT;
    if (sst != GMAF_OK) return sst;
    if (res[72] != 0.0) return GMAF_NONFINITE;
    std::memcpy(state->e, res + 64, 4 * sizeof(double));
    std::memcpy(state->edot, res + 68, 4 * sizeof(double));
    return GMAF_OK;
}

extern "C" {

int gmaf_picard_step(gmaf_ctx *c, const gmaf_grid *grid, const gmaf_physics *phys,
                     const gmaf_texture *tex, gmaf_state *state, const double e_prev[4], double dt,
                     const double F_ext[4], double d_e, double d_edot, const gmaf_solver_opts *opts,
                     double loads_out[12], double J_out[48], double G_out[4], int32_t *iters_out)
{
    return picard_impl(c, grid, phys, tex, state, e_prev, dt, F_ext, d_e, d_edot, opts, loads_out,
                       J_out, G_out, iters_out, false);
}

int gmaf_picard_step_simplified(gmaf_ctx *c, const gmaf_grid *grid, const gmaf_physics *phys,
                                const gmaf_texture *tex, gmaf_state *state, double dt,
                                const double F_ext[4], double d_edot, const gmaf_solver_opts *opts,
                                double loads_out[12], double J_out[48], double G_out[4],
                                int32_t *iters_out)
{
    if (!state) return GMAF_INVALID_ARG;
    return picard_impl(c, grid, phys, tex, state, state->e, dt, F_ext, 1.0, d_edot, opts, loads_out,
                       J_out, G_out, iters_out, true);
}

}  // extern "C"
