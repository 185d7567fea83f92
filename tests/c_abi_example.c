/*
 * A plain C caller of the library's C ABI (include/gmaf.h): one general Picard
 * iteration of a textured piston on an n_theta x n_z gap, every argument in host
 * memory, no CUDA headers and no Python.  The test-suite builds it with gcc
 * against libgmaf.so and compares what it prints with the oracle's Picard step.
 *
 *   usage: c_abi_example n_theta n_z precision     (precision 0 FP64, 1 mixed)
 *
 * Output (one line each): status and PCG iterations, the 12 loads of the base
 * condition, the generalized force G, the updated state (e, edot).
 */
#include <stdio.h>
#include <stdlib.h>

#include "gmaf.h"

int main(int argc, char **argv)
{
    if (argc != 4) {
        fprintf(stderr, "usage: %s n_theta n_z precision\n", argv[0]);
        return 2;
    }
    gmaf_grid grid = {atoi(argv[1]), atoi(argv[2])};
    const int precision = atoi(argv[3]);

    /* piston radius, gap length, clearance, viscosity, sliding speed, chamber and case pressure */
    gmaf_physics phys = {1e-2, 4e-2, 2e-5, 0.04, 5.0, 2e7, 1e5};
    /* dimples of 0.5 mm radius and 5 um depth, 20 % of the surface */
    gmaf_texture tex = {1, 5e-4, 5e-6, 0.2, 1e-4, 2e-4};
    gmaf_state state = {{2e-6, -1e-6, 3e-6, 1e-6}, {1e-5, 0.0, -2e-5, 0.0}};
    double e_prev[4];
    for (int i = 0; i < 4; ++i) e_prev[i] = state.e[i] - 2e-8;
    const double F_ext[4] = {25.0, -10.0, 4.0, 3.0};
    gmaf_solver_opts opts = {1, 1.2, 1e-12, 100000, precision, 1, 0};

    gmaf_ctx *ctx = NULL;
    int st = gmaf_create(&ctx, 0, NULL);
    if (st != GMAF_OK) {
        fprintf(stderr, "gmaf_create: %d\n", st);
        return 1;
    }
    double loads[12], J[48], G[4];
    int32_t iters = 0;
    st = gmaf_picard_step(ctx, &grid, &phys, &tex, &state, e_prev, 2.78e-4, F_ext, 2e-8, 1e-6, &opts,
                          loads, J, G, &iters);
    printf("status %d iters %d\n", st, (int)iters);
    printf("loads");
    for (int i = 0; i < 12; ++i) printf(" %.17g", loads[i]);
    printf("\nG");
    for (int i = 0; i < 4; ++i) printf(" %.17g", G[i]);
    printf("\nstate");
    for (int i = 0; i < 4; ++i) printf(" %.17g", state.e[i]);
    for (int i = 0; i < 4; ++i) printf(" %.17g", state.edot[i]);
    printf("\n");
    const int st2 = gmaf_destroy(ctx);
    return (st == GMAF_OK && st2 == GMAF_OK) ? 0 : 1;
}
