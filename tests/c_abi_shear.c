/* A coupled shear run driven through the C ABI alone (include/cellfsi.h),
 * with no Python in the process: the test suite compiles this file with gcc
 * against libcellfsi.so and compares what it writes with the same run made
 * through the Python binding and with the FP64 oracle.
 *
 * Usage: c_abi_shear <in> <out> <steps>
 *   in:  int32 nx, ny, nz; double tau, u_lo, u_hi, mu, kappa, w;
 *        int32 nv, nt; double x_ref[nv][3]; double y0[nv][3]; int32 tets[nt][4]
 *   out: double positions[nv][3] after <steps> steps, then double
 *        velocity[nz][ny][nx][3]
 * Runs with the fixed-point (order-independent) spread, so that two runs of
 * the same inputs give the same bits. Exit status 0 on success; on any
 * failing call the status name and cf_last_error() go to stderr. */
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>

#include "cellfsi.h"

static cf_ctx *ctx = NULL;

static void check(cf_status s, const char *what) {
    if (s == CF_OK) return;
    fprintf(stderr, "%s failed with status %d: %s\n", what, (int)s, ctx ? cf_last_error(ctx) : "(no context)");
    if (ctx) cf_destroy(ctx);
    exit(1);
}

static void read_exact(FILE *f, void *p, size_t size, size_t n) {
    if (fread(p, size, n, f) != n) {
        fprintf(stderr, "short input\n");
        exit(2);
    }
}

int main(int argc, char **argv) {
    if (argc != 4) {
        fprintf(stderr, "usage: %s <in> <out> <steps>\n", argv[0]);
        return 2;
    }
    FILE *in = fopen(argv[1], "rb");
    if (!in) return 2;
    int32_t dims[3], counts[2];
    double par[6];
    read_exact(in, dims, sizeof(int32_t), 3);
    read_exact(in, par, sizeof(double), 6);
    read_exact(in, counts, sizeof(int32_t), 2);
    const int32_t nv = counts[0], nt = counts[1];
    const long long nodes = (long long)dims[0] * dims[1] * dims[2];
    double *x = malloc(sizeof(double) * 3 * (size_t)nv);
    double *y = malloc(sizeof(double) * 3 * (size_t)nv);
    int32_t *tets = malloc(sizeof(int32_t) * 4 * (size_t)nt);
    double *u = malloc(sizeof(double) * 3 * (size_t)nodes);
    if (!x || !y || !tets || !u) return 3;
    read_exact(in, x, sizeof(double), 3 * (size_t)nv);
    read_exact(in, y, sizeof(double), 3 * (size_t)nv);
    read_exact(in, tets, sizeof(int32_t), 4 * (size_t)nt);
    fclose(in);

    int32_t cell = -1;
    check(cf_create(&ctx, 0, NULL), "cf_create");
    check(cf_set_spread(ctx, CF_SPREAD_FIXED), "cf_set_spread");
    check(cf_lbm_init(ctx, dims[0], dims[1], dims[2], par[0], par[1], par[2], NULL), "cf_lbm_init");
    check(cf_mesh_init(ctx, nv, x, nt, tets, y, &cell), "cf_mesh_init");
    check(cf_set_material(ctx, cell, par[3], par[4], par[5]), "cf_set_material");
    check(cf_step(ctx, atoi(argv[3])), "cf_step");
    check(cf_get_positions(ctx, cell, y), "cf_get_positions");
    check(cf_get_velocity(ctx, u), "cf_get_velocity");
    cf_destroy(ctx);

    FILE *out = fopen(argv[2], "wb");
    if (!out) return 2;
    if (fwrite(y, sizeof(double), 3 * (size_t)nv, out) != 3 * (size_t)nv ||
        fwrite(u, sizeof(double), 3 * (size_t)nodes, out) != 3 * (size_t)nodes)
        return 2;
    fclose(out);
    free(x);
    free(y);
    free(tets);
    free(u);
    return 0;
}
