/* host_call.c -- a plain C caller of libfemenergy.so (no Python, no CUDA headers).
 *
 * Reads a mesh, a model, a load and a vector from argv[1], evaluates J(v) and the exact
 * gradient with fe_energy_gradient_host (host buffers in and out), and writes them to
 * argv[2].  Input: int64 dim, d, n_nodes, n_elems, model; double p, C1, D1; then
 * coords[n_nodes*dim] (double), elems[n_elems*(dim+1)] (int32), dirichlet[n_nodes*d] (uint8),
 * f[n_nodes*d] (double), v[n_nodes*d] (double).  Output: int64 status; double J;
 * g[n_nodes*d] (double).  Exit code 0 when every call returned FE_OK. */
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>

#include "femenergy.h"

static int rd(FILE* fp, void* p, size_t size, size_t n) { return fread(p, size, n, fp) == n; }

int main(int argc, char** argv) {
    if (argc != 3) {
        fprintf(stderr, "usage: %s input output\n", argv[0]);
        return 2;
    }
    FILE* in = fopen(argv[1], "rb");
    if (!in) return 2;
    int64_t hdr[5];
    double par[3];
    if (!rd(in, hdr, sizeof(int64_t), 5) || !rd(in, par, sizeof(double), 3)) return 2;
    const int dim = (int)hdr[0], d = (int)hdr[1], model = (int)hdr[4];
    const int64_t nn = hdr[2], ne = hdr[3], ndof = nn * d;
    double* coords = malloc(sizeof(double) * (size_t)(nn * dim));
    int32_t* elems = malloc(sizeof(int32_t) * (size_t)(ne * (dim + 1)));
    uint8_t* dir = malloc((size_t)ndof);
    double* f = malloc(sizeof(double) * (size_t)ndof);
    double* v = malloc(sizeof(double) * (size_t)ndof);
    double* g = malloc(sizeof(double) * (size_t)ndof);
    if (!coords || !elems || !dir || !f || !v || !g) return 2;
    if (!rd(in, coords, sizeof(double), (size_t)(nn * dim)) || !rd(in, elems, sizeof(int32_t), (size_t)(ne * (dim + 1))) ||
        !rd(in, dir, 1, (size_t)ndof) || !rd(in, f, sizeof(double), (size_t)ndof) ||
        !rd(in, v, sizeof(double), (size_t)ndof))
        return 2;
    fclose(in);

    fe_ctx* ctx = NULL;
    double J = 0.0;
    fe_status st = fe_create(&ctx, 0, NULL);
    if (!st) st = fe_mesh_upload(ctx, dim, d, nn, coords, ne, elems, dir, FE_ORDER_MORTON);
    if (!st) st = fe_set_model(ctx, model, par[0], par[1], par[2]);
    if (!st) st = fe_set_load(ctx, f);
    if (!st) st = fe_precompute(ctx, 1u << FE_F64);
    if (!st) st = fe_energy_gradient_host(ctx, v, &J, g);
    if (st) fprintf(stderr, "libfemenergy: %s\n", fe_last_error());
    fe_destroy(ctx);

    FILE* out = fopen(argv[2], "wb");
    if (!out) return 2;
    const int64_t s64 = st;
    fwrite(&s64, sizeof(int64_t), 1, out);
    fwrite(&J, sizeof(double), 1, out);
    fwrite(g, sizeof(double), (size_t)ndof, out);
    fclose(out);
    free(coords), free(elems), free(dir), free(f), free(v), free(g);
    return st ? 1 : 0;
}
