/* node_order.c -- a plain C caller of fe_node_order (host only: no context, no device).
 *
 * Builds a strip of n squares cut into triangles, numbered so that the two rows alternate
 * far apart (row 0 first, then row 1), asks the library for its reverse Cuthill-McKee and
 * Morton renumberings, and prints for each order its bandwidth (the largest index distance
 * between two nodes of one triangle) after checking that it is a permutation.  Also checks
 * that a node id out of range is rejected with FE_EINVAL.  Exit code 0 when every check holds. */
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>

#include "femenergy.h"

static int bandwidth(int64_t ne, const int32_t* elems, const int32_t* perm, int64_t nn) {
    int32_t* inv = malloc(sizeof(int32_t) * (size_t)nn);
    if (!inv) return -1;
    for (int64_t i = 0; i < nn; ++i) inv[perm[i]] = (int32_t)i;
    int bw = 0;
    for (int64_t e = 0; e < ne; ++e)
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) {
                int d = inv[elems[3 * e + a]] - inv[elems[3 * e + b]];
                if (d > bw) bw = d;
            }
    free(inv);
    return bw;
}

static int is_permutation(const int32_t* perm, int64_t nn) {
    char* seen = calloc((size_t)nn, 1);
    if (!seen) return 0;
    int ok = 1;
    for (int64_t i = 0; i < nn && ok; ++i) {
        if (perm[i] < 0 || perm[i] >= nn || seen[perm[i]]) ok = 0;
        else seen[perm[i]] = 1;
    }
    free(seen);
    return ok;
}

int main(void) {
    const int n = 40;                       /* squares */
    const int64_t nn = 2 * (n + 1), ne = 2 * n;
    double* X = malloc(sizeof(double) * (size_t)(2 * nn));
    int32_t* E = malloc(sizeof(int32_t) * (size_t)(3 * ne));
    int32_t* perm = malloc(sizeof(int32_t) * (size_t)nn);
    if (!X || !E || !perm) return 2;
    for (int i = 0; i <= n; ++i) {          /* node i: (i, 0); node n + 1 + i: (i, 1) */
        X[2 * i] = i, X[2 * i + 1] = 0.0;
        X[2 * (n + 1 + i)] = i, X[2 * (n + 1 + i) + 1] = 1.0;
    }
    for (int i = 0; i < n; ++i) {
        const int32_t a = i, b = i + 1, c = n + 1 + i, d = n + 2 + i;
        E[6 * i + 0] = a, E[6 * i + 1] = b, E[6 * i + 2] = d;
        E[6 * i + 3] = a, E[6 * i + 4] = d, E[6 * i + 5] = c;
    }
    const int orders[3] = {FE_ORDER_NONE, FE_ORDER_RCM, FE_ORDER_MORTON};
    for (int k = 0; k < 3; ++k) {
        fe_status st = fe_node_order(2, nn, X, ne, E, orders[k], perm);
        if (st != FE_OK) {
            fprintf(stderr, "fe_node_order: %s\n", fe_last_error());
            return 1;
        }
        if (!is_permutation(perm, nn)) return 1;
        printf("order %d bandwidth %d\n", orders[k], bandwidth(ne, E, perm, nn));
    }
    E[0] = (int32_t)nn;                     /* out of range */
    if (fe_node_order(2, nn, X, ne, E, FE_ORDER_RCM, perm) != FE_EINVAL) return 1;
    free(X), free(E), free(perm);
    return 0;
}
