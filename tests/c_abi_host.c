/*
 * A plain C consumer of the library's ABI (include/xyl.h), host side only:
 * build both graph ensembles, read their CSR, create plans for every engine
 * and print what a caller needs to allocate.  Exits non-zero on any surprise.
 * Built and run by tests/test_c_abi_cpu.py; needs no GPU.
 */
#include <stdio.h>
#include <stdlib.h>

#include "xyl.h"

#define CHECK(call)                                                                       \
    do {                                                                                  \
        int rc_ = (call);                                                                 \
        if (rc_ != XYL_OK) {                                                              \
            fprintf(stderr, "%s failed: %d (%s)\n", #call, rc_, xyl_last_error());       \
            return 1;                                                                     \
        }                                                                                 \
    } while (0)

int main(void)
{
    xyl_graph *g = NULL, *b = NULL;
    CHECK(xyl_build_graph_csr(32, 6, 3.5, 1, 0, &g));
    CHECK(xyl_build_levy_bonds(32, 10.0 / 3.0, 2 * 32 * 32, XYL_PBC, 1, 0, &b));
    int32_t n, q, md, rs;
    int64_t ne;
    CHECK(xyl_graph_info(g, &n, &ne, &q, &md, &rs));
    if (n != 1024 || ne != 3 * 1024 || md != 6) return 2;
    int32_t *perm = malloc(sizeof(int32_t) * n), *row_ptr = malloc(sizeof(int32_t) * (n + 1));
    int32_t *col = malloc(sizeof(int32_t) * 2 * ne), *color_ptr = malloc(sizeof(int32_t) * (q + 1));
    CHECK(xyl_graph_export_csr(g, perm, row_ptr, col, color_ptr));
    if (row_ptr[n] != 2 * ne || color_ptr[q] != n) return 3;
    for (int i = 0; i < n; ++i)
        for (int k = row_ptr[i]; k < row_ptr[i + 1]; ++k) {
            const int j = col[k];
            if (j < 0 || j >= n || j == i || (k > row_ptr[i] && col[k - 1] >= j)) return 4;
        }
    int32_t bn, bq, bmd, brs;
    int64_t bne;
    CHECK(xyl_graph_info(b, &bn, &bne, &bq, &bmd, &brs));
    if (bn != 1024 || bne != 2048) return 5;

    double beta[4] = { 1.0, 0.8, 0.6, 0.5 }, delta[4] = { 1.0, 1.2, 1.4, 1.6 };
    xyl_sample s[2] = { { g, 0, 4, beta, delta }, { b, 1, 4, beta, delta } };
    const int engines[3] = { XYL_FP64_PLAIN, XYL_FP32_BATCHED, XYL_FP32_PLAIN };
    for (int e = 0; e < 3; ++e) {
        xyl_plan *p = NULL;
        size_t bytes = 0;
        CHECK(xyl_plan_create(s, 2, engines[e], 7, NULL, &p, &bytes));
        xyl_tuning t;
        CHECK(xyl_get_tuning(p, &t));
        printf("engine %d: workspace %zu bytes, state %zu bytes, resident %d, spin_dim %d\n", engines[e], bytes,
               xyl_state_bytes(p), t.resident, t.spin_dim);
        /* every device-side call needs a bound workspace first */
        if (xyl_sweep(p, 1, XYL_OP_MET | XYL_OP_OR, 1, NULL) != XYL_ESTATE) return 6;
        xyl_plan_free(p);
    }
    /* O(3) spins: plain engines, and the batched engine's resident shape only */
    xyl_tuning o3 = { 0, 0, 0, 0, 0, 0, 3, 0, 0 };
    xyl_plan *p = NULL;
    size_t bytes = 0;
    CHECK(xyl_plan_create(s, 2, XYL_FP32_PLAIN, 7, &o3, &p, &bytes));
    xyl_plan_free(p);
    CHECK(xyl_plan_create(s, 2, XYL_FP32_BATCHED, 7, &o3, &p, &bytes));
    if (xyl_part_count(p) != 1) return 7; /* both graphs have 1024 sites: one part */
    xyl_plan_free(p);
    o3.resident = -1;
    if (xyl_plan_create(s, 2, XYL_FP32_BATCHED, 7, &o3, &p, &bytes) != XYL_EINVAL) return 8;
    printf("ok\n");
    free(perm); free(row_ptr); free(col); free(color_ptr);
    xyl_graph_free(g);
    xyl_graph_free(b);
    return 0;
}
