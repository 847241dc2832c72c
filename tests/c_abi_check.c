/* c_abi_check.c -- the C-ABI used from C alone: read flat elements and points, solve with
 * one conductor at 1 V (FP64), evaluate potential and field, write the results.
 *   c_abi_check elements.bin points.bin out.bin
 * elements.bin: int64 n, then n records of nebem_element (128 bytes each)
 * points.bin:   int64 m, then m x 3 doubles
 * out.bin:      n doubles sigma, m doubles phi, 3 m doubles E
 * Exit status 0 on success; otherwise the failing call's status string is printed. */
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>

#include "nebem.h"

static int check(int rc, const char *what) {
    if (rc != NEBEM_OK) {
        fprintf(stderr, "%s: %s (%s)\n", what, nebem_status_string(rc), nebem_last_error());
        exit(1);
    }
    return rc;
}

static void *read_all(const char *path, int64_t *count, size_t item) {
    FILE *f = fopen(path, "rb");
    if (!f || fread(count, sizeof(int64_t), 1, f) != 1) {
        fprintf(stderr, "cannot read %s\n", path);
        exit(2);
    }
    void *buf = malloc((size_t)*count * item + 1);
    if (fread(buf, item, (size_t)*count, f) != (size_t)*count) {
        fprintf(stderr, "short file %s\n", path);
        exit(2);
    }
    fclose(f);
    return buf;
}

int main(int argc, char **argv) {
    if (argc != 4) {
        fprintf(stderr, "usage: %s elements.bin points.bin out.bin\n", argv[0]);
        return 2;
    }
    if (sizeof(nebem_element) != 128) {
        fprintf(stderr, "nebem_element is not 128 bytes\n");
        return 2;
    }
    int64_t n = 0, m = 0;
    nebem_element *el = (nebem_element *)read_all(argv[1], &n, sizeof(nebem_element));
    double *pts = (double *)read_all(argv[2], &m, 3 * sizeof(double));
    nebem_ctx *ctx = NULL;
    check(nebem_create(&ctx, NULL), "nebem_create");
    check(nebem_set_geometry(ctx, el, n, NULL, 0, 0), "nebem_set_geometry");
    const double volt = 1.0;
    check(nebem_set_bc(ctx, &volt, 1), "nebem_set_bc");
    double *out = (double *)malloc(sizeof(double) * (size_t)(n + 4 * m));
    nebem_solve_info info;
    check(nebem_solve(ctx, NEBEM_FP64, out, &info), "nebem_solve");
    check(nebem_eval(ctx, pts, m, out + n, out + n + m, NEBEM_FP64), "nebem_eval");
    /* an out-of-order call reports its status instead of failing silently */
    nebem_ctx *empty = NULL;
    check(nebem_create(&empty, NULL), "nebem_create");
    if (nebem_eval(empty, pts, m, out + n, out + n + m, NEBEM_FP64) != NEBEM_BAD_STATE) {
        fprintf(stderr, "eval before set_geometry did not return NEBEM_BAD_STATE\n");
        return 3;
    }
    nebem_destroy(empty);
    FILE *f = fopen(argv[3], "wb");
    if (!f || fwrite(out, sizeof(double), (size_t)(n + 4 * m), f) != (size_t)(n + 4 * m)) return 2;
    fclose(f);
    printf("residual %.3e\n", info.residual);
    nebem_destroy(ctx);
    free(out);
    free(el);
    free(pts);
    return 0;
}
