/* A plain C99 consumer of the library's C ABI (include/colatus.h): no C++,
 * no Python.  It reads a system from a binary file, evaluates the Eq. 1
 * acceleration, advances nsteps KDK steps with FP32 compensated forces, and
 * writes the acceleration, the final state, (t, a) and the diagnostics.
 *
 *     c_client <in> <out>
 *
 * in:  int64 N, int64 nsteps, double eps, double a_start, double tau,
 *      N doubles (masses), N x 3 floats (x), N x 3 floats (v)
 * out: N x 3 floats (acceleration at the initial state), N x 3 floats (x),
 *      N x 3 floats (v), double t, double a, COLATUS_NDIAG doubles
 *
 *     c_client selftest
 *
 * runs the host-only self-tests of the pair-once scheduling tables (no GPU):
 * the 32^3 force plan (2048-body tiles, 32 sub-phases, 147 CTAs) and the
 * ensemble plan of four realisations, and prints each one's five figures.
 *
 * Exit status: 0 on success, 1 on a file error, 2 + the colatus_status of
 * the first failing call otherwise (its message goes to stderr). */
#include <stdio.h>
#include <stdlib.h>

#include "colatus.h"

static int fail(colatus_t ctx, const char *what, colatus_status st) {
    fprintf(stderr, "%s: status %d: %s\n", what, (int)st, colatus_last_error(ctx));
    colatus_destroy(ctx);
    return 2 + (int)st;
}

static int read_all(FILE *f, void *p, size_t size, size_t n) {
    return fread(p, size, n, f) == n;
}

int main(int argc, char **argv) {
    FILE *in, *out;
    int64_t N, nsteps;
    double eps, a_start, tau, t, a, diag[COLATUS_NDIAG];
    double *m;
    float *x, *v, *acc;
    colatus_t ctx = NULL;
    colatus_status st;
    int ok;

    if (argc == 2 && argv[1][0] == 's') {
        int64_t r[5];
        const int64_t sizes[4] = {1028, 4096, 4097, 32675};
        st = colatus_selftest_sym_tables(32768, 2048, 32, 147, 11, 14, r);
        if (st != COLATUS_OK) return fail(NULL, "colatus_selftest_sym_tables", st);
        printf("sym %lld %lld %lld %lld %lld\n", (long long)r[0], (long long)r[1], (long long)r[2],
               (long long)r[3], (long long)r[4]);
        st = colatus_selftest_ens_sym_tables(4, sizes, 592, 11, 14, r);
        if (st != COLATUS_OK) return fail(NULL, "colatus_selftest_ens_sym_tables", st);
        printf("ens %lld %lld %lld %lld %lld\n", (long long)r[0], (long long)r[1], (long long)r[2],
               (long long)r[3], (long long)r[4]);
        return 0;
    }
    if (argc != 3) {
        fprintf(stderr, "usage: %s <in> <out> | %s selftest\n", argv[0], argv[0]);
        return 1;
    }
    in = fopen(argv[1], "rb");
    if (!in) return 1;
    ok = read_all(in, &N, sizeof N, 1) && read_all(in, &nsteps, sizeof nsteps, 1) &&
         read_all(in, &eps, sizeof eps, 1) && read_all(in, &a_start, sizeof a_start, 1) &&
         read_all(in, &tau, sizeof tau, 1) && N > 0;
    if (!ok) {
        fclose(in);
        return 1;
    }
    m = (double *)malloc((size_t)N * sizeof(double));
    x = (float *)malloc((size_t)N * 3 * sizeof(float));
    v = (float *)malloc((size_t)N * 3 * sizeof(float));
    acc = (float *)malloc((size_t)N * 3 * sizeof(float));
    if (!m || !x || !v || !acc) return 1;
    ok = read_all(in, m, sizeof(double), (size_t)N) && read_all(in, x, sizeof(float), (size_t)N * 3) &&
         read_all(in, v, sizeof(float), (size_t)N * 3);
    fclose(in);
    if (!ok) return 1;

    /* flat LCDM (Omega_M = 0.3, Omega_L = 0.7), H0 = G = 1 */
    st = colatus_init(&ctx, N, m, eps, 0.0, 0.3, 0.0, 0.7, 1.0, a_start);
    if (st != COLATUS_OK) return fail(NULL, "colatus_init", st);
    st = colatus_set_config(ctx, COLATUS_FP32_COMP, COLATUS_KDK, 1.0, NULL);
    if (st != COLATUS_OK) return fail(ctx, "colatus_set_config", st);
    st = colatus_set_state(ctx, x, v, COLATUS_F32, 0);
    if (st != COLATUS_OK) return fail(ctx, "colatus_set_state", st);
    st = colatus_forces(ctx, acc, COLATUS_F32, 0);
    if (st != COLATUS_OK) return fail(ctx, "colatus_forces", st);
    st = colatus_step(ctx, tau, nsteps);
    if (st != COLATUS_OK) return fail(ctx, "colatus_step", st);
    st = colatus_get_state(ctx, x, v, COLATUS_F32, 0, &t, &a);
    if (st != COLATUS_OK) return fail(ctx, "colatus_get_state", st);
    st = colatus_diagnostics(ctx, diag);
    if (st != COLATUS_OK) return fail(ctx, "colatus_diagnostics", st);
    colatus_destroy(ctx);

    out = fopen(argv[2], "wb");
    if (!out) return 1;
    ok = fwrite(acc, sizeof(float), (size_t)N * 3, out) == (size_t)N * 3 &&
         fwrite(x, sizeof(float), (size_t)N * 3, out) == (size_t)N * 3 &&
         fwrite(v, sizeof(float), (size_t)N * 3, out) == (size_t)N * 3 &&
         fwrite(&t, sizeof t, 1, out) == 1 && fwrite(&a, sizeof a, 1, out) == 1 &&
         fwrite(diag, sizeof(double), COLATUS_NDIAG, out) == COLATUS_NDIAG;
    fclose(out);
    free(m);
    free(x);
    free(v);
    free(acc);
    return ok ? 0 : 1;
}
