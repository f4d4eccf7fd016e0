/* A plain C99 client of the library's C ABI (include/dgfs.h), used by
 * tests/test_c_client.py to check that the header compiles as C, that the
 * library links into a C program, and that a C caller gets the operator of
 * Algorithm 2 through the host-buffer entry point.
 *
 *   dgfs_client info
 *       prints the library version and two status strings, and checks that an
 *       invalid plan request is refused before any device work (no GPU needed)
 *   dgfs_client collide <precision> <in.bin> <out.bin>
 *       in.bin : int32 N, M, N_rho, S, P; float64 L; float64 masses[S];
 *                float64 (omega, alpha, d) per pair [S*S]; float64 f[P][S][N^3]
 *       out.bin: float64 Q[P][S][S][N^3] computed by dgfs_collide_host
 */
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include "dgfs.h"

static int fail(const char *what, dgfs_status s)
{
    fprintf(stderr, "%s: %s (%s)\n", what, dgfs_status_string(s), dgfs_last_error());
    return 1;
}

static int read_all(FILE *fp, void *dst, size_t size, size_t count)
{
    return fread(dst, size, count, fp) == count ? 0 : 1;
}

static int run_info(void)
{
    dgfs_plan plan = NULL;
    double masses[1] = {1.0};
    dgfs_pair pair = {0.8, 1.0, 1.0, NAN};
    dgfs_status s;
    printf("version %s\n", dgfs_version());
    printf("status %s %s\n", dgfs_status_string(DGFS_OK), dgfs_status_string(DGFS_ETIMEOUT));
    /* N = 5 is not a supported grid: refused before any device work */
    s = dgfs_plan_create(&plan, 5, 1.0, 6, 4, 1, masses, &pair, DGFS_FP64, 1, 0);
    printf("refused %d %s\n", (int)s, plan == NULL ? "null" : "non-null");
    return (s == DGFS_EINVAL || s == DGFS_EUNSUPPORTED) && plan == NULL ? 0 : 1;
}

static int run_collide(const char *prec_name, const char *in_path, const char *out_path)
{
    int hdr[5], N, M, Nrho, S, P, k;
    double L, *masses = NULL, *pp = NULL, *f64 = NULL, *Q64 = NULL;
    dgfs_pair *pairs = NULL;
    void *f = NULL, *Q = NULL;
    dgfs_precision prec;
    dgfs_plan plan = NULL;
    dgfs_status s;
    long n, nf, nq;
    int rc = 1;
    FILE *fp;

    if (strcmp(prec_name, "fp64") == 0) prec = DGFS_FP64;
    else if (strcmp(prec_name, "fp32_tc") == 0) prec = DGFS_FP32_TC;
    else return fail("unknown precision", DGFS_EINVAL);
    fp = fopen(in_path, "rb");
    if (!fp) return fail("cannot open the input", DGFS_EINVAL);
    if (read_all(fp, hdr, sizeof(int), 5) || read_all(fp, &L, sizeof(double), 1)) goto done_in;
    N = hdr[0], M = hdr[1], Nrho = hdr[2], S = hdr[3], P = hdr[4];
    n = (long)N * N * N;
    nf = (long)P * S * n;
    nq = (long)P * S * S * n;
    masses = malloc(sizeof(double) * S);
    pp = malloc(sizeof(double) * 3 * S * S);
    pairs = malloc(sizeof(dgfs_pair) * S * S);
    f64 = malloc(sizeof(double) * nf);
    Q64 = malloc(sizeof(double) * nq);
    if (!masses || !pp || !pairs || !f64 || !Q64) goto done_in;
    if (read_all(fp, masses, sizeof(double), S) || read_all(fp, pp, sizeof(double), 3 * S * S) ||
        read_all(fp, f64, sizeof(double), nf))
        goto done_in;
    fclose(fp);
    fp = NULL;
    for (k = 0; k < S * S; ++k) {
        pairs[k].omega = pp[3 * k];
        pairs[k].alpha = pp[3 * k + 1];
        pairs[k].d = pp[3 * k + 2];
        pairs[k].beta_override = NAN;
    }
    s = dgfs_plan_create(&plan, N, L, M, Nrho, S, masses, pairs, prec, P, 0);
    if (s != DGFS_OK) {
        rc = fail("dgfs_plan_create", s);
        goto done;
    }
    if (prec == DGFS_FP64) {
        f = f64;
        Q = Q64;
    } else {
        float *f32 = malloc(sizeof(float) * nf), *Q32 = malloc(sizeof(float) * nq);
        long i;
        f = f32;
        Q = Q32;
        if (!f32 || !Q32) goto done;
        for (i = 0; i < nf; ++i) f32[i] = (float)f64[i];
    }
    s = dgfs_collide_host(plan, P, f, Q, NULL);
    if (s != DGFS_OK) {
        rc = fail("dgfs_collide_host", s);
        goto done;
    }
    if (prec != DGFS_FP64) {
        long i;
        for (i = 0; i < nq; ++i) Q64[i] = (double)((float *)Q)[i];
    }
    fp = fopen(out_path, "wb");
    if (!fp || fwrite(Q64, sizeof(double), nq, fp) != (size_t)nq) {
        rc = fail("cannot write the output", DGFS_EINVAL);
        goto done;
    }
    rc = 0;
done:
    if (plan) dgfs_plan_destroy(plan);
    if (prec != DGFS_FP64) {
        free(f);
        free(Q);
    }
    if (fp) fclose(fp);
    free(masses);
    free(pp);
    free(pairs);
    free(f64);
    free(Q64);
    return rc;
done_in:
    fclose(fp);
    free(masses);
    free(pp);
    free(pairs);
    free(f64);
    free(Q64);
    return fail("cannot read the input", DGFS_EINVAL);
}

int main(int argc, char **argv)
{
    if (argc >= 2 && strcmp(argv[1], "info") == 0) return run_info();
    if (argc == 5 && strcmp(argv[1], "collide") == 0) return run_collide(argv[2], argv[3], argv[4]);
    fprintf(stderr, "usage: dgfs_client info | dgfs_client collide <fp64|fp32_tc> <in.bin> <out.bin>\n");
    return 2;
}
