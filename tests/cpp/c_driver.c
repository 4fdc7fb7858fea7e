/* c_driver.c -- the library called from plain C through include/fp.h (no
 * Python, no ctypes).  Mode "host": calls that need no GPU (descriptor
 * validation, the derived-quantity helpers).  Mode "trace": one brickwork
 * ensemble (n = 8, l = 4, seed 1), FP64 traces of pairs 0..15 printed as
 * "re im" lines, then F^(1..3) of 4096 pairs. */
#include <math.h>
#include <stdio.h>
#include <string.h>

#include "fp.h"

static int host_mode(void) {
    fp_ensemble_desc d;
    memset(&d, 0, sizeof d);
    d.kind = FP_PARALLEL;
    d.n = 1000;                       /* outside [2, 64] */
    d.depth_min = d.depth_max = 4;
    fp_ensemble *e = NULL;
    if (fp_ensemble_create(&d, NULL, &e) != FP_ERR_ARG || e != NULL || strlen(fp_last_error()) == 0) return 1;
    d.n = 8;
    d.depth_min = 5;                  /* depth_max < depth_min */
    if (fp_ensemble_create(&d, NULL, &e) != FP_ERR_ARG) return 2;
    double le = 0;
    if (fp_epsilon_max(2.0 + 1e-6, 2, 10, 2, &le) != FP_OK) return 3;
    /* log10(2^20 sqrt(1e-6)) = 20 log10 2 - 3 */
    if (fabs(le - (20 * log10(2.0) - 3)) > 1e-9) return 4;
    printf("host ok\n");
    return 0;
}

static int trace_mode(void) {
    fp_ensemble_desc d;
    memset(&d, 0, sizeof d);
    d.kind = FP_PARALLEL;
    d.n = 8;
    d.depth_min = d.depth_max = 4;
    d.seed = 1;
    fp_ensemble *e = NULL;
    if (fp_ensemble_create(&d, NULL, &e) != FP_OK) { fprintf(stderr, "%s\n", fp_last_error()); return 1; }
    double tr[32];
    if (fp_trace_batch(e, 0, 16, FP_PREC_FP64, tr, NULL, NULL, NULL) != FP_OK) {
        fprintf(stderr, "%s\n", fp_last_error());
        return 2;
    }
    for (int i = 0; i < 16; ++i) printf("%.17g %.17g\n", tr[2 * i], tr[2 * i + 1]);
    double F[3], se[3];
    fp_run_stats st;
    if (fp_frame_potential(e, 100, 4096, 3, 0.0, FP_PREC_FP64, F, se, &st) != FP_OK) return 3;
    printf("F %.17g %.17g %.17g pairs %llu\n", F[0], F[1], F[2], (unsigned long long)st.pairs);
    fp_ensemble_destroy(e);
    return 0;
}

int main(int argc, char **argv) {
    if (argc > 1 && strcmp(argv[1], "trace") == 0) return trace_mode();
    return host_mode();
}
