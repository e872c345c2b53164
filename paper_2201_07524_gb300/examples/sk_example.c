/*
 * The C ABI from plain C: an entropic optimal-transport problem between two
 * point clouds in the ball of radius 0.2, solved by NFFT-accelerated
 * Sinkhorn (Alg. 3) with host buffers only.
 *
 *   sk_example d n m eps iters
 *
 * Points come from a 64-bit linear congruential generator (multiplier
 * 6364136223846793005, increment 1442695040888963407, top 53 bits as a
 * uniform double) by rejection in the cube [-0.2, 0.2]^d, x first, then y;
 * weights are uniform.  Prints the value s and the row residual.
 */
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>

#include "sk.h"

static uint64_t lcg_state = 12345u;

static double uniform01(void) {
    lcg_state = lcg_state * 6364136223846793005ull + 1442695040888963407ull;
    return (double)(lcg_state >> 11) * (1.0 / 9007199254740992.0);
}

static void ball_points(double* p, int64_t n, int d) {
    for (int64_t i = 0; i < n; ++i) {
        for (;;) {
            double r2 = 0.0;
            for (int t = 0; t < d; ++t) {
                p[i * d + t] = 0.4 * uniform01() - 0.2;
                r2 += p[i * d + t] * p[i * d + t];
            }
            if (r2 <= 0.04) break;
        }
    }
}

int main(int argc, char** argv) {
    if (argc != 6) {
        fprintf(stderr, "usage: %s d n m eps iters\n", argv[0]);
        return 2;
    }
    const int d = atoi(argv[1]);
    const int64_t n = atoll(argv[2]), m = atoll(argv[3]);
    const double eps = atof(argv[4]);
    const int iters = atoi(argv[5]);
    if (d < 1 || d > 3 || n < 1 || m < 1 || iters < 0) return 2;
    double* x = malloc(sizeof(double) * (size_t)(n * d));
    double* y = malloc(sizeof(double) * (size_t)(m * d));
    double* a = malloc(sizeof(double) * (size_t)n);
    double* b = malloc(sizeof(double) * (size_t)m);
    if (!x || !y || !a || !b) return 3;
    ball_points(x, n, d);
    ball_points(y, m, d);
    for (int64_t i = 0; i < n; ++i) a[i] = 1.0 / (double)n;
    for (int64_t j = 0; j < m; ++j) b[j] = 1.0 / (double)m;

    sk_nfft_params prm;
    sk_default_params(&prm);
    sk_plan* plan = NULL;
    int st = sk_init(&plan, d, n, x, a, m, y, b, eps, 2.0, &prm, NULL);
    if (st != SK_OK) {
        fprintf(stderr, "sk_init: %s\n", sk_error_string(st));
        return 1;
    }
    sk_result res;
    st = sk_solve(plan, iters, 0.0, 10, NULL, NULL, &res, NULL);
    if (st != SK_OK) {
        fprintf(stderr, "sk_solve: %s\n", sk_error_string(st));
        sk_destroy(plan);
        return 1;
    }
    printf("s %.17g\nerr_row %.6g\niters %d\n", res.s, res.err_row, res.iters);
    sk_destroy(plan);
    free(x);
    free(y);
    free(a);
    free(b);
    return 0;
}
