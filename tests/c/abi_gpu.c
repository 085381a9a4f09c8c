/* Plain C99 program driving a simulation through include/lbm.h alone (host pointers): a D3Q19
 * C-S droplet, 100 steps; checks the status, mass conservation of the FP64 totals and that the
 * droplet stays a droplet (liquid at the centre, vapour in the corner). */
#include <math.h>
#include <stdio.h>
#include <stdlib.h>

#include "lbm.h"

#define CHECK(cond)                                               \
    do {                                                          \
        if (!(cond)) {                                            \
            printf("FAILED: %s (line %d)\n", #cond, __LINE__);    \
            return 1;                                             \
        }                                                         \
    } while (0)

int main(void) {
    const int n = 32;
    const double T = 0.03301504609688092, rl = 0.35813094118772437, rv = 0.009294146215100382;
    lbm_params p;
    lbm_ctx* ctx = NULL;
    double s0[4], s1[4];
    long long N = (long long)n * n * n, i;
    float *rho = malloc(sizeof(float) * N), *u = calloc(3 * N, sizeof(float));
    int x, y, z;

    lbm_default_params(&p);
    p.nx = p.ny = p.nz = n;
    p.eos = LBM_EOS_CS;
    p.eos_p[0] = 0.5; p.eos_p[1] = 4.0; p.eos_p[2] = 1.0; p.eos_p[3] = T;
    p.sigma = 0.1;
    for (z = 0; z < n; ++z)
        for (y = 0; y < n; ++y)
            for (x = 0; x < n; ++x) {
                const double r = sqrt((x - 15.5) * (x - 15.5) + (y - 15.5) * (y - 15.5) + (z - 15.5) * (z - 15.5));
                rho[((long long)z * n + y) * n + x] = (float)(0.5 * (rl + rv) - 0.5 * (rl - rv) * tanh(2.0 * (r - 8.0) / 2.0));
            }
    CHECK(lbm_create(&p, NULL, &ctx) == LBM_OK);
    CHECK(lbm_init_fields(ctx, rho, u, NULL, 0) == LBM_OK);
    CHECK(lbm_get_moments(ctx, NULL, NULL, s0, 0) == LBM_OK);
    CHECK(lbm_step(ctx, 100) == LBM_OK);
    CHECK(lbm_get_moments(ctx, rho, u, s1, 0) == LBM_OK);
    CHECK(lbm_step_count(ctx) == 100);
    CHECK(fabs(s1[0] - s0[0]) < 1e-6 * s0[0]);
    CHECK(rho[((long long)16 * n + 16) * n + 16] > 0.3f);
    CHECK(rho[0] < 0.05f);
    for (i = 0; i < 3 * N; ++i) CHECK(fabsf(u[i]) < 0.05f);
    lbm_destroy(ctx);
    free(rho);
    free(u);
    printf("ok\n");
    return 0;
}
