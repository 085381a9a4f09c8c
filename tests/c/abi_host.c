/* Plain C99 client of include/lbm.h: compiles without C++ and calls the entry points that need no
 * GPU (parameter defaults, the memory estimate, argument validation, status strings). */
#include <stdio.h>
#include <string.h>

#include "lbm.h"

#define CHECK(cond)                                               \
    do {                                                          \
        if (!(cond)) {                                            \
            printf("FAILED: %s (line %d)\n", #cond, __LINE__);    \
            return 1;                                             \
        }                                                         \
    } while (0)

int main(void) {
    lbm_params p;
    size_t bytes = 0;
    lbm_ctx* ctx = NULL;
    long long n, plane, blocks, want;

    memset(&p, 0xff, sizeof p);
    lbm_default_params(&p);
    CHECK(p.lattice == 19 && p.nx == 32 && p.ny == 32 && p.nz == 32);
    CHECK(p.store == LBM_STORE_FP32 && p.onepass == 0);

    /* populations (planes padded to 64 cells), psi, status word, reduction scratch */
    p.nx = 40; p.ny = 36; p.nz = 24;
    CHECK(lbm_estimate_bytes(&p, 0, &bytes) == LBM_OK);
    n = 40LL * 36 * 24;
    plane = (n + 63) / 64 * 64;
    blocks = ((40 + 31) / 32) * ((36 + 3) / 4) * ((24 + 1) / 2);
    want = 19 * plane * 4 + n * 4 + 64 + blocks * 32 + 32;
    CHECK((long long)bytes == want);
    p.onepass = 1;
    CHECK(lbm_estimate_bytes(&p, 0, &bytes) == LBM_OK && (long long)bytes == want + 19 * plane * 4);
    p.onepass = 0;

    /* invalid parameters are rejected before any device work, with a message */
    p.lattice = 21;
    CHECK(lbm_create(&p, NULL, &ctx) == LBM_ERR_ARG && ctx == NULL);
    CHECK(strlen(lbm_last_error(NULL)) > 0);
    p.lattice = 27;
    p.nz = LBM_MAX_EXTENT + 1;
    CHECK(lbm_create(&p, NULL, &ctx) == LBM_ERR_ARG && ctx == NULL);
    CHECK(lbm_estimate_bytes(&p, 0, &bytes) == LBM_ERR_ARG);

    CHECK(strcmp(lbm_status_string(LBM_OK), "LBM_OK") == 0);
    CHECK(lbm_step(NULL, 1) == LBM_ERR_ARG);
    lbm_destroy(NULL);
    printf("ok\n");
    return 0;
}
