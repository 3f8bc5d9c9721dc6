/* A C client of libabp.so: the calls a program that does not use Python makes.
 * Integrates a small batch (two parameter sets of the model of arXiv 1104.2499,
 * Sec. 2) on the default device and prints, per set, the eight moments of
 * abp_reduce as hexadecimal doubles (exact bits) and the x-histogram total.
 * Usage: c_abi_client <seed>.  Exit status: 0 on success, 1 + the failing
 * call's status otherwise. */
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include "abp.h"

#define CHECK(call)                                                                    \
    do {                                                                               \
        abp_status st_ = (call);                                                       \
        if (st_ != ABP_OK) {                                                           \
            fprintf(stderr, "%s failed: %d (%s)\n", #call, (int)st_, abp_last_error(ctx)); \
            return 1 + (int)st_;                                                       \
        }                                                                              \
    } while (0)

int main(int argc, char **argv) {
    abp_ctx *ctx = NULL;
    abp_config cfg;
    memset(&cfg, 0, sizeof(cfg));
    cfg.seed = argc > 1 ? strtoull(argv[1], NULL, 10) : 7;
    cfg.dt = 1e-3;
    cfg.v0_mode = 1;
    cfg.hist_x_bins = 16;
    cfg.v_lo = -5.0;
    cfg.v_hi = 5.0;
    cfg.particles_per_thread = 2; /* fixed, so that the tiles -- and the order of the FP64 sums -- */
    cfg.schedule = 1;             /* do not depend on the autotuner's measurements */
    abp_params sets[2] = {{1.0, 0.1, 1.0, 1.0, 0.0, 0.1, 1.0, 1.0, 0.25},
                          {2.0, 0.1, 1.0, 1.0, -0.2, 0.3, 1.0, 1.0, 0.1}};
    const int64_t n_traj[2] = {1000, 517};
    const int64_t n_steps[2] = {2000, 1500};
    CHECK(abp_create(&ctx, &cfg, NULL));
    CHECK(abp_set_params(ctx, 2, sets, n_traj, n_steps));
    CHECK(abp_integrate(ctx, -1));
    double moments[2][8];
    uint32_t hist[2][16];
    CHECK(abp_reduce(ctx, &moments[0][0], &hist[0][0], NULL)); /* host outputs: the call copies and waits */
    CHECK(abp_synchronize(ctx));
    for (int s = 0; s < 2; ++s) {
        uint64_t total = 0;
        for (int b = 0; b < 16; ++b) total += hist[s][b];
        printf("set %d", s);
        for (int j = 0; j < 8; ++j) printf(" %a", moments[s][j]);
        printf(" hist %llu\n", (unsigned long long)total);
    }
    abp_destroy(ctx);
    return 0;
}
