/* Drives every entry point of the oracle on small inputs, including
 * degenerate hits (zero radius, NaN, infinities, y = 0, huge values), for
 * a build with AddressSanitizer and UndefinedBehaviorSanitizer. */
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>

#include "ht_oracle.c"

static uint32_t lcg(uint32_t *s) { return *s = *s * 1664525u + 1013904223u; }
static float uni(uint32_t *s, float lo, float hi) { return lo + (hi - lo) * (float)(lcg(s) >> 8) / 16777216.0f; }

static int run(const uint32_t *bins, const float *rng, int64_t n, uint32_t seed)
{
    float *x = malloc(n * sizeof *x), *y = malloc(n * sizeof *y), *z = malloc(n * sizeof *z);
    for (int64_t i = 0; i < n; ++i) {
        x[i] = uni(&seed, -1100.f, 1100.f);
        y[i] = uni(&seed, -1100.f, 1100.f);
        z[i] = uni(&seed, -2500.f, 2500.f);
    }
    /* degenerate hits */
    if (n >= 8) {
        x[0] = 0.f; y[0] = 0.f;
        x[1] = NAN;
        y[2] = INFINITY;
        x[3] = 500.f; y[3] = 0.f;
        x[4] = 3e38f; y[4] = -3e38f;
        z[5] = NAN;
        x[6] = 1e-30f; y[6] = -1e-30f;
        z[7] = -INFINITY;
    }
    const uint64_t cells = (uint64_t)bins[0] * bins[1] * bins[2] * bins[3];
    uint32_t *M = calloc(cells, 4);
    float et[1025], ep[1025];
    uint32_t ma = (2 * bins[4] + 1) * (2 * bins[5] + 1);
    uint32_t *slices = malloc((size_t)n * ma * 4), *count = malloc((size_t)n * 4);
    int64_t stats[5], diffs[64 * 4];
    uint32_t ids[5 * 256];
    float cen[2 * 256];
    int bad = 0;
    bad |= ho_edges(bins, rng, et, ep) != 0;
    bad |= ho_admit_hits(bins, rng, x, y, z, n, slices, count) < 0;   /* returns the slices per hit */
    bad |= ho_fill(bins, rng, x, y, z, n, M) < 0;
    uint32_t sl[2] = {0, bins[0] * bins[1] - 1};
    uint32_t *Ms = calloc((uint64_t)2 * bins[2] * bins[3], 4);
    bad |= ho_fill_slices(bins, rng, x, y, z, n, sl, 2, Ms) < 0;
    bad |= ho_find_maxima(bins, rng, M, 2, ids, cen, 256) < 0;
    bad |= ho_find_maxima4d(bins, rng, M, 2, ids, cen, 256) < 0;
    bad |= ho_bins_f32_vs_f64(bins, rng, x, y, z, n, stats, diffs, 64) != 0;
    free(x); free(y); free(z); free(M); free(Ms); free(slices); free(count);
    return bad;
}

int main(void)
{
    const float full[8] = {0.f, 3.14159274f, -3.14159274f, 3.14159274f, -2000.f, 2000.f, -2000.f, 2000.f};
    const float part[8] = {0.4f, 2.6f, -2.0f, 1.5f, -1500.f, 1700.f, -900.f, 2100.f};
    const uint32_t b1[6] = {2, 4, 64, 64, 0, 0}, b2[6] = {3, 5, 37, 29, 1, 1}, b3[6] = {1, 1, 8, 8, 0, 0};
    int bad = run(b1, full, 400, 1u) | run(b2, part, 300, 2u) | run(b3, full, 50, 3u) | run(b2, full, 8, 4u);
    /* an invalid binning is refused, not read past */
    const uint32_t b0[6] = {0, 4, 64, 64, 0, 0};
    float et[8], ep[8];
    bad |= ho_edges(b0, full, et, ep) == 0;
    printf(bad ? "FAIL\n" : "OK\n");
    return bad;
}
