/*
 * collective.c -- helpers of the collective movements (fish-school search
 * variant, collective_mode 1) shared by both precisions of the oracle.
 * TEST INFRASTRUCTURE ONLY (see fsb_oracle.h).
 *
 * Exact school sums use a fixed grid: each term v becomes the integer
 * nearest to v * 2^k (ties to even), and integers add exactly in any order
 * (reproducible summation by pre-rounding, after Demmel and Nguyen, with a
 * grid fixed by the school's configuration).  The grid exponent k is the
 * largest integer in [-100, 100] with n * bound * 2^k <= 2^62: the sum of n
 * terms bounded by `bound` stays below 2^62 in magnitude.
 */
#include "fsb_oracle.h"

int fsbo_grid_exponent(uint64_t n, double bound)
{
    const double lim = 4611686018427387904.0;  /* 2^62 */
    double t = (double)n * bound;
    int k = 0;
    if (t > lim) {
        while (t > lim && k > -100) {
            t *= 0.5;
            --k;
        }
        return k;
    }
    while (2.0 * t <= lim && k < 100) {
        t *= 2.0;
        ++k;
    }
    return k;
}
