/*
 * fsb_oracle.h -- plain single-threaded CPU oracle of the Fish School
 * Behaviour (FSB) per-step update.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may include, link
 * or call this code: only the tests, the smoke check and the CPU-baseline leg
 * of the benchmark use it.  It shares no code with the CUDA library.
 *
 * What it computes (paper: Sec. 2.1.1 Fish structure and initialisation,
 * Sec. 2.1.2 pond and random movement, Sec. 2.1.3 Config, Sec. 2.3.2 the
 * eat() max reduction).  The paper does not write the update rules out; the
 * readings taken where it is silent are listed in the design notes and
 * repeated next to each function in fsb_oracle.c.
 *
 * Every function exists twice: a `_f32` version whose fish state and
 * per-fish arithmetic are IEEE binary32, and a `_f64` version in binary64.
 * The file fsb_oracle.c is compiled once per precision.
 */
#ifndef FSB_ORACLE_H
#define FSB_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Sec. 2.1.3 Config: fish population, initial weight, pond dimensions.
 * Iteration counts are passed to fsbo_run_*; the OpenMP knobs are not part
 * of the method. */
typedef struct {
    uint64_t n_fish;
    uint64_t seed;            /* Philox key = (seed lo32, seed hi32) */
    uint32_t school_id;       /* folded into counter word 1 */
    int32_t  init_weight_mode;/* 0: w = w0; 1: w = w0 * (0.5 + u2) */
    double   pond_half;       /* P: pond is [-P, P]^2 (200x200 -> 100) */
    double   step;            /* s: swim half-width */
    double   w0;              /* initial weight */
    double   w_min;           /* weight floor */
    double   w_max;           /* weight cap */
    int32_t  swim_mode;       /* 0: move half-width s; 1: s * (w / w0) */
    int32_t  feed_mode;       /* 0: w += delta / max|delta|;
                                 1: w += (prev - cur) / max(prev - cur)  */
    int32_t  collective_mode; /* 1: instinctive and volitive movements
                                 after each step's eat (fish-school search) */
    double   step_vol;        /* volitive step s_vol                     */
} fsbo_config;

/* Per-step statistics. */
typedef struct {
    double max_abs_delta;  /* M_t = max_i |cur_i - prev_i| (exact)           */
    double eat_max_diff;   /* max_i (prev_i - cur_i), the paper's eat() value */
    double sum_w;          /* reference sums over the school, compensated    */
    double sum_wx;         /*   in binary64 with exact products: error below */
    double sum_wy;         /*   ~1e-15 of sum_abs_* for N <= 2^30             */
    double sum_abs_wx;     /* sum_i |w_i x_i|: normaliser of the bary error  */
    double sum_abs_wy;
    /* collective_mode 1 only (0 otherwise): the instinctive vector, the
     * barycentre the volitive move used, and W_t - W_{t-1} in grid units */
    double inst_x, inst_y;
    double vol_bx, vol_by;
    double vol_dw;
} fsbo_stats;

/* Fixed-point grid exponent of an exact school sum (collective movements):
 * the largest k in [-100, 100] with n * bound * 2^k <= 2^62 (the sum of
 * n terms bounded by `bound` stays below 2^62). */
int fsbo_grid_exponent(uint64_t n, double bound);

/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): out = bijection of ctr
 * under key.  Shared by both precisions. */
void fsbo_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2],
                        uint32_t out[4]);

/* The raw swim words (r0, r1) of fish i at step t (t >= 1): words
 * 2 (i % 2) and 2 (i % 2) + 1 of the block of fish pair i / 2.  The raw
 * init words (r0, r1, r2) of fish i: words 0, 1, 2 of its own block. */
void fsbo_swim_words(const fsbo_config* cfg, uint64_t i, uint32_t t,
                     uint32_t out[2]);
void fsbo_init_words(const fsbo_config* cfg, uint64_t i, uint32_t out[3]);
/* The volitive draw of fish i at step t (collective_mode 1): word i % 2 of
 * the domain-2 block of pair i / 2. */
uint32_t fsbo_volitive_word(const fsbo_config* cfg, uint64_t i, uint32_t t);

/* Fish state in the paper's layout (Sec. 2.1.1). */
typedef struct { float  x, y, weight, prevObjective, currentObjective; } fsbo_fish_f32;
typedef struct { double x, y, weight, prevObjective, currentObjective; } fsbo_fish_f64;

/* Initialise a school (t = 0).  Returns 0, or -1 on a bad argument. */
int fsbo_init_f32(const fsbo_config* cfg, fsbo_fish_f32* school);
int fsbo_init_f64(const fsbo_config* cfg, fsbo_fish_f64* school);

/* Advance a school from step t0 to t0 + n_steps.  `stats` (may be NULL)
 * receives n_steps records.  `draws` (may be NULL) replaces Philox: it holds
 * n_steps * n_fish * 2 raw 32-bit words, step-major, fish, then (r0, r1);
 * tests use it to inject hand-chosen draws.  Returns 0, or -1 on a bad
 * argument. */
int fsbo_run_f32(const fsbo_config* cfg, uint64_t t0, uint32_t n_steps,
                 fsbo_fish_f32* school, fsbo_stats* stats,
                 const uint32_t* draws);
int fsbo_run_f64(const fsbo_config* cfg, uint64_t t0, uint32_t n_steps,
                 fsbo_fish_f64* school, fsbo_stats* stats,
                 const uint32_t* draws);

/* fsbo_run with the per-fish loops on n_threads OpenMP threads (<= 0: the
 * OpenMP default), the multi-core CPU baseline: per-fish state and maxima
 * equal fsbo_run's bit for bit, barycentre sums to rounding.  No injected
 * draws; collective_mode 1 -> -1. */
int fsbo_run_omp_f32(const fsbo_config* cfg, uint64_t t0, uint32_t n_steps,
                     fsbo_fish_f32* school, fsbo_stats* stats, int n_threads);
int fsbo_run_omp_f64(const fsbo_config* cfg, uint64_t t0, uint32_t n_steps,
                     fsbo_fish_f64* school, fsbo_stats* stats, int n_threads);

/* One fish's positions and deltas over n_steps, starting from `fish` at
 * step t0 (positions do not depend on weights, so one fish can be followed
 * alone).  out_* hold n_steps values each; `fish` is advanced in place but
 * its weight is left untouched. */
void fsbo_track_fish_f32(const fsbo_config* cfg, uint64_t i, uint64_t t0,
                         uint32_t n_steps, fsbo_fish_f32* fish,
                         float* out_x, float* out_y, float* out_delta);
void fsbo_track_fish_f64(const fsbo_config* cfg, uint64_t i, uint64_t t0,
                         uint32_t n_steps, fsbo_fish_f64* fish,
                         double* out_x, double* out_y, double* out_delta);

/* The eat rule applied to one weight over n_steps, given that fish's
 * deltas and the school's maxima M_t.  Returns the final weight and writes
 * each step's weight to out_w (may be NULL). */
float  fsbo_eat_fish_f32(const fsbo_config* cfg, float w, uint32_t n_steps,
                         const float* delta, const double* max_abs_delta,
                         float* out_w);
double fsbo_eat_fish_f64(const fsbo_config* cfg, double w, uint32_t n_steps,
                         const double* delta, const double* max_abs_delta,
                         double* out_w);

#ifdef __cplusplus
}
#endif
#endif
