/*
 * fsb_oracle.c -- plain single-threaded CPU oracle of the Fish School
 * Behaviour per-step update.  TEST INFRASTRUCTURE ONLY (see fsb_oracle.h).
 *
 * Compiled twice: with FSBO_REAL=float / FSBO_SFX=f32 and with
 * FSBO_REAL=double / FSBO_SFX=f64.  Build flags must keep IEEE semantics:
 * -O2 -ffp-contract=off -fno-fast-math (no fused multiply-add contraction,
 * no reassociation, subnormals kept).
 *
 * The method, fish by fish in index order, as the paper describes it and
 * with the readings taken where the paper is silent:
 *
 *   state  (Sec. 2.1.1)  Fish {x, y, weight, prevObjective, currentObjective}
 *   pond   (Sec. 2.1.2)  200 x 200 plane, read as [-P, P]^2 centred on the
 *                        origin, P = 100.
 *   init   (Sec. 2.1.1)  position from the random number generator, uniform
 *                        over the pond; currentObjective = Euclidean distance
 *                        to the pond centre; prevObjective = the same value;
 *                        weight = the Config's initial weight (Sec. 2.1.3),
 *                        or optionally w0 * (0.5 + u) (reading: the paper
 *                        says the weight also comes from the generator).
 *   step t (Sec. 2.1.2, and Sec. 2.2.1, which names moving and feeding as
 *          the per-step work), in order
 *     swim        random move: x += (2u0 - 1) s, y += (2u1 - 1) s, then each
 *                 coordinate clamped to [-P, P] (reading: uniform step of
 *                 half-width s, independent of weight; clamp at the bank)
 *     objective   prevObjective <- currentObjective;
 *                 currentObjective <- sqrt(x*x + y*y)
 *     delta       delta_i = currentObjective - prevObjective
 *     max         M_t = max_i |delta_i|; the paper's eat() reduction
 *                 (Sec. 2.3.2) max_i (prevObjective - currentObjective) is
 *                 reported beside it
 *     eat         if M_t > 0: weight <- clamp(weight + delta_i / M_t,
 *                 w_min, w_max) (reading: feeding normalised by the max,
 *                 capped); if M_t == 0 no fish eats
 *     barycentre  S_w = sum w, S_x = sum w x, S_y = sum w y over the
 *                 positions after this step's swim and the weights after
 *                 this step's eat (reading: weighted centre of the school)
 *
 * Variants (off by default; the paper ties a fish's movement to its weight
 * without a rule, Sec. 2.1.1 / 2.1.2, and its eat() reduces max(prev - cur),
 * Sec. 2.3.2):
 *   swim_mode 1   the move's half-width is s * (w / w0) with the fish's
 *                 weight before this step's eat: heavier fish swim farther,
 *                 a fish of weight 0 stays put
 *   feed_mode 1   feeding is normalised by the paper's eat() value
 *                 E_t = max_i (prev_i - cur_i): if E_t > 0,
 *                 w <- clamp(w + (prev - cur) / E_t, w_min, w_max); else no
 *                 fish eats
 *   collective_mode 1   after the eat and the barycentre sums, the two
 *                 collective movements of fish-school search (not in the
 *                 paper; the method family it belongs to):
 *                 instinctive  every fish moves by I = sum_{g>0} dx g /
 *                              sum_{g>0} g, g = prev - cur the fish's
 *                              improvement, dx its swim displacement
 *                 volitive     with B the barycentre after the instinctive
 *                              move and W the weight sum, each fish moves
 *                              s_vol u |x - B|^-1 (x - B) toward B if W grew
 *                              in the step, away from B otherwise
 *                 The school sums are exact fixed-point sums (collective.c),
 *                 and currentObjective becomes the final position's.
 *
 * Draws: u(r) = (r >> 8) * 2^-24 from Philox4x32-10 words (philox.c), so
 * 2u - 1 is exact in binary32.  Each arithmetic operation rounds once to
 * nearest-even in FSBO_REAL.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include "fsb_oracle.h"

#ifndef FSBO_REAL
#error "compile with -DFSBO_REAL=float -DFSBO_SFX=f32 (or double / f64)"
#endif

typedef FSBO_REAL real;

#define FSBO_CAT2(a, b) a##_##b
#define FSBO_CAT(a, b) FSBO_CAT2(a, b)
#define FN(name) FSBO_CAT(name, FSBO_SFX)
#define FISH FSBO_CAT(fsbo_fish, FSBO_SFX)

/* sqrt in the state precision: both are correctly rounded (IEEE 754). */
static real sqrt_r(real v)
{
    if (sizeof(real) == sizeof(float)) return (real)sqrtf((float)v);
    return (real)sqrt((double)v);
}

static real clamp_r(real v, real lo, real hi)
{
    return v < lo ? lo : (v > hi ? hi : v);
}

/* 2u - 1 for the draw word r, u = (r >> 8) * 2^-24.  Exact in binary32. */
static real centred_uniform(uint32_t r)
{
    real u = (real)(r >> 8) * (real)0x1p-24;
    return (real)2 * u - (real)1;
}

static real objective(real x, real y)
{
    return sqrt_r(x * x + y * y);
}

/* Neumaier-compensated binary64 sum; the products are split exactly with
 * fma so sum_w, sum_wx, sum_wy are the exact sums up to a relative error of
 * a few units in 2^-53 plus n * 2^-106 of the sum of magnitudes. */
typedef struct { double s, c; } csum;

static void csum_add(csum* a, double v)
{
    double t = a->s + v;
    if (fabs(a->s) >= fabs(v)) a->c += (a->s - t) + v;
    else                      a->c += (v - t) + a->s;
    a->s = t;
}

static void csum_add_product(csum* a, double p, double q)
{
    double hi = p * q;
    double lo = fma(p, q, -hi);
    csum_add(a, hi);
    csum_add(a, lo);
}

/* Swim of one fish at step t with draw words r0, r1 and half-width s;
 * updates the objective fields and returns delta = currentObjective -
 * prevObjective. */
static real swim_one(FISH* f, uint32_t r0, uint32_t r1, real P, real s)
{
    real nx = f->x + centred_uniform(r0) * s;
    real ny = f->y + centred_uniform(r1) * s;
    f->x = clamp_r(nx, -P, P);
    f->y = clamp_r(ny, -P, P);
    f->prevObjective = f->currentObjective;
    f->currentObjective = objective(f->x, f->y);
    return f->currentObjective - f->prevObjective;
}

static real eat_one(real w, real delta, real M, real wmin, real wmax)
{
    return clamp_r(w + delta / M, wmin, wmax);
}

/* Half-width of one fish's move: s, or s * (w / w0) in swim_mode 1. */
static real swim_width(const fsbo_config* cfg, real s, real w0, real w)
{
    if (cfg->swim_mode == 0) return s;
    return (w / w0) * s;
}

/* One term of an exact school sum: v * 2^k (exact: a power-of-two scaling)
 * rounded to the nearest integer, ties to even. */
static long long grid_term(real v, int k)
{
    if (sizeof(real) == sizeof(float))
        return llrintf((float)v * ldexpf(1.0f, k));
    return llrint((double)v * ldexp(1.0, k));
}

/* Grid exponents of the collective sums: swim products dx * g (kp),
 * improvements g (kg), weight sums w, w x, w y (kw).  The bounds hold for
 * every value the school can take (see fsbo_grid_exponent). */
static void collective_grids(const fsbo_config* cfg, int* kp, int* kg, int* kw)
{
    const double a = fmax(fmax(fabs(cfg->w_min), fabs(cfg->w_max)), 1.5 * fabs(cfg->w0));
    const double sm = cfg->swim_mode == 1 ? 2.0 * cfg->step * fmax(1.0, a / cfg->w0)
                                          : 2.0 * cfg->step;
    const double e = ldexp(1.0, -20) * fmax(cfg->pond_half, 1.0);
    const double bd = sm + e;
    *kp = fsbo_grid_exponent(cfg->n_fish, 2.0 * bd * bd);
    *kg = fsbo_grid_exponent(cfg->n_fish, 2.0 * bd);
    *kw = fsbo_grid_exponent(cfg->n_fish, 2.0 * a * fmax(cfg->pond_half, 1.0));
}

static int config_ok(const fsbo_config* cfg)
{
    if (!cfg || cfg->n_fish == 0) return 0;
    if (cfg->collective_mode != 0 && cfg->collective_mode != 1) return 0;
    if (cfg->collective_mode == 1 && !(cfg->step_vol >= 0.0)) return 0;
    if (cfg->swim_mode != 0 && cfg->swim_mode != 1) return 0;
    if (cfg->feed_mode != 0 && cfg->feed_mode != 1) return 0;
    if (cfg->swim_mode == 1 && !(cfg->w0 > 0.0)) return 0;
    if (!(cfg->pond_half > 0.0) || !(cfg->step >= 0.0)) return 0;
    if (!(cfg->w_min <= cfg->w_max)) return 0;
    if (cfg->init_weight_mode != 0 && cfg->init_weight_mode != 1) return 0;
    return 1;
}

int FN(fsbo_init)(const fsbo_config* cfg, FISH* school)
{
    if (!config_ok(cfg) || !school) return -1;
    const real P = (real)cfg->pond_half;
    const real w0 = (real)cfg->w0;
    for (uint64_t i = 0; i < cfg->n_fish; ++i) {
        uint32_t r[3];
        fsbo_init_words(cfg, i, r);
        FISH* f = &school[i];
        f->x = centred_uniform(r[0]) * P;
        f->y = centred_uniform(r[1]) * P;
        if (cfg->init_weight_mode == 0) {
            f->weight = w0;
        } else {
            real u2 = (real)(r[2] >> 8) * (real)0x1p-24;
            f->weight = w0 * ((real)0.5 + u2);
        }
        f->currentObjective = objective(f->x, f->y);
        f->prevObjective = f->currentObjective;
    }
    return 0;
}

int FN(fsbo_run)(const fsbo_config* cfg, uint64_t t0, uint32_t n_steps,
                 FISH* school, fsbo_stats* stats, const uint32_t* draws)
{
    if (!config_ok(cfg) || !school) return -1;
    if (t0 + (uint64_t)n_steps > 0xFFFFFFFFull) return -1;
    const uint64_t N = cfg->n_fish;
    const real P = (real)cfg->pond_half;
    const real s = (real)cfg->step;
    const real w0 = (real)cfg->w0;
    const real wmin = (real)cfg->w_min;
    const real wmax = (real)cfg->w_max;

    const int coll = cfg->collective_mode == 1;
    int kp = 0, kg = 0, kw = 0;
    if (coll) collective_grids(cfg, &kp, &kg, &kw);
    const real s_vol = (real)cfg->step_vol;

    real* delta = (real*)malloc(sizeof(real) * N);
    real* dxs = coll ? (real*)malloc(sizeof(real) * N) : NULL;
    real* dys = coll ? (real*)malloc(sizeof(real) * N) : NULL;
    if (!delta || (coll && (!dxs || !dys))) {
        free(delta);
        free(dxs);
        free(dys);
        return -1;
    }

    for (uint32_t k = 0; k < n_steps; ++k) {
        const uint32_t t = (uint32_t)(t0 + k + 1);

        /* the school's weight on the grid before this step's eat */
        long long w_before = 0;
        if (coll)
            for (uint64_t i = 0; i < N; ++i) w_before += grid_term(school[i].weight, kw);

        /* swim, objective, delta */
        for (uint64_t i = 0; i < N; ++i) {
            uint32_t r[2];
            if (draws) {
                r[0] = draws[((uint64_t)k * N + i) * 2 + 0];
                r[1] = draws[((uint64_t)k * N + i) * 2 + 1];
            } else {
                fsbo_swim_words(cfg, i, t, r);
            }
            const real x_before = school[i].x, y_before = school[i].y;
            delta[i] = swim_one(&school[i], r[0], r[1], P,
                                swim_width(cfg, s, w0, school[i].weight));
            if (coll) {
                dxs[i] = school[i].x - x_before;
                dys[i] = school[i].y - y_before;
            }
        }

        /* max |delta| and the paper's eat() statistic, initialised to
         * -infinity as in Sec. 2.3.2 */
        double M = 0.0;
        double eat_max = -INFINITY;
        for (uint64_t i = 0; i < N; ++i) {
            double a = fabs((double)delta[i]);
            if (a > M) M = a;
            double diff = (double)(school[i].prevObjective -
                                   school[i].currentObjective);
            if (diff > eat_max) eat_max = diff;
        }

        /* eat */
        if (cfg->feed_mode == 0 && M > 0.0) {
            const real Mr = (real)M;   /* exact: M is one of the deltas */
            for (uint64_t i = 0; i < N; ++i)
                school[i].weight = eat_one(school[i].weight, delta[i], Mr,
                                           wmin, wmax);
        } else if (cfg->feed_mode == 1 && eat_max > 0.0) {
            const real Er = (real)eat_max;  /* exact: one fish's prev - cur */
            for (uint64_t i = 0; i < N; ++i)
                school[i].weight = eat_one(school[i].weight,
                                           school[i].prevObjective -
                                               school[i].currentObjective,
                                           Er, wmin, wmax);
        }

        /* barycentre sums */
        if (stats) {
            csum sw = {0, 0}, sx = {0, 0}, sy = {0, 0};
            csum ax = {0, 0}, ay = {0, 0};
            for (uint64_t i = 0; i < N; ++i) {
                double w = (double)school[i].weight;
                double x = (double)school[i].x;
                double y = (double)school[i].y;
                csum_add(&sw, w);
                csum_add_product(&sx, w, x);
                csum_add_product(&sy, w, y);
                csum_add_product(&ax, w, fabs(x));
                csum_add_product(&ay, w, fabs(y));
            }
            stats[k].max_abs_delta = M;
            stats[k].eat_max_diff = eat_max;
            stats[k].sum_w = sw.s + sw.c;
            stats[k].sum_wx = sx.s + sx.c;
            stats[k].sum_wy = sy.s + sy.c;
            stats[k].sum_abs_wx = ax.s + ax.c;
            stats[k].sum_abs_wy = ay.s + ay.c;
            stats[k].inst_x = stats[k].inst_y = 0.0;
            stats[k].vol_bx = stats[k].vol_by = stats[k].vol_dw = 0.0;
        }

        if (coll) {
            /* collective-instinctive movement: I = sum dx g / sum g over
             * the fish that improved, from exact grid sums */
            long long nx = 0, ny = 0, den = 0;
            for (uint64_t i = 0; i < N; ++i) {
                const real g = school[i].prevObjective - school[i].currentObjective;
                if (g > 0) {
                    nx += grid_term(dxs[i] * g, kp);
                    ny += grid_term(dys[i] * g, kp);
                    den += grid_term(g, kg);
                }
            }
            real ix = 0, iy = 0;
            if (den != 0) {
                ix = (real)ldexp((double)nx / (double)den, kg - kp);
                iy = (real)ldexp((double)ny / (double)den, kg - kp);
            }
            for (uint64_t i = 0; i < N; ++i) {
                school[i].x = clamp_r(school[i].x + ix, -P, P);
                school[i].y = clamp_r(school[i].y + iy, -P, P);
            }

            /* collective-volitive movement: barycentre of the moved school
             * with its eaten weights; contract if the weight sum grew */
            long long sw = 0, sx = 0, sy = 0;
            for (uint64_t i = 0; i < N; ++i) {
                const real w = school[i].weight;
                sw += grid_term(w, kw);
                sx += grid_term(w * school[i].x, kw);
                sy += grid_term(w * school[i].y, kw);
            }
            real bx = 0, by = 0;
            if (sw != 0) {
                bx = (real)((double)sx / (double)sw);
                by = (real)((double)sy / (double)sw);
                const int contract = sw > w_before;
                for (uint64_t i = 0; i < N; ++i) {
                    FISH* f = &school[i];
                    const real u = (real)(fsbo_volitive_word(cfg, i, t) >> 8) * (real)0x1p-24;
                    const real dx = f->x - bx;
                    const real dy = f->y - by;
                    const real dist = sqrt_r(dx * dx + dy * dy);
                    if (dist > 0) {
                        const real m = (s_vol * u) / dist;
                        f->x = clamp_r(contract ? f->x - m * dx : f->x + m * dx, -P, P);
                        f->y = clamp_r(contract ? f->y - m * dy : f->y + m * dy, -P, P);
                    }
                }
            }
            for (uint64_t i = 0; i < N; ++i)
                school[i].currentObjective = objective(school[i].x, school[i].y);
            if (stats) {
                stats[k].inst_x = (double)ix;
                stats[k].inst_y = (double)iy;
                stats[k].vol_bx = (double)bx;
                stats[k].vol_by = (double)by;
                stats[k].vol_dw = (double)(sw - w_before);
            }
        }
    }
    free(delta);
    free(dxs);
    free(dys);
    return 0;
}

#ifdef _OPENMP
#include <omp.h>

/* fsbo_run's step with its per-fish loops shared among OpenMP threads, the
 * parallelisation the paper studies (Sec. 2.3): a static schedule, and the
 * two maxima taken by OpenMP max reductions (Sec. 2.3.2's reduction
 * construct).  Each fish's arithmetic is fsbo_run's, so the per-fish state
 * and both maxima equal fsbo_run's bit for bit; the barycentre sums are
 * compensated per thread and the partials added in thread order, so they
 * agree with fsbo_run's to a few units in 2^-53 of the sum of magnitudes.
 * A multi-core CPU baseline only: no injected draws and no collective
 * movements (returns -1).  n_threads <= 0 takes OpenMP's default. */
int FN(fsbo_run_omp)(const fsbo_config* cfg, uint64_t t0, uint32_t n_steps,
                     FISH* school, fsbo_stats* stats, int n_threads)
{
    if (!config_ok(cfg) || !school || cfg->collective_mode != 0) return -1;
    if (t0 + (uint64_t)n_steps > 0xFFFFFFFFull) return -1;
    const int64_t N = (int64_t)cfg->n_fish;
    const real P = (real)cfg->pond_half;
    const real s = (real)cfg->step;
    const real w0 = (real)cfg->w0;
    const real wmin = (real)cfg->w_min;
    const real wmax = (real)cfg->w_max;
    const int nt = n_threads > 0 ? n_threads : omp_get_max_threads();

    real* delta = (real*)malloc(sizeof(real) * (size_t)N);
    csum* part = (csum*)calloc((size_t)nt * 5, sizeof(csum));
    if (!delta || !part) {
        free(delta);
        free(part);
        return -1;
    }

    for (uint32_t k = 0; k < n_steps; ++k) {
        const uint32_t t = (uint32_t)(t0 + k + 1);

        /* swim, objective, delta; max |delta| and the eat() statistic */
        double M = 0.0;
        double eat_max = -INFINITY;
#pragma omp parallel for schedule(static) num_threads(nt) reduction(max : M, eat_max)
        for (int64_t i = 0; i < N; ++i) {
            uint32_t r[2];
            fsbo_swim_words(cfg, (uint64_t)i, t, r);
            delta[i] = swim_one(&school[i], r[0], r[1], P,
                                swim_width(cfg, s, w0, school[i].weight));
            const double a = fabs((double)delta[i]);
            if (a > M) M = a;
            const double diff = (double)(school[i].prevObjective -
                                         school[i].currentObjective);
            if (diff > eat_max) eat_max = diff;
        }

        /* eat */
        if (M > 0.0 && cfg->feed_mode == 0) {
            const real Mr = (real)M;
#pragma omp parallel for schedule(static) num_threads(nt)
            for (int64_t i = 0; i < N; ++i)
                school[i].weight = eat_one(school[i].weight, delta[i], Mr, wmin, wmax);
        } else if (cfg->feed_mode == 1 && eat_max > 0.0) {
            const real E = (real)eat_max;
#pragma omp parallel for schedule(static) num_threads(nt)
            for (int64_t i = 0; i < N; ++i)
                school[i].weight = eat_one(school[i].weight,
                                           school[i].prevObjective -
                                               school[i].currentObjective,
                                           E, wmin, wmax);
        }

        /* barycentre sums: one compensated partial per thread */
        if (stats) {
            memset(part, 0, sizeof(csum) * (size_t)nt * 5);
#pragma omp parallel num_threads(nt)
            {
                csum q[5] = {{0, 0}, {0, 0}, {0, 0}, {0, 0}, {0, 0}};
#pragma omp for schedule(static)
                for (int64_t i = 0; i < N; ++i) {
                    const double w = (double)school[i].weight;
                    const double x = (double)school[i].x;
                    const double y = (double)school[i].y;
                    csum_add(&q[0], w);
                    csum_add_product(&q[1], w, x);
                    csum_add_product(&q[2], w, y);
                    csum_add_product(&q[3], w, fabs(x));
                    csum_add_product(&q[4], w, fabs(y));
                }
                memcpy(&part[(size_t)omp_get_thread_num() * 5], q, sizeof(q));
            }
            csum tot[5] = {{0, 0}, {0, 0}, {0, 0}, {0, 0}, {0, 0}};
            for (int th = 0; th < nt; ++th)
                for (int j = 0; j < 5; ++j) {
                    csum_add(&tot[j], part[th * 5 + j].s);
                    csum_add(&tot[j], part[th * 5 + j].c);
                }
            memset(&stats[k], 0, sizeof(stats[k]));
            stats[k].max_abs_delta = M;
            stats[k].eat_max_diff = eat_max;
            stats[k].sum_w = tot[0].s + tot[0].c;
            stats[k].sum_wx = tot[1].s + tot[1].c;
            stats[k].sum_wy = tot[2].s + tot[2].c;
            stats[k].sum_abs_wx = tot[3].s + tot[3].c;
            stats[k].sum_abs_wy = tot[4].s + tot[4].c;
        }
    }
    free(delta);
    free(part);
    return 0;
}
#endif

/* Positions do not depend on weights only in swim_mode 0; this helper
 * follows one fish in that mode (the fish's weight is not touched). */
void FN(fsbo_track_fish)(const fsbo_config* cfg, uint64_t i, uint64_t t0,
                         uint32_t n_steps, FISH* fish, real* out_x,
                         real* out_y, real* out_delta)
{
    const real P = (real)cfg->pond_half;
    const real s = (real)cfg->step;
    for (uint32_t k = 0; k < n_steps; ++k) {
        uint32_t r[2];
        fsbo_swim_words(cfg, i, (uint32_t)(t0 + k + 1), r);
        real d = swim_one(fish, r[0], r[1], P, s);
        if (out_x) out_x[k] = fish->x;
        if (out_y) out_y[k] = fish->y;
        if (out_delta) out_delta[k] = d;
    }
}

real FN(fsbo_eat_fish)(const fsbo_config* cfg, real w, uint32_t n_steps,
                       const real* delta, const double* max_abs_delta,
                       real* out_w)
{
    const real wmin = (real)cfg->w_min;
    const real wmax = (real)cfg->w_max;
    for (uint32_t k = 0; k < n_steps; ++k) {
        if (max_abs_delta[k] > 0.0)
            w = eat_one(w, delta[k], (real)max_abs_delta[k], wmin, wmax);
        if (out_w) out_w[k] = w;
    }
    return w;
}
