/*
 * philox.c -- Philox4x32-10 for the CPU oracle (test infrastructure only).
 *
 * Counter-based generator of Salmon, Moraes, Dror and Shaw, "Parallel random
 * numbers: as easy as 1, 2, 3" (SC'11).  One round maps the counter
 * (c0, c1, c2, c3) under the round key (k0, k1) to
 *     (hi(B*c2) ^ c1 ^ k0,  lo(B*c2),  hi(A*c0) ^ c3 ^ k1,  lo(A*c0))
 * with the 32x32->64 products of the two published multipliers A, B; the key
 * is then bumped by the two published Weyl constants.  Ten rounds.
 *
 * The counter and key layout used by the fish school (which words carry the
 * fish index, school, step and domain) is the reading taken for the paper's
 * unnamed random number generator (Sec. 2.1.1, Sec. 2.1.2); it is
 * fish_counter below.
 */
#include "fsb_oracle.h"

#define PHILOX_MUL_A   0xD2511F53u
#define PHILOX_MUL_B   0xCD9E8D57u
#define PHILOX_WEYL_0  0x9E3779B9u
#define PHILOX_WEYL_1  0xBB67AE85u

void fsbo_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2],
                        uint32_t out[4])
{
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        uint64_t pa = (uint64_t)PHILOX_MUL_A * (uint64_t)c0;
        uint64_t pb = (uint64_t)PHILOX_MUL_B * (uint64_t)c2;
        uint32_t n0 = (uint32_t)(pb >> 32) ^ c1 ^ k0;
        uint32_t n1 = (uint32_t)pb;
        uint32_t n2 = (uint32_t)(pa >> 32) ^ c3 ^ k1;
        uint32_t n3 = (uint32_t)pa;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
        k0 += PHILOX_WEYL_0;
        k1 += PHILOX_WEYL_1;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Counter layout (reading of the unnamed RNG): word 0 = index low 32 bits,
 * word 1 = index high 32 bits XOR school id, word 2 = step, word 3 = domain
 * (0 = swim, 1 = initialisation, 2 = volitive move).  Key = seed.  The
 * index is the fish for the initialisation draws and the fish pair i / 2
 * for the swim and volitive draws. */
static void fish_counter(const fsbo_config* cfg, uint64_t i, uint32_t step,
                         uint32_t domain, uint32_t ctr[4], uint32_t key[2])
{
    ctr[0] = (uint32_t)i;
    ctr[1] = (uint32_t)(i >> 32) ^ cfg->school_id;
    ctr[2] = step;
    ctr[3] = domain;
    key[0] = (uint32_t)cfg->seed;
    key[1] = (uint32_t)(cfg->seed >> 32);
}

/* One swim draw serves a pair of neighbouring fish: fish 2p moves with
 * words 0 and 1 of the pair's block, fish 2p + 1 with words 2 and 3. */
void fsbo_swim_words(const fsbo_config* cfg, uint64_t i, uint32_t t,
                     uint32_t out[2])
{
    uint32_t ctr[4], key[2], r[4];
    const unsigned half = (unsigned)(i & 1u);
    fish_counter(cfg, i >> 1, t, 0u, ctr, key);
    fsbo_philox4x32_10(ctr, key, r);
    out[0] = r[2 * half];
    out[1] = r[2 * half + 1];
}

/* The volitive draw of fish i at step t (collective_mode 1): domain 2,
 * indexed by the fish pair i / 2; fish 2p takes word 0, fish 2p + 1 word 1. */
uint32_t fsbo_volitive_word(const fsbo_config* cfg, uint64_t i, uint32_t t)
{
    uint32_t ctr[4], key[2], r[4];
    fish_counter(cfg, i >> 1, t, 2u, ctr, key);
    fsbo_philox4x32_10(ctr, key, r);
    return r[i & 1u];
}

void fsbo_init_words(const fsbo_config* cfg, uint64_t i, uint32_t out[3])
{
    uint32_t ctr[4], key[2], r[4];
    fish_counter(cfg, i, 0u, 1u, ctr, key);
    fsbo_philox4x32_10(ctr, key, r);
    out[0] = r[0];
    out[1] = r[1];
    out[2] = r[2];
}
