/*
 * philox.c -- Philox4x32-10 counter-based generator (oracle side).
 * TEST INFRASTRUCTURE ONLY; see sdmm_oracle.h.
 *
 * Written from the published definition: J. K. Salmon, M. A. Moraes,
 * R. O. Dror, D. E. Shaw, "Parallel Random Numbers: As Easy as 1, 2, 3",
 * SC'11.  Each of the 10 rounds multiplies two counter words by fixed
 * 32-bit constants, takes the high and low halves of the products, and
 * mixes them with the other two words and the round key; the key is bumped
 * by two Weyl constants between rounds.
 *
 * The paper under test draws its random numbers from the renderer; the
 * generator only serves the query-side benchmark.  Uniforms in [0, 1) are
 * u = (x >> 8) * 2^-24 (exact in FP32); query i uses counter (i_lo, i_hi, 0, 0)
 * and key (seed_lo, seed_hi), and takes words 0, 1, 2.
 */
#include "sdmm_oracle.h"

static const uint32_t PH_M0 = 0xD2511F53u, PH_M1 = 0xCD9E8D57u;
static const uint32_t PH_W0 = 0x9E3779B9u, PH_W1 = 0xBB67AE85u;

void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += PH_W0;
            k1 += PH_W1;
        }
        uint64_t p0 = (uint64_t)PH_M0 * (uint64_t)c0;
        uint64_t p1 = (uint64_t)PH_M1 * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

void or_uniforms(uint64_t seed, int64_t Q, float *out3)
{
    const uint32_t key[2] = { (uint32_t)seed, (uint32_t)(seed >> 32) };
    for (int64_t i = 0; i < Q; ++i) {
        const uint64_t q = (uint64_t)i;
        const uint32_t ctr[4] = { (uint32_t)q, (uint32_t)(q >> 32), 0u, 0u };
        uint32_t x[4];
        or_philox4x32_10(ctr, key, x);
        for (int c = 0; c < 3; ++c)
            out3[3 * i + c] = (float)(x[c] >> 8) * (1.0f / 16777216.0f);
    }
}
