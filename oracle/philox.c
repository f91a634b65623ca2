/*
 * Oracle: Philox4x32-10 (test infrastructure only; see oracle.h).
 *
 * The paper draws its random numbers on the CPU and copies them to constant
 * memory (Sec. 3.1.3). The engine replaces that with a counter-based
 * generator, so the oracle implements the same generator from its published
 * definition: Salmon, Moraes, Dror, Shaw, "Parallel Random Numbers: As Easy as
 * 1, 2, 3", SC'11. One round maps (c0, c1, c2, c3) under key (k0, k1) to
 *     (hi(M1 c2) ^ c1 ^ k0,  lo(M1 c2),  hi(M0 c0) ^ c3 ^ k1,  lo(M0 c0))
 * with M0 = 0xD2511F53, M1 = 0xCD9E8D57; between rounds the key is bumped by
 * the Weyl constants (0x9E3779B9, 0xBB67AE85). Ten rounds.
 */
#include "oracle.h"

void oracle_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2],
                          uint32_t out[4])
{
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ k0;
        uint32_t n1 = (uint32_t)p1;
        uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ k1;
        uint32_t n3 = (uint32_t)p0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

void oracle_philox4x32_10_n(const uint32_t *ctr, uint64_t n, uint64_t seed,
                            uint32_t *out)
{
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    for (uint64_t i = 0; i < n; ++i)
        oracle_philox4x32_10(ctr + 4 * i, key, out + 4 * i);
}

/* Top 23 bits, centred in their cell: (r >> 9) 2^-23 + 2^-24, never 0 or 1.
 * Every such value is exact in single precision (at most 24 significant
 * bits), so a single- and a double-precision walk draw identical u. */
double oracle_uniform(uint32_t r)
{
    return (double)(r >> 9) * 0x1p-23 + 0x1p-24;
}
