/*
 * Philox4x32-10 counter-based generator for the oracle (test infrastructure).
 *
 * Restated from its published definition: J. K. Salmon, M. A. Moraes,
 * R. O. Dror, D. E. Shaw, "Parallel random numbers: as easy as 1, 2, 3",
 * SC'11.  Each round multiplies counter words 0 and 2 by the Philox
 * multipliers, keeps the 32-bit high/low halves and mixes in the round key;
 * the key is bumped by the Weyl constants between rounds.  The CUDA library
 * implements the same published definition independently; both are checked
 * against the known-answer vectors of the paper's reference distribution
 * (tests/golden/philox4x32_10_kat.txt).
 *
 * Counter layout shared by both sides (a specification, not code):
 *   key  = (lo32(seed), hi32(seed))
 *   MV color charges:  ctr = (site, nucleus*n_sheets + sheet, k, 1), k = 0,1
 *                      -> 8 Gaussians (colors 0..3 from k=0, 4..7 from k=1)
 *   particle j:        ctr = (j, 0, k, 2); k = 0: uniforms (x, y, |p|, phi);
 *                      k = 1..5: 20 Gaussians, the first 18 feed the Haar matrix.
 * Uniform: u = (r + 0.5) / 2^32.  Gaussian pair (Box-Muller):
 *   g0 = sqrt(-2 ln u0) cos(2 pi u1), g1 = sqrt(-2 ln u0) sin(2 pi u1).
 */
#include <math.h>
#include "oracle.h"

#define PHILOX_M0 0xD2511F53u
#define PHILOX_M1 0xCD9E8D57u
#define PHILOX_W0 0x9E3779B9u
#define PHILOX_W1 0xBB67AE85u

void o_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; r++) {
        if (r > 0) { k0 += PHILOX_W0; k1 += PHILOX_W1; }
        uint64_t p0 = (uint64_t)PHILOX_M0 * (uint64_t)c0;
        uint64_t p1 = (uint64_t)PHILOX_M1 * (uint64_t)c2;
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

double o_u01(uint32_t r) { return ((double)r + 0.5) * (1.0 / 4294967296.0); }

void o_box_muller(uint32_t r0, uint32_t r1, double *g0, double *g1) {
    double u0 = o_u01(r0), u1 = o_u01(r1);
    double rad = sqrt(-2.0 * log(u0));
    double ang = 2.0 * M_PI * u1;
    *g0 = rad * cos(ang);
    *g1 = rad * sin(ang);
}
