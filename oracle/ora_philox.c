/* Philox4x32-10 counter-based generator of the oracle (test infrastructure; see
 * oracle.h), written from its published
 * definition (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as
 * 1, 2, 3", SC'11): ten rounds of two 32x32->64 multiplications with the
 * round constants 0xD2511F53 and 0xCD9E8D57, the key bumped by the Weyl
 * constants 0x9E3779B9 and 0xBB67AE85 between rounds.
 * The random points of the Monte Carlo sum (Sec. 2, Eq. "sum") are drawn from it.
 * Part of the test oracle (see oracle.h). */
#include "oracle.h"

static void mulhilo32(uint32_t a, uint32_t b, uint32_t* hi, uint32_t* lo) {
  uint64_t p = (uint64_t)a * (uint64_t)b;
  *hi = (uint32_t)(p >> 32);
  *lo = (uint32_t)p;
}

void ora_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int r = 0; r < 10; ++r) {
    if (r > 0) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    uint32_t hi0, lo0, hi1, lo1;
    mulhilo32(0xD2511F53u, c0, &hi0, &lo0);
    mulhilo32(0xCD9E8D57u, c2, &hi1, &lo1);
    uint32_t n0 = hi1 ^ c1 ^ k0;
    uint32_t n1 = lo1;
    uint32_t n2 = hi0 ^ c3 ^ k1;
    uint32_t n3 = lo0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* 23 random bits: ((x >> 9) + 0.5) 2^-23 = (2k+1) 2^-24 is exactly representable
 * in FP32 over all of (0,1) (a 24-bit version would need 25 mantissa bits above 1/2). */
double ora_u01(uint32_t x) { return ((double)(x >> 9) + 0.5) * (1.0 / 8388608.0); }

/* Counter layout: (point index, draw block << 8 | stream tag, event id, perm);
 * key = (seed low word, seed high word). Stream tags: 0 = integration on the
 * VEGAS grid, 2 = base draws of the learned sampler. Draw block b supplies
 * dimensions 4b .. 4b+3. */
void ora_point_u_tag(uint64_t seed, uint64_t event_id, int perm, uint64_t idx, int d, int tag,
                     double* u) {
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  for (int b = 0; 4 * b < d; ++b) {
    uint32_t ctr[4] = {(uint32_t)idx, (uint32_t)(b << 8) | (uint32_t)(tag & 0xff),
                       (uint32_t)event_id, (uint32_t)perm};
    uint32_t o[4];
    ora_philox4x32_10(ctr, key, o);
    for (int j = 0; j < 4 && 4 * b + j < d; ++j) u[4 * b + j] = ora_u01(o[j]);
  }
}

void ora_point_u(uint64_t seed, uint64_t event_id, int perm, uint64_t idx, int d, double* u) {
  ora_point_u_tag(seed, event_id, perm, idx, d, 0, u);
}
