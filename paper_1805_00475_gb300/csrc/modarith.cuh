// Residue arithmetic shared by the device code of libtnc.
#pragma once

#include <cstdint>

namespace tnc_dev {

// One residue group: RG <= 4 primes processed together; an entry of a tensor
// holds RG u32 residues side by side (16 bytes for RG = 4).
//
// Tensor entries are held in Montgomery form, a R mod p with R = 2^32: the
// product of two such residues is a b R^2, and a sum x < p R of such products
// reduces to (sum a b) R mod p by one Montgomery reduction (REDC: four
// integer operations, against about fifteen for a Barrett reduction of a
// 64-bit value).  Leaves enter the form once (v -> v R mod p) and results
// leave it once (REDC of the residue).
struct ModGroup {
  uint32_t p[4];
  uint64_t mu[4];     // floor(2^64 / p), Barrett constant (sums, conversions)
  uint32_t pinv[4];   // -p^{-1} mod 2^32
  uint32_t r1[4];     // R mod p
  uint32_t red_mask;  // products per REDC minus one: the largest power of two n
                      // <= 16 with n (p-1)^2 < p R for every p of the group
                      // (4 for primes below 2^30, 2 below 2^31)
  uint32_t pad;
};

// x mod p for any 64-bit x (Barrett reduction with mu = floor(2^64/p):
// the quotient estimate is at most one short, so one correction suffices;
// a second one is kept as a margin).
__device__ __forceinline__ uint32_t mod_reduce(uint64_t x, uint32_t p, uint64_t mu) {
  const uint64_t q = __umul64hi(x, mu);
  uint64_t r = x - q * (uint64_t)p;
  if (r >= p) r -= p;
  if (r >= p) r -= p;
  return (uint32_t)r;
}

// Montgomery reduction: x R^{-1} mod p for x < p R (odd p < 2^31).  m makes
// x + m p divisible by R; (x + m p) / R < 2p.
__device__ __forceinline__ uint32_t redc(uint64_t x, uint32_t p, uint32_t pinv) {
  const uint32_t m = (uint32_t)x * pinv;
  const uint32_t t = (uint32_t)(((uint64_t)m * p + x) >> 32);
  return t >= p ? t - p : t;
}

__device__ __forceinline__ uint32_t add_mod(uint32_t a, uint32_t b, uint32_t p) {
  const uint32_t s = a + b;  // a, b < p < 2^31
  return s >= p ? s - p : s;
}

// v R mod p: a value (below 2^32) into Montgomery form.
__device__ __forceinline__ uint32_t to_mont(uint32_t v, const ModGroup& mg, int r) {
  return mod_reduce((uint64_t)v * mg.r1[r], mg.p[r], mg.mu[r]);
}

// Host: the constants of a group of four primes (repeat a prime to fill the
// unused slots).
inline ModGroup make_mod_group(const uint32_t (&p)[4]) {
  ModGroup m{};
  m.red_mask = 16;
  for (int r = 0; r < 4; r++) {
    m.p[r] = p[r];
    m.mu[r] = ~0ull / p[r];
    uint32_t inv = p[r];  // Newton: inv = p^{-1} mod 2^32 (p odd)
    for (int i = 0; i < 5; i++) inv *= 2u - p[r] * inv;
    m.pinv[r] = 0u - inv;
    m.r1[r] = (uint32_t)((1ull << 32) % p[r]);
    const unsigned __int128 sq = (unsigned __int128)(p[r] - 1) * (p[r] - 1);
    uint32_t n = 16;
    while (n > 1 && (unsigned __int128)n * sq >= (unsigned __int128)p[r] << 32) n >>= 1;
    if (n < m.red_mask) m.red_mask = n;
  }
  m.red_mask -= 1;
  return m;
}

}  // namespace tnc_dev
