// Residue arithmetic shared by the device code of libtnc.
#pragma once

#include <cstdint>

namespace tnc_dev {

// One residue group: RG <= 4 primes processed together; an entry of a tensor
// holds RG u32 residues side by side (16 bytes for RG = 4).
struct ModGroup {
  uint32_t p[4];
  uint64_t mu[4];     // floor(2^64 / p), Barrett constant
  uint32_t c32[4];    // 2^32 mod p
  uint32_t mu32[4];   // floor(2^61 / p) (used when every p is in (2^29, 2^30))
  uint32_t red_mask;  // reduce after every (red_mask + 1) products: the largest
                      // power of two n (<= 16) with n (p-1)^2 + p < 2^64 for
                      // every p of the group (16 for primes below 2^30, 4
                      // below 2^31)
  uint32_t fast;      // 1: every p of the group lies in (2^29, 2^30)
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

// x mod p for any 64-bit x and a prime 2^29 < p < 2^30, in 32-bit steps.
// Two folds of the high word (x = h 2^32 + l == h c + l, c = 2^32 mod p)
// bring x below 2^60 + 2^32 < 2^61; then a Barrett step on the top 32 bits,
// s = t >> 29 and mu32 = floor(2^61 / p), gives a quotient at most 2 short
// (s mu32 / 2^32 > s 2^29 / p - 1 and the dropped low bits add less than one
// p), so r = t - q p < 3p < 2^32 is exact in 32 bits and two conditional
// subtractions finish it.
__device__ __forceinline__ uint32_t mod_reduce_fast(uint64_t x, uint32_t p, uint32_t c32, uint32_t mu32) {
  uint64_t t = (uint64_t)(uint32_t)(x >> 32) * c32 + (uint32_t)x;  // < 2^62 + 2^32
  t = (uint64_t)(uint32_t)(t >> 32) * c32 + (uint32_t)t;           // < 2^60 + 2^32
  const uint32_t q = __umulhi((uint32_t)(t >> 29), mu32);
  uint32_t r = (uint32_t)t - q * p;
  r = min(r, r - p);
  r = min(r, r - p);
  return r;
}

// Residue r of the group: the fast path when every prime allows it (a
// warp-uniform branch on a kernel parameter).
__device__ __forceinline__ uint32_t mod_reduce_g(uint64_t x, const ModGroup& mg, int r) {
  return mg.fast ? mod_reduce_fast(x, mg.p[r], mg.c32[r], mg.mu32[r]) : mod_reduce(x, mg.p[r], mg.mu[r]);
}

// Host: the constants of a group of four primes (repeat a prime to fill the
// unused slots).
inline ModGroup make_mod_group(const uint32_t (&p)[4]) {
  ModGroup m{};
  m.red_mask = 16;
  m.fast = 1;
  for (int r = 0; r < 4; r++) {
    m.p[r] = p[r];
    m.mu[r] = ~0ull / p[r];
    m.c32[r] = (uint32_t)((1ull << 32) % p[r]);
    m.mu32[r] = (uint32_t)((1ull << 61) / p[r]);
    if (p[r] <= (1u << 29) || p[r] >= (1u << 30)) m.fast = 0;
    const unsigned __int128 sq = (unsigned __int128)(p[r] - 1) * (p[r] - 1);
    uint32_t n = 16;
    while (n > 1 && (unsigned __int128)n * sq + p[r] >= ((unsigned __int128)1 << 64)) n >>= 1;
    if (n < m.red_mask) m.red_mask = n;
  }
  m.red_mask -= 1;
  return m;
}

}  // namespace tnc_dev
