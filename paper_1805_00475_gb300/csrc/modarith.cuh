// Residue arithmetic shared by the device code of libtnc.
#pragma once

#include <cstdint>

namespace tnc_dev {

// One residue group: RG <= 4 primes processed together; an entry of a tensor
// holds RG u32 residues side by side (16 bytes for RG = 4).
struct ModGroup {
  uint32_t p[4];
  uint64_t mu[4];     // floor(2^64 / p), Barrett constant
  uint32_t red_mask;  // reduce after every (red_mask + 1) products: the largest
                      // power of two n with n (p-1)^2 + p < 2^64 for every p of
                      // the group (16 for primes below 2^30, 4 below 2^31)
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

// Host: the constants of a group of four primes (repeat a prime to fill the
// unused slots).
inline ModGroup make_mod_group(const uint32_t (&p)[4]) {
  ModGroup m{};
  m.red_mask = 16;
  for (int r = 0; r < 4; r++) {
    m.p[r] = p[r];
    m.mu[r] = ~0ull / p[r];
    const unsigned __int128 sq = (unsigned __int128)(p[r] - 1) * (p[r] - 1);
    uint32_t n = 16;
    while (n > 1 && (unsigned __int128)n * sq + p[r] >= ((unsigned __int128)1 << 64)) n >>= 1;
    if (n < m.red_mask) m.red_mask = n;
  }
  m.red_mask -= 1;
  return m;
}

}  // namespace tnc_dev
