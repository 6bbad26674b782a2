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
  uint32_t red_mask;  // reduce after every (red_mask + 1) products: the largest
                      // power of two n with n (p-1)^2 + p < 2^64 for every p of
                      // the group (16 for primes below 2^30, 4 below 2^31)
  uint32_t near30;    // every p of the group is in (2^30 - 2^10, 2^30): kernels
                      // launched for such a group reduce with mod_reduce_near30
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

// x mod p for a 32-bit x (p < 2^31) with m = floor(2^32 / p) = mu >> 32: the
// quotient estimate is at most one short; a second correction is kept as a
// margin.
__device__ __forceinline__ uint32_t mod_reduce32(uint32_t x, uint32_t p, uint32_t m) {
  uint32_t r = x - __umulhi(x, m) * p;
  if (r >= p) r -= p;
  if (r >= p) r -= p;
  return r;
}

// x mod p for any 64-bit x when 2^30 - 2^10 < p < 2^30 (the default primes),
// with c = 2^32 mod p = 4 (2^30 - p) < 2^12: two folds x -> (x >> 32) c +
// (x mod 2^32) keep the residue and leave z < 2^32 + 2^24; then q = z >> 30
// <= floor(z / p) (p < 2^30) and r = z - q p < 2^30 + 4 (2^30 - p) < 2p, so
// one conditional subtraction finishes.  r < 2^31 is exact in 32-bit
// arithmetic.
__device__ __forceinline__ uint32_t mod_reduce_near30(uint64_t x, uint32_t p, uint32_t c) {
  const uint64_t y = (uint64_t)(uint32_t)(x >> 32) * c + (uint32_t)x;
  const uint64_t z = (uint64_t)(uint32_t)(y >> 32) * c + (uint32_t)y;
  const uint32_t r = (uint32_t)z - (uint32_t)(z >> 30) * p;
  return r >= p ? r - p : r;
}

// x mod p_r of the group for any 64-bit x.  The reduction is a template
// parameter, fixed per launch from the group's near30 flag (a run-time
// branch here made the kernels compute both).
template <bool N30>
__device__ __forceinline__ uint32_t reduce64(uint64_t x, const ModGroup& mg, int r) {
  if constexpr (N30) return mod_reduce_near30(x, mg.p[r], mg.c32[r]);
  else return mod_reduce(x, mg.p[r], mg.mu[r]);
}

// Host: the constants of a group of four primes (repeat a prime to fill the
// unused slots).
inline ModGroup make_mod_group(const uint32_t (&p)[4]) {
  ModGroup m{};
  m.red_mask = 16;
  m.near30 = 1;
  for (int r = 0; r < 4; r++) {
    m.p[r] = p[r];
    m.mu[r] = ~0ull / p[r];
    m.c32[r] = (uint32_t)((1ull << 32) % p[r]);
    if (!(p[r] < (1u << 30) && p[r] > (1u << 30) - (1u << 10))) m.near30 = 0;
    const unsigned __int128 sq = (unsigned __int128)(p[r] - 1) * (p[r] - 1);
    uint32_t n = 16;
    while (n > 1 && (unsigned __int128)n * sq + p[r] >= ((unsigned __int128)1 << 64)) n >>= 1;
    if (n < m.red_mask) m.red_mask = n;
  }
  m.red_mask -= 1;
  return m;
}

}  // namespace tnc_dev
