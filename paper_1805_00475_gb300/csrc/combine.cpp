// Host-side combine of residues computed in several processes: Garner's
// mixed-radix Chinese remaindering (the exact counts of Sec. 3.2 rebuilt from
// residues) and the modular sum of slices' residues (bond slicing splits the
// trace of Eq. z into a sum).  A process that counted modulo its own subset
// of the primes, or its own subset of the slices, sends its small residue
// array; the host adds or remainders them.  Pure host code, no device work.
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "tnc_internal.h"

namespace {

uint32_t mulmod(uint32_t a, uint32_t b, uint32_t p) { return (uint32_t)((uint64_t)a * b % p); }

uint32_t powmod(uint32_t a, uint64_t e, uint32_t p) {
  uint32_t r = 1 % p;
  a %= p;
  while (e) {
    if (e & 1) r = mulmod(r, a, p);
    a = mulmod(a, a, p);
    e >>= 1;
  }
  return r;
}

int check_primes(const uint32_t* primes, int R) {
  using tnc::set_error;
  if (!primes || R < 1 || R > 64) return set_error(TNC_ERR_INVALID, "need 1..64 primes");
  for (int i = 0; i < R; i++) {
    if (primes[i] < 3 || primes[i] >= (1u << 31) || !tnc::is_prime_u32(primes[i]))
      return set_error(TNC_ERR_INVALID, "primes must be odd primes below 2^31");
    for (int j = 0; j < i; j++)
      if (primes[j] == primes[i]) return set_error(TNC_ERR_INVALID, "primes must be distinct");
  }
  return TNC_OK;
}

}  // namespace

extern "C" int tnc_crt_host(const uint32_t* primes, int32_t R, const uint32_t* residues, int64_t n, uint32_t* limbs,
                            int32_t cap_limbs, int32_t* n_limbs) {
  using namespace tnc;
  clear_error();
  int rc = check_primes(primes, R);
  if (rc) return rc;
  if (n < 0 || (n > 0 && (!residues || !limbs))) return set_error(TNC_ERR_INVALID, "NULL argument");
  double bits = 0;
  for (int i = 0; i < R; i++) bits += std::log2((double)primes[i]);
  const int need = (int)(bits / 32.0) + 1;  // prod p < 2^(32 need)
  if (n_limbs) *n_limbs = need;
  if (cap_limbs < need) return set_error(TNC_ERR_BUFFER, "need " + std::to_string(need) + " limbs");
  // inv[i] = (p0 ... p_{i-1})^{-1} mod p_i
  std::vector<uint32_t> inv(R, 1);
  for (int i = 1; i < R; i++) {
    uint32_t prod = 1;
    for (int j = 0; j < i; j++) prod = mulmod(prod, primes[j] % primes[i], primes[i]);
    inv[i] = powmod(prod, primes[i] - 2, primes[i]);
  }
  std::vector<uint32_t> v(R);
  std::vector<uint32_t> x(need);
  for (int64_t e = 0; e < n; e++) {
    const uint32_t* r = residues + e * R;
    for (int i = 0; i < R; i++) {
      const uint32_t p = primes[i];
      const uint32_t ri = r[i] % p;
      // t = v0 + v1 p0 + ... + v_{i-1} p0..p_{i-2}  (mod p), by Horner
      uint32_t t = 0;
      for (int j = i - 1; j >= 0; j--) t = (uint32_t)(((uint64_t)t * (primes[j] % p) + v[j]) % p);
      v[i] = mulmod(ri >= t ? ri - t : ri + (p - t), inv[i], p);
    }
    std::fill(x.begin(), x.end(), 0u);
    x[0] = v[R - 1];
    for (int i = R - 2; i >= 0; i--) {  // X = v_i + p_i X
      uint64_t carry = v[i];
      for (int l = 0; l < need; l++) {
        const uint64_t t = (uint64_t)x[l] * primes[i] + carry;
        x[l] = (uint32_t)t;
        carry = t >> 32;
      }
    }
    std::memcpy(limbs + e * cap_limbs, x.data(), need * sizeof(uint32_t));
    for (int l = need; l < cap_limbs; l++) limbs[e * cap_limbs + l] = 0;
  }
  return TNC_OK;
}

extern "C" int tnc_residue_add_host(const uint32_t* primes, int32_t R, uint32_t* acc, const uint32_t* src, int64_t n) {
  using namespace tnc;
  clear_error();
  int rc = check_primes(primes, R);
  if (rc) return rc;
  if (n < 0 || (n > 0 && (!acc || !src))) return set_error(TNC_ERR_INVALID, "NULL argument");
  for (int64_t i = 0; i < n * R; i++) {
    const uint32_t p = primes[i % R];
    acc[i] = (uint32_t)(((uint64_t)(acc[i] % p) + src[i] % p) % p);
  }
  return TNC_OK;
}
