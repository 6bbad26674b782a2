// Device code of libtnc: modular arithmetic, leaf tensors, the fused
// permute-and-multiply step, the persistent batch kernel and the CRT.
#pragma once

#include <cstdint>
#include <type_traits>

#include "modarith.cuh"
#include "step_desc.h"

namespace tnc_dev {

// An entry holds the RG residues of its group side by side, one word W per
// residue: u32 words for primes below 2^31, bytes for the 8-bit primes of the
// TNC_PATH_TC_P8 arithmetic (four residues in one 32-bit word).
template <int RG, typename W = uint32_t>
__device__ __forceinline__ void load_entry(const W* src, uint32_t (&v)[RG]) {
  if constexpr (sizeof(W) == 1) {
    if constexpr (RG == 4) {
      const uint32_t t = *reinterpret_cast<const uint32_t*>(src);
      v[0] = t & 0xFFu; v[1] = (t >> 8) & 0xFFu; v[2] = (t >> 16) & 0xFFu; v[3] = t >> 24;
    } else if constexpr (RG == 2) {
      const uint32_t t = *reinterpret_cast<const uint16_t*>(src);
      v[0] = t & 0xFFu; v[1] = t >> 8;
    } else {
      v[0] = *src;
    }
  } else if constexpr (RG == 4) {
    const uint4 t = *reinterpret_cast<const uint4*>(src);
    v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
  } else if constexpr (RG == 2) {
    const uint2 t = *reinterpret_cast<const uint2*>(src);
    v[0] = t.x; v[1] = t.y;
  } else {
    v[0] = *src;
  }
}

// (byte words: every residue is below 2^8)
template <int RG, typename W = uint32_t>
__device__ __forceinline__ void store_entry(W* dst, const uint32_t (&v)[RG]) {
  if constexpr (sizeof(W) == 1) {
    if constexpr (RG == 4) {
      *reinterpret_cast<uint32_t*>(dst) = v[0] | (v[1] << 8) | (v[2] << 16) | (v[3] << 24);
    } else if constexpr (RG == 2) {
      *reinterpret_cast<uint16_t*>(dst) = (uint16_t)(v[0] | (v[1] << 8));
    } else {
      dst[0] = (W)v[0];
    }
  } else if constexpr (RG == 4) {
    *reinterpret_cast<uint4*>(dst) = make_uint4(v[0], v[1], v[2], v[3]);
  } else if constexpr (RG == 2) {
    *reinterpret_cast<uint2*>(dst) = make_uint2(v[0], v[1]);
  } else {
    dst[0] = v[0];
  }
}

// Operand addresses of output entry o (descriptor in global or shared memory).
__device__ __forceinline__ void map_addr(const StepDesc& d, uint64_t o, uint64_t& ia, uint64_t& ib) {
  ia = 0;
  ib = 0;
  if (d.nra != TNC_BITMAP) {
    for (int i = 0; i < d.nra; i++) {
      const TncRun r = d.map.runs.ra[i];
      ia |= ((o >> r.src) & ((1ull << r.len) - 1ull)) << r.dst;
    }
    for (int i = 0; i < d.nrb; i++) {
      const TncRun r = d.map.runs.rb[i];
      ib |= ((o >> r.src) & ((1ull << r.len) - 1ull)) << r.dst;
    }
  } else {
    for (int j = 0; j < d.c; j++) {
      const uint32_t m = d.map.bit[j];
      const uint64_t bit = ((o >> j) & 1ull) << (m & 63u);
      if (m & 0x80u) ib |= bit;
      else ia |= bit;
    }
  }
}

// Leaf tensor entry (Sec. 2.1, Sec. 3.2): COPY (Eq. var; rank 0 is the sum
// over the variable's two values, 2), exactly-one (Eq. 1in3), OR (Eq. or),
// NAND, or an explicit table already permuted to the leaf's layout.
__device__ __forceinline__ uint32_t leaf_value(uint32_t kind, uint32_t rank, uint32_t idx,
                                               const uint32_t* tables, uint32_t toff, uint32_t p) {
  const uint32_t all = (uint32_t)((1ull << rank) - 1ull);
  switch (kind) {
    case 0: return __popc(idx) == 1 ? 1u : 0u;
    case 1: return idx != 0u ? 1u : 0u;
    case 2: return idx != all ? 1u : 0u;
    case 3: return tables[toff + idx] % p;
    default: return rank == 0 ? 2u : ((idx == 0u || idx == all) ? 1u : 0u);
  }
}

// Sum over the 2^k shared-bond values of A*B for every residue of the group
// (A, B point at the operands' first shared-bond entry; consecutive shared
// values are 2^ka and 2^kb entries apart).  A product of residues is below
// (p-1)^2, so red_mask+1 of them plus a reduced partial sum fit in 64 bits:
// reduce after every (red_mask+1)-th product and once at the end.
template <int RG, typename W = uint32_t, bool N30 = false>
__device__ __forceinline__ void step_sum(uint32_t k, uint32_t ka, uint32_t kb, const W* A, const W* B,
                                         const ModGroup& mg, uint32_t (&out)[RG]) {
  const uint64_t sa = (uint64_t)RG << ka, sb = (uint64_t)RG << kb;
  const uint32_t K = 1u << k;
  if constexpr (sizeof(W) == 1) {
    // byte residues (primes <= 251): a product is below 2^16, so red_mask + 1
    // <= 16 of them plus a reduced sum stay below 2^32 -- 32-bit multiply-adds
    uint32_t acc[RG];
#pragma unroll
    for (int r = 0; r < RG; r++) acc[r] = 0;
    uint32_t q = 0;
    for (; q + 4 <= K; q += 4) {
#pragma unroll
      for (int u = 0; u < 4; u++) {
        uint32_t va[RG], vb[RG];
        load_entry<RG, W>(A + (uint64_t)(q + u) * sa, va);
        load_entry<RG, W>(B + (uint64_t)(q + u) * sb, vb);
#pragma unroll
        for (int r = 0; r < RG; r++) acc[r] += va[r] * vb[r];
      }
      if (((q + 4) & mg.red_mask) == 0) {
#pragma unroll
        for (int r = 0; r < RG; r++) acc[r] = mod_reduce32(acc[r], mg.p[r], (uint32_t)(mg.mu[r] >> 32));
      }
    }
    for (; q < K; q++) {
      uint32_t va[RG], vb[RG];
      load_entry<RG, W>(A + (uint64_t)q * sa, va);
      load_entry<RG, W>(B + (uint64_t)q * sb, vb);
#pragma unroll
      for (int r = 0; r < RG; r++) acc[r] += va[r] * vb[r];
    }
#pragma unroll
    for (int r = 0; r < RG; r++) out[r] = mod_reduce32(acc[r], mg.p[r], (uint32_t)(mg.mu[r] >> 32));
    return;
  }
  uint64_t acc[RG];
#pragma unroll
  for (int r = 0; r < RG; r++) acc[r] = 0;
  uint32_t q = 0;
  for (; q + 4 <= K; q += 4) {
#pragma unroll
    for (int u = 0; u < 4; u++) {
      uint32_t va[RG], vb[RG];
      load_entry<RG, W>(A + (uint64_t)(q + u) * sa, va);
      load_entry<RG, W>(B + (uint64_t)(q + u) * sb, vb);
#pragma unroll
      for (int r = 0; r < RG; r++) acc[r] += (uint64_t)va[r] * vb[r];
    }
    if (((q + 4) & mg.red_mask) == 0) {
#pragma unroll
      for (int r = 0; r < RG; r++) acc[r] = reduce64<N30>(acc[r], mg, r);
    }
  }
  for (; q < K; q++) {  // K < 4 here: at most 3 products on a reduced sum
    uint32_t va[RG], vb[RG];
    load_entry<RG, W>(A + (uint64_t)q * sa, va);
    load_entry<RG, W>(B + (uint64_t)q * sb, vb);
#pragma unroll
    for (int r = 0; r < RG; r++) acc[r] += (uint64_t)va[r] * vb[r];
  }
#pragma unroll
  for (int r = 0; r < RG; r++) out[r] = reduce64<N30>(acc[r], mg, r);
}

// A partial sum reduced mod p_r: 64-bit sums by reduce64, 32-bit sums (byte
// residues) by a 32-bit Barrett step.
template <bool N30>
__device__ __forceinline__ uint32_t reduce_acc(uint64_t x, const ModGroup& mg, int r) {
  return reduce64<N30>(x, mg, r);
}
template <bool N30>
__device__ __forceinline__ uint32_t reduce_acc(uint32_t x, const ModGroup& mg, int r) {
  return mod_reduce32(x, mg.p[r], (uint32_t)(mg.mu[r] >> 32));
}

// One output entry of a pairwise step (Sec. 2.1: the permuted operands
// multiplied as matrices): entry o of C from the operand entries ia, ib.
template <int RG, typename W = uint32_t, bool N30 = false>
__device__ __forceinline__ void step_entry_at(uint32_t k, uint32_t ka, uint32_t kb, uint64_t o, uint64_t ia,
                                              uint64_t ib, const W* A0, const W* B0, W* C0, const ModGroup& mg) {
  uint32_t out[RG];
  step_sum<RG, W, N30>(k, ka, kb, A0 + ia * RG, B0 + ib * RG, mg, out);
  store_entry<RG, W>(C0 + o * RG, out);
}

template <int RG, typename W = uint32_t, bool N30 = false>
__device__ __forceinline__ void step_entry(const StepDesc& d, uint64_t o, const W* A0, const W* B0, W* C0,
                                           const ModGroup& mg) {
  uint64_t ia, ib;
  map_addr(d, o, ia, ib);
  step_entry_at<RG, W, N30>(d.k, d.ka, d.kb, o, ia, ib, A0, B0, C0, mg);
}

// ------------------------------------------------------------------ kernels

template <int RG, typename W = uint32_t>
__global__ void __launch_bounds__(256) leaf_fill_kernel(const LeafDesc* __restrict__ leaves, int n_leaves,
                                                        const uint32_t* __restrict__ tables,
                                                        W* __restrict__ arena, ModGroup mg) {
  for (int l = blockIdx.x; l < n_leaves; l += gridDim.x) {
    const LeafDesc ld = leaves[l];
    const uint64_t n = 1ull << ld.rank;
    W* dst = arena + ld.off * RG;
    for (uint64_t idx = threadIdx.x; idx < n; idx += blockDim.x) {
      uint32_t v[RG];
#pragma unroll
      for (int r = 0; r < RG; r++) v[r] = leaf_value(ld.kind, ld.rank, (uint32_t)idx, tables, ld.table_off, mg.p[r]);
      store_entry<RG, W>(dst + idx * RG, v);
    }
  }
}

// A step launched over the whole GPU.  With S = 2^s threads in the grid, a
// thread visits o, o + S, o + 2S, ...: from one to the next the counter o >> s
// gains one, which clears its trailing ones and sets bit t, so each operand
// address changes by the precomputed delta[t] = w[t] - sum_{s <= j < t} w[j]
// (w[j] = operand weight of output bit j).  Any bit permutation costs the
// same two adds per entry.
struct GridStep {
  StepDesc d;
  uint64_t wA[32], wB[32];  // operand address weight of output bit j
  uint64_t dA[32], dB[32];  // address delta when the counter sets bit t
  uint32_t s;               // log2(total threads)
  uint32_t pad[3];
};

template <int RG, typename W = uint32_t, bool N30 = false>
__global__ void __launch_bounds__(256) step_kernel(const GridStep* __restrict__ g, W* __restrict__ arena,
                                                   ModGroup mg) {
  const uint32_t c = g->d.c, k = g->d.k, ka = g->d.ka, kb = g->d.kb, s = g->s;
  const uint64_t n = 1ull << c;
  const W* A0 = arena + g->d.a_off * RG;
  const W* B0 = arena + g->d.b_off * RG;
  W* C0 = arena + g->d.c_off * RG;
  uint64_t o = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (o >= n) return;
  uint64_t ia = 0, ib = 0;
  for (uint32_t j = 0; j < c; j++)
    if ((o >> j) & 1ull) {
      ia += g->wA[j];
      ib += g->wB[j];
    }
  for (;;) {
    step_entry_at<RG, W, N30>(k, ka, kb, o, ia, ib, A0, B0, C0, mg);
    const uint64_t u = o >> s;
    o += 1ull << s;
    if (o >= n) break;
    const uint32_t t = s + (uint32_t)(__ffsll((long long)~u) - 1);
    ia += g->dA[t];
    ib += g->dB[t];
  }
}

// A big step with one small operand (Sec. 2.1 with a skinny matrix): S has
// 2^fs <= 16 rows, the shared dimension 2^k <= 8, the large operand L 2^fl
// rows.  S's 2^(fs+k) entries are staged in shared memory; a thread takes a
// row l of L, loads its 2^k entries once (consecutive threads, consecutive
// rows: coalesced) and writes the 2^fs outputs C[oS(s) + oL(l)].  When S's
// free bits are C's lowest bits (contig) those outputs are contiguous and a
// thread writes them with vector stores (byte residues, 4 per entry).
struct OuterStep {
  uint64_t s_off, l_off, c_off;  // entry offsets of S, L, C in the arena
  uint64_t oS[16];               // output offset of S's row s
  uint64_t oL[32];               // output weight of L's free bit i
  uint32_t fs, fl, k, contig;
};

template <int RG, typename W = uint32_t, bool N30 = false>
__global__ void __launch_bounds__(256) outer_kernel(const __grid_constant__ OuterStep os, W* __restrict__ arena,
                                                    ModGroup mg) {
  __shared__ uint32_t sm[256 * RG];  // S entry (s, q) at (s + (q << fs)) * RG + r
  const uint32_t fs = os.fs, fl = os.fl, K = 1u << os.k, NS = 1u << fs;
  for (uint32_t i = threadIdx.x; i < (NS << os.k); i += blockDim.x) {
    uint32_t v[RG];
    load_entry<RG, W>(arena + (os.s_off + i) * RG, v);
#pragma unroll
    for (int r = 0; r < RG; r++) sm[i * RG + r] = v[r];
  }
  __syncthreads();
  using Acc = std::conditional_t<sizeof(W) == 1, uint32_t, uint64_t>;
  const W* L0 = arena + os.l_off * RG;
  W* C0 = arena + os.c_off * RG;
  const uint64_t nl = 1ull << fl;
  for (uint64_t l = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; l < nl; l += (uint64_t)gridDim.x * blockDim.x) {
    uint32_t lv[8][RG];
#pragma unroll
    for (uint32_t q = 0; q < 8; q++)
      if (q < K) load_entry<RG, W>(L0 + (l + ((uint64_t)q << fl)) * RG, lv[q]);
    uint64_t ol = 0;
    for (uint32_t i = 0; i < fl; i++)
      if ((l >> i) & 1ull) ol += os.oL[i];
    // output s of this row: sum over q of S(s, q) L(l, q), reduced
    auto entry = [&](uint32_t s, uint32_t (&out)[RG]) {
      Acc acc[RG];
#pragma unroll
      for (int r = 0; r < RG; r++) acc[r] = 0;
#pragma unroll
      for (uint32_t q = 0; q < 8; q++) {
        if (q < K) {
          const uint32_t* sv = sm + (s + (q << fs)) * RG;
#pragma unroll
          for (int r = 0; r < RG; r++) acc[r] += (Acc)sv[r] * lv[q][r];
          if (((q + 1) & mg.red_mask) == 0 && q + 1 < K) {
#pragma unroll
            for (int r = 0; r < RG; r++) acc[r] = reduce_acc<N30>(acc[r], mg, r);
          }
        }
      }
#pragma unroll
      for (int r = 0; r < RG; r++) out[r] = reduce_acc<N30>(acc[r], mg, r);
    };
    bool done = false;
    if constexpr (sizeof(W) == 1 && RG == 4) {
      if (os.contig) {  // C entries ol .. ol + NS - 1, 4 bytes each; ol is a multiple of NS
        uint32_t* dst = reinterpret_cast<uint32_t*>(C0 + ol * RG);
        for (uint32_t s0 = 0; s0 < NS; s0 += 4) {
          uint32_t w[4] = {0, 0, 0, 0};
#pragma unroll
          for (uint32_t j = 0; j < 4; j++)
            if (s0 + j < NS) {
              uint32_t out[RG];
              entry(s0 + j, out);
              w[j] = out[0] | (out[1] << 8) | (out[2] << 16) | (out[3] << 24);
            }
          if (NS >= 4) *reinterpret_cast<uint4*>(dst + s0) = make_uint4(w[0], w[1], w[2], w[3]);
          else if (NS == 2) *reinterpret_cast<uint2*>(dst) = make_uint2(w[0], w[1]);
          else dst[0] = w[0];
        }
        done = true;
      }
    }
    if (!done)
      for (uint32_t s = 0; s < NS; s++) {
        uint32_t out[RG];
        entry(s, out);
        store_entry<RG, W>(C0 + (os.oS[s] + ol) * RG, out);
      }
  }
}

// Split-K for steps with few output entries and a long shared dimension (a
// final dot product, a rank-19 tensor against a rank-19 tensor, ...): block
// (o, part) sums A*B over its slice of the 2^k shared values, the block's
// threads combine their residues with modular additions, and a second kernel
// adds the parts of each output.  part[o * n_split + j] holds RG residues.
template <int RG, typename W = uint32_t, bool N30 = false>
__global__ void __launch_bounds__(256) splitk_partial_kernel(const GridStep* __restrict__ g, const W* arena,
                                                             uint32_t* __restrict__ part, uint32_t log_split,
                                                             ModGroup mg) {
  __shared__ uint32_t red[256 * RG];
  const uint32_t n_split = 1u << log_split;
  const uint64_t o = blockIdx.x >> log_split;
  const uint32_t j = blockIdx.x & (n_split - 1);
  const uint32_t k = g->d.k, ka = g->d.ka, kb = g->d.kb, c = g->d.c;
  uint64_t ia = 0, ib = 0;
  for (uint32_t b = 0; b < c; b++)
    if ((o >> b) & 1ull) {
      ia += g->wA[b];
      ib += g->wB[b];
    }
  const W* A = arena + (g->d.a_off + ia) * RG;
  const W* B = arena + (g->d.b_off + ib) * RG;
  const uint64_t per = (1ull << k) >> log_split;
  // byte residues: products below 2^16, sums of 16 of them in 32 bits
  using Acc = std::conditional_t<sizeof(W) == 1, uint32_t, uint64_t>;
  Acc acc[RG];
#pragma unroll
  for (int r = 0; r < RG; r++) acc[r] = 0;
  uint32_t cnt = 0;
  bool dot = false;
  if constexpr (sizeof(W) == 1 && RG == 4) {
    // a dot product of contiguous byte-residue operands (no free bits): a
    // thread loads 4 entries of each operand (16 bytes), regroups the bytes
    // by residue (two rounds of byte permutes) and adds 4 products per
    // residue with one dp4a; 1024 products (below 2^26) between reductions
    if (ka == 0 && kb == 0 && (per & 1023u) == 0) {
      dot = true;
      for (uint64_t q = j * per + 4u * threadIdx.x; q < (j + 1) * per; q += 4u * blockDim.x) {
        const uint4 a4 = *reinterpret_cast<const uint4*>(A + q * 4);
        const uint4 b4 = *reinterpret_cast<const uint4*>(B + q * 4);
        const uint32_t ta0 = __byte_perm(a4.x, a4.y, 0x5140), ta1 = __byte_perm(a4.x, a4.y, 0x7362);
        const uint32_t ta2 = __byte_perm(a4.z, a4.w, 0x5140), ta3 = __byte_perm(a4.z, a4.w, 0x7362);
        const uint32_t tb0 = __byte_perm(b4.x, b4.y, 0x5140), tb1 = __byte_perm(b4.x, b4.y, 0x7362);
        const uint32_t tb2 = __byte_perm(b4.z, b4.w, 0x5140), tb3 = __byte_perm(b4.z, b4.w, 0x7362);
        acc[0] = __dp4a(__byte_perm(ta0, ta2, 0x5410), __byte_perm(tb0, tb2, 0x5410), acc[0]);
        acc[1] = __dp4a(__byte_perm(ta0, ta2, 0x7632), __byte_perm(tb0, tb2, 0x7632), acc[1]);
        acc[2] = __dp4a(__byte_perm(ta1, ta3, 0x5410), __byte_perm(tb1, tb3, 0x5410), acc[2]);
        acc[3] = __dp4a(__byte_perm(ta1, ta3, 0x7632), __byte_perm(tb1, tb3, 0x7632), acc[3]);
        if ((++cnt & 255u) == 0) {
#pragma unroll
          for (int r = 0; r < RG; r++) acc[r] = reduce_acc<N30>(acc[r], mg, r);
        }
      }
    }
  }
  if (!dot)
  for (uint64_t q = j * per + threadIdx.x; q < (j + 1) * per; q += blockDim.x) {
    uint32_t va[RG], vb[RG];
    load_entry<RG, W>(A + (q << ka) * RG, va);
    load_entry<RG, W>(B + (q << kb) * RG, vb);
#pragma unroll
    for (int r = 0; r < RG; r++) acc[r] += (Acc)va[r] * vb[r];
    if ((++cnt & mg.red_mask) == 0) {
#pragma unroll
      for (int r = 0; r < RG; r++) acc[r] = reduce_acc<N30>(acc[r], mg, r);
    }
  }
#pragma unroll
  for (int r = 0; r < RG; r++) red[threadIdx.x * RG + r] = reduce_acc<N30>(acc[r], mg, r);
  __syncthreads();
  for (uint32_t h = blockDim.x >> 1; h > 0; h >>= 1) {
    if (threadIdx.x < h) {
#pragma unroll
      for (int r = 0; r < RG; r++) {
        uint32_t x = red[threadIdx.x * RG + r] + red[(threadIdx.x + h) * RG + r];
        if (x >= mg.p[r]) x -= mg.p[r];
        red[threadIdx.x * RG + r] = x;
      }
    }
    __syncthreads();
  }
  if (threadIdx.x < RG) part[(uint64_t)blockIdx.x * RG + threadIdx.x] = red[threadIdx.x];
}

// One block per output entry: its threads add the parts, then combine.
template <int RG, typename W = uint32_t, bool N30 = false>
__global__ void __launch_bounds__(256) splitk_final_kernel(const GridStep* __restrict__ g, W* arena,
                                                           const uint32_t* __restrict__ part, uint32_t log_split,
                                                           ModGroup mg) {
  __shared__ uint32_t red[256 * RG];
  const uint64_t o = blockIdx.x;
  uint64_t s[RG];
#pragma unroll
  for (int r = 0; r < RG; r++) s[r] = 0;
  for (uint32_t j = threadIdx.x; j < (1u << log_split); j += blockDim.x) {
#pragma unroll
    for (int r = 0; r < RG; r++) s[r] += part[((o << log_split) + j) * RG + r];  // < 2^31 each, < 2^20 of them
  }
#pragma unroll
  for (int r = 0; r < RG; r++) red[threadIdx.x * RG + r] = reduce64<N30>(s[r], mg, r);
  __syncthreads();
  for (uint32_t h = blockDim.x >> 1; h > 0; h >>= 1) {
    if (threadIdx.x < h) {
#pragma unroll
      for (int r = 0; r < RG; r++) {
        uint32_t x = red[threadIdx.x * RG + r] + red[(threadIdx.x + h) * RG + r];
        if (x >= mg.p[r]) x -= mg.p[r];
        red[threadIdx.x * RG + r] = x;
      }
    }
    __syncthreads();
  }
  if (threadIdx.x < RG) arena[(g->d.c_off + o) * RG + threadIdx.x] = (W)red[threadIdx.x];
}

// All the small steps of one tree level in one launch: they are independent,
// so their output entries form one index space (step i owns [work_lo,
// work_lo + 2^c)); each thread finds its step by binary search.
template <int RG, typename W = uint32_t, bool N30 = false>
__global__ void __launch_bounds__(256) level_kernel(const StepDesc* __restrict__ steps, uint32_t n_steps,
                                                    uint32_t total, W* arena, ModGroup mg) {
  for (uint32_t w = blockIdx.x * blockDim.x + threadIdx.x; w < total; w += gridDim.x * blockDim.x) {
    uint32_t lo = 0, hi = n_steps - 1;
    while (lo < hi) {
      const uint32_t mid = (lo + hi + 1) >> 1;
      if (steps[mid].work_lo <= w) lo = mid;
      else hi = mid - 1;
    }
    const StepDesc& d = steps[lo];
    step_entry<RG, W, N30>(d, w - d.work_lo, arena + d.a_off * RG, arena + d.b_off * RG, arena + d.c_off * RG, mg);
  }
}

struct RootMap {
  uint8_t perm[24];  // root bit j -> open variable index
  int n_open;
};

// Root tensor -> result residues [entry][R], entry index bit i = open var i.
template <int RG, typename W = uint32_t>
__global__ void extract_kernel(const W* __restrict__ arena, uint64_t root_off, RootMap rm,
                               uint32_t* __restrict__ results, int R, int col) {
  const uint32_t n_out = 1u << rm.n_open;
  for (uint32_t J = blockIdx.x * blockDim.x + threadIdx.x; J < n_out; J += gridDim.x * blockDim.x) {
    uint64_t a = 0;
#pragma unroll
    for (int j = 0; j < 24; j++)
      if (j < rm.n_open) a |= (uint64_t)((J >> rm.perm[j]) & 1u) << j;
#pragma unroll
    for (int r = 0; r < RG; r++) results[(uint64_t)J * R + col + r] = arena[(root_off + a) * RG + r];
  }
}

// Chinese remaindering by Garner's mixed radix:
//   v0 = r0,  v_i = (r_i - (v0 + v1 p0 + ... + v_{i-1} p0..p_{i-2})) * inv_i  mod p_i,
//   X = v0 + p0 (v1 + p1 (v2 + ...)),  0 <= X < p0 p1 ... p_{R-1}.
constexpr int kCrtMaxResidues = 64;
constexpr int kCrtMaxLimbs = 17;
struct CrtConsts {
  uint32_t p[kCrtMaxResidues];
  uint64_t mu[kCrtMaxResidues];
  uint32_t inv[kCrtMaxResidues];  // (p0 ... p_{i-1})^{-1} mod p_i
  int R;
  int n_limbs;                    // <= kCrtMaxLimbs
};

__global__ void crt_kernel(const uint32_t* __restrict__ residues, uint64_t n_entries, CrtConsts cc,
                           uint32_t* __restrict__ limbs) {
  for (uint64_t e = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n_entries;
       e += (uint64_t)gridDim.x * blockDim.x) {
    uint32_t v[kCrtMaxResidues];
    const uint32_t* r = residues + e * cc.R;
    for (int i = 0; i < cc.R; i++) {
      const uint32_t p = cc.p[i];
      const uint64_t mu = cc.mu[i];
      uint32_t ri = r[i] % p;
      if (i == 0) {
        v[0] = ri;
        continue;
      }
      uint32_t t = mod_reduce(v[i - 1], p, mu);
      for (int j = i - 2; j >= 0; j--) t = mod_reduce((uint64_t)t * cc.p[j] + v[j], p, mu);
      const uint32_t diff = ri >= t ? ri - t : ri + (p - t);
      v[i] = mod_reduce((uint64_t)diff * cc.inv[i], p, mu);
    }
    uint32_t x[kCrtMaxLimbs];
    for (int l = 0; l < kCrtMaxLimbs; l++) x[l] = 0;
    x[0] = v[cc.R - 1];
    for (int i = cc.R - 2; i >= 0; i--) {
      uint64_t carry = v[i];
      for (int l = 0; l < cc.n_limbs; l++) {
        const uint64_t t = (uint64_t)x[l] * cc.p[i] + carry;
        x[l] = (uint32_t)t;
        carry = t >> 32;
      }
    }
    for (int l = 0; l < cc.n_limbs; l++) limbs[e * cc.n_limbs + l] = x[l];
  }
}

// ------------------------------------------------------- persistent batch

// Packed batch descriptors.  Everything one formula's contraction looks up is
// one contiguous, 16-byte aligned blob (steps, segments, packed items, bit-map
// runs, address deltas, level table), copied to shared memory in one coalesced
// pass when a CTA starts the formula.  Offsets are relative to the formula's
// own arena; a run is a u16: src | dst << 5 | len << 10.
struct BStep {
  uint32_t a_off, b_off, c_off;
  uint16_t run0;  // first run of A's map (blob-relative); B's map follows
  uint16_t dl0;   // first address delta (blob-relative, int2 units)
  uint8_t c, k, ka, kb;
  uint8_t nra, nrb, g, pad;  // g: log2 of the entry stride of a lane group (5 - sh)
};

// The unit of work of one warp.  An output entry whose sum runs over 2^k
// shared values may be split over 2^sh lanes (sh <= min(k, 5)): lane slice j
// sums the shared values j, j + 2^sh, ..., and the lanes of the entry add
// their residues with butterfly shuffles.  A segment is either a block of one
// step: step = step index, o0 = first entry, n = V entries per lane group: the
// 2^(5 - sh) lane groups take entries o0 + group + i 2^(5 - sh), i < V, the
// operand addresses advancing from one to the next by the step's precomputed
// deltas (the output counter o >> g gains one, clearing its trailing ones and
// setting bit t: each address changes by delta[t - g]); or, for steps whose
// entries need fewer than 32 lanes, the lanes of several such entries packed
// side by side: step = kPacked, o0 = first of n lane items, each item =
// step | entry << 16 | slice << 21 | sh << 26, the entries' lane groups
// aligned to their size; sh is then the largest split in the segment.
constexpr uint16_t kPacked = 0xFFFF;
struct Seg {
  uint32_t o0;
  uint16_t step;
  uint8_t n;   // whole-warp block: entries per lane group V; packed: active lanes
  uint8_t sh;  // log2 lanes per entry (packed: the largest)
};

// Sum of A*B over 2^KK shared values (KK <= 4) for residues whose products
// fit 16 to a 64-bit accumulator (the default primes below 2^30): fully
// unrolled, one reduction per residue at the end.  Operand entries of the
// batch arena are addressed by 32-bit entry indices.
template <int RG, bool N30, int KK>
__device__ __forceinline__ void step_sum_fixed(uint32_t ka, uint32_t kb, const uint32_t* A, const uint32_t* B,
                                               const ModGroup& mg, uint32_t (&out)[RG]) {
  uint64_t acc[RG];
#pragma unroll
  for (int r = 0; r < RG; r++) acc[r] = 0;
  const size_t sa = (size_t)RG << ka, sb = (size_t)RG << kb;
#pragma unroll
  for (uint32_t q = 0; q < (1u << KK); q++) {
    uint32_t va[RG], vb[RG];
    load_entry<RG>(A, va);
    load_entry<RG>(B, vb);
    A += sa;
    B += sb;
#pragma unroll
    for (int r = 0; r < RG; r++) acc[r] += (uint64_t)va[r] * vb[r];
  }
#pragma unroll
  for (int r = 0; r < RG; r++) out[r] = reduce64<N30>(acc[r], mg, r);
}

// step_sum for the batch kernel.  For the default primes (16 products fit a
// 64-bit accumulator between reductions): up to 4 products fully unrolled;
// longer sums in unrolled groups of 4 (one group's loads in flight at a
// time, which bounds the registers), reduced after every 16th product.
// Other primes: the general loop.
template <int RG, bool N30>
__device__ __forceinline__ void batch_sum(uint32_t k, uint32_t ka, uint32_t kb, const uint32_t* A, const uint32_t* B,
                                          const ModGroup& mg, uint32_t (&out)[RG]) {
  if (N30) {
    switch (k) {
      case 0: step_sum_fixed<RG, N30, 0>(ka, kb, A, B, mg, out); return;
      case 1: step_sum_fixed<RG, N30, 1>(ka, kb, A, B, mg, out); return;
      case 2: step_sum_fixed<RG, N30, 2>(ka, kb, A, B, mg, out); return;
      default: {
        uint64_t acc[RG];
#pragma unroll
        for (int r = 0; r < RG; r++) acc[r] = 0;
        const uint32_t K = 1u << k;
        const size_t sa = (size_t)RG << ka, sb = (size_t)RG << kb;
#pragma unroll 1
        for (uint32_t q = 0; q < K; q += 4) {
#pragma unroll
          for (uint32_t u = 0; u < 4; u++) {
            uint32_t va[RG], vb[RG];
            load_entry<RG>(A, va);
            load_entry<RG>(B, vb);
            A += sa;
            B += sb;
#pragma unroll
            for (int r = 0; r < RG; r++) acc[r] += (uint64_t)va[r] * vb[r];
          }
          if (((q + 4) & 15u) == 0 && q + 4 < K) {
#pragma unroll
            for (int r = 0; r < RG; r++) acc[r] = reduce64<N30>(acc[r], mg, r);
          }
        }
#pragma unroll
        for (int r = 0; r < RG; r++) out[r] = reduce64<N30>(acc[r], mg, r);
        return;
      }
    }
  }
  step_sum<RG, uint32_t, N30>(k, ka, kb, A, B, mg, out);
}

struct BLeaf {
  uint32_t off;
  uint32_t table_off;
  uint8_t kind, rank, pad0, pad1;
};

struct BForm {
  uint32_t blob;                     // first uint4 of the formula's blob
  uint32_t blob_n;                   // uint4 count
  uint32_t segs_at, items_at, runs_at, lvl_at;  // byte offsets of the blob sections (steps at 0)
  uint32_t nlev, leaf0, nleaf, res_off, n_out, perm_off;
  uint32_t n_open, root_off, arena, dl_at;  // arena: entries this formula needs; dl_at: deltas
};

struct BatchArgs {
  const BForm* forms;
  const uint4* blobs;
  const BLeaf* leaves;
  const uint32_t* tables;
  const uint8_t* perms;
  const uint32_t* order;  // queue slot -> formula (largest first)
  uint32_t n_forms;
  uint32_t* queue;        // work counter, zeroed before the launch
  uint32_t* results;      // [entry][R]
  uint32_t* garena;       // global arenas, one slot per CTA, reused by every formula the CTA takes
  uint64_t slot_entries;  // entries of a slot (the largest formula's arena)
  uint32_t blob_cap;      // bytes of dynamic shared memory reserved for a blob
  uint32_t smem_cap;      // entries of dynamic shared memory available for an arena
  int R;
  int col;                // first residue column of this group
};

__device__ __forceinline__ uint32_t map_runs(uint32_t o, const uint16_t* runs, int n) {
  uint32_t a = 0;
  for (int i = 0; i < n; i++) {
    const uint32_t r = runs[i];
    const uint32_t src = r & 31u, dst = (r >> 5) & 31u, len = r >> 10;
    a |= ((o >> src) & ((1u << len) - 1u)) << dst;
  }
  return a;
}

// Each CTA repeatedly takes the next formula from the queue and contracts it
// alone, tree level by tree level: all steps of a level are independent, so
// the level is a list of segments shared out over the CTA's warps, with one
// barrier per level.  Descriptors are read from shared memory; the tensors
// live in shared memory when the formula's arena fits, else in the CTA's own
// slot of global memory, reused by each formula the CTA takes, so that the
// live arenas (CTAs x slot) stay in L2 instead of every formula's arena being
// written back to DRAM.
template <int RG, bool N30 = false>
__global__ void __launch_bounds__(256) batch_kernel(BatchArgs a, ModGroup mg) {
  extern __shared__ uint4 smem_raw[];
  __shared__ uint32_t task;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  uint4* blob = smem_raw;
  uint32_t* sarena = reinterpret_cast<uint32_t*>(smem_raw + (a.blob_cap >> 4));
  for (;;) {
    if (threadIdx.x == 0) task = atomicAdd(a.queue, 1u);
    __syncthreads();
    const uint32_t t = task;
    if (t >= a.n_forms) break;
    const BForm f = a.forms[a.order[t]];
    for (uint32_t i = threadIdx.x; i < f.blob_n; i += blockDim.x) blob[i] = a.blobs[f.blob + i];
    uint32_t* arena = f.arena <= a.smem_cap ? sarena : a.garena + (uint64_t)blockIdx.x * a.slot_entries * RG;
    for (uint32_t l = threadIdx.x; l < f.nleaf; l += blockDim.x) {
      const BLeaf ld = a.leaves[f.leaf0 + l];
      uint32_t* dst = arena + (uint64_t)ld.off * RG;
      const uint32_t n = 1u << ld.rank;
      for (uint32_t idx = 0; idx < n; idx++) {
        uint32_t v[RG];
#pragma unroll
        for (int r = 0; r < RG; r++) v[r] = leaf_value(ld.kind, ld.rank, idx, a.tables, ld.table_off, mg.p[r]);
        store_entry<RG>(dst + (uint64_t)idx * RG, v);
      }
    }
    __syncthreads();
    const char* bb = reinterpret_cast<const char*>(blob);
    const BStep* steps = reinterpret_cast<const BStep*>(bb);
    const Seg* segs = reinterpret_cast<const Seg*>(bb + f.segs_at);
    const uint32_t* items = reinterpret_cast<const uint32_t*>(bb + f.items_at);
    const uint16_t* runs_all = reinterpret_cast<const uint16_t*>(bb + f.runs_at);
    const uint32_t* lvl = reinterpret_cast<const uint32_t*>(bb + f.lvl_at);
    const int2* deltas = reinterpret_cast<const int2*>(bb + f.dl_at);
    for (uint32_t l = 0; l < f.nlev; l++) {
      const uint32_t s1 = lvl[l + 1];
      for (uint32_t sg = lvl[l] + warp; sg < s1; sg += nwarps) {
        const Seg seg = segs[sg];
        if (seg.step != kPacked) {
          // a block of V entries per lane group of one step
          const BStep d = steps[seg.step];
          const uint32_t sh = seg.sh, g = d.g;
          uint32_t o = seg.o0 + (lane >> sh);
          const uint32_t slice = lane & ((1u << sh) - 1u);
          const uint16_t* runs = runs_all + d.run0;
          uint32_t ia = map_runs(o, runs, d.nra) + (slice << d.ka);
          uint32_t ib = map_runs(o, runs + d.nra, d.nrb) + (slice << d.kb);
          const uint32_t* A0 = arena + (uint64_t)d.a_off * RG;
          const uint32_t* B0 = arena + (uint64_t)d.b_off * RG;
          uint32_t* C0 = arena + (uint64_t)d.c_off * RG;
          const int2* dl = deltas + d.dl0;
          for (uint32_t v = 0; v < seg.n; v++) {
            uint32_t out[RG];
            batch_sum<RG, N30>(d.k - sh, d.ka + sh, d.kb + sh, A0 + ia * RG, B0 + ib * RG, mg, out);
            for (uint32_t m = 1; m < (1u << sh); m <<= 1) {
#pragma unroll
              for (int r = 0; r < RG; r++) {
                const uint32_t t = out[r] + __shfl_xor_sync(0xFFFFFFFFu, out[r], m);
                out[r] = t >= mg.p[r] ? t - mg.p[r] : t;
              }
            }
            if (slice == 0) store_entry<RG>(C0 + o * RG, out);
            if (v + 1 < seg.n) {
              const int2 dd = dl[__ffs(~(o >> g)) - 1];
              o += 1u << g;
              ia += (uint32_t)dd.x;
              ib += (uint32_t)dd.y;
            }
          }
          continue;
        }
        // packed lanes of small steps, one entry per lane
        const bool active = lane < seg.n;
        const uint32_t it = items[seg.o0 + (active ? lane : 0)];
        const uint32_t st = it & 0xFFFFu, o = (it >> 16) & 31u, slice = (it >> 21) & 31u, sh = it >> 26;
        const BStep d = steps[st];
        uint32_t out[RG];
        if (active) {
          const uint16_t* runs = runs_all + d.run0;
          const uint32_t ia = map_runs(o, runs, d.nra) + (slice << d.ka);
          const uint32_t ib = map_runs(o, runs + d.nra, d.nrb) + (slice << d.kb);
          batch_sum<RG, N30>(d.k - sh, d.ka + sh, d.kb + sh, arena + ((uint64_t)d.a_off + ia) * RG,
                             arena + ((uint64_t)d.b_off + ib) * RG, mg, out);
        } else {
#pragma unroll
          for (int r = 0; r < RG; r++) out[r] = 0;
        }
        // lanes of one entry add their partial sums (all lanes take part in
        // every shuffle; a lane keeps only its own group's partners)
        for (uint32_t m = 1; m < (1u << seg.sh); m <<= 1) {
#pragma unroll
          for (int r = 0; r < RG; r++) {
            const uint32_t v = __shfl_xor_sync(0xFFFFFFFFu, out[r], m);
            if (m < (1u << sh)) {
              const uint32_t t = out[r] + v;
              out[r] = t >= mg.p[r] ? t - mg.p[r] : t;
            }
          }
        }
        if (active && slice == 0) store_entry<RG>(arena + ((uint64_t)d.c_off + o) * RG, out);
      }
      __syncthreads();
    }
    for (uint32_t J = threadIdx.x; J < f.n_out; J += blockDim.x) {
      uint32_t ad = 0;
      for (uint32_t j = 0; j < f.n_open; j++) ad |= ((J >> a.perms[f.perm_off + j]) & 1u) << j;
#pragma unroll
      for (int r = 0; r < RG; r++)
        a.results[((uint64_t)f.res_off + J) * a.R + a.col + r] = arena[((uint64_t)f.root_off + ad) * RG + r];
    }
    __syncthreads();
  }
}

}  // namespace tnc_dev
