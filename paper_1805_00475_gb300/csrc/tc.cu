// Dense pairwise steps on the 5th-generation tensor cores (tcgen05), exact.
//
// A step C[m,n] = sum_q A[m,q] B[n,q] mod p (A: M x K, B: N x K, residues
// below 2^30; the bit maps of the lowering make both operands plain
// column-major matrices) is computed from 8-bit limbs:
//   a = sum_i a_i 256^i,  b = sum_j b_j 256^j,  0 <= a_i, b_j <= 255,
//   C = sum_s 256^s C_s mod p,  C_s = sum_{i+j=s} A_i B_j^T   (s = 0..6).
// Limb values are exact in bf16 and products below 2^16, so C_s accumulates
// exactly in the fp32 tensor-core accumulators as long as it stays below
// 2^24: at most 4 limb pairs share an s, 4 * 255^2 * 64 < 2^24, so K is
// processed in chunks of 64 and every chunk's C_s is folded into 64-bit
// integer accumulators, C += sum_s 256^s C_s mod p.  No precision is lost.
// The tensor cores run kind::f16 with fp16 inputs and fp32 accumulation: the
// 8-bit integer form (kind::i8) does not exist for sm_103a, and fp16 carries
// 8-bit limbs exactly (a limb v becomes the half 1024 + v by
// bit operations, minus 1024 in one packed subtract).
//
// CTA tile: 128 rows of C (TMEM lanes) x 32 columns, 256 threads (8 warps);
// warp w reads TMEM lane quarter w%4 and columns 16*(w/4) .. +16.  Pipeline:
// two shared-memory stages of limbs (canonical K-major, no-swizzle layout: 8 x
// 16-byte core matrices) and two sets of 7 TMEM accumulators (7 x 32 columns
// each); while the MMAs of chunk c run, the threads stage chunk c+1 and fold
// the accumulators of chunk c-1.  One thread issues the 16 limb pairs x 4 MMAs
// of 128 x 32 x 16 per chunk and commits them to that stage's mbarrier.
// Every wait is bounded: on timeout the kernel records an error word, frees
// its TMEM and returns.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstring>
#include <string>
#include <vector>

#include "modarith.cuh"
#include "tnc_internal.h"

namespace tnc_tc {

constexpr int kTileM = 128;
constexpr int kTileN = 32;
constexpr int kChunkK = 64;
constexpr int kThreads = 256;
constexpr uint32_t kTmemCols = 512;  // 2 buffers x 7 accumulators x 32 columns = 448
constexpr uint32_t kAccStride = 256; // columns between the two accumulator buffers
constexpr uint32_t kSpinLimit = 1u << 22;

// Shared memory per stage: A limbs 4 x (128 x 64 bf16) + B limbs 4 x (32 x 64 bf16).
constexpr uint32_t kALimbBytes = kTileM * kChunkK * 2;  // 16 KiB
constexpr uint32_t kBLimbBytes = kTileN * kChunkK * 2;  // 4 KiB
constexpr uint32_t kStageBytes = 4 * kALimbBytes + 4 * kBLimbBytes;  // 80 KiB
constexpr uint32_t kSmemBytes = 2 * kStageBytes + 1024;

struct TcStep {
  uint64_t a_off, b_off, c_off;  // entries (one residue per entry)
  uint32_t fa, fb, k;            // M = 2^fa, N = 2^fb, K = 2^k
  uint32_t log_split;            // K split over 2^log_split CTAs per tile (partials summed after)
  uint64_t wm[32], wn[32];       // output address weight of row bit j / column bit j
  uint32_t p, red_pad;
  uint64_t mu;
  uint32_t w256[7];              // 256^s mod p (w256[5] = 2^40 mod p is used)
  uint32_t pad2;
};

// ---- PTX helpers -----------------------------------------------------------

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// Canonical K-major, no-swizzle shared-memory matrix descriptor: core matrices
// of 8 rows x 16 bytes, LBO = byte distance between core matrices adjacent in
// K, SBO = between core matrices adjacent in M/N; version 1; layout 0.
__device__ __forceinline__ uint64_t make_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// Instruction descriptor, kind::f16: D = F32 (bits 4-5 = 1), A = B = F16
// (bits 7-9, 10-12 = 0), both K-major, N >> 3 at bits 17-22, M >> 4 at 24-28.
__host__ __device__ constexpr uint32_t make_idesc(uint32_t M, uint32_t N) {
  return (1u << 4) | ((N >> 3) << 17) | ((M >> 4) << 24);
}

__device__ __forceinline__ void mma_f16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ void mma_commit(uint32_t mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
               : "memory");
}

__device__ __forceinline__ void mbar_init(uint32_t mbar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(mbar), "r"(count) : "memory");
}

// Bounded wait for phase `parity` of an mbarrier; false on timeout.
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity) {
  for (uint32_t i = 0; i < kSpinLimit; i++) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.b32 %0, 1, 0, p;\n\t}\n"
        : "=r"(done)
        : "r"(mbar), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

// Zero 16 TMEM columns of this warp's 32 lanes.
__device__ __forceinline__ void tmem_zero16(uint32_t taddr) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1};" ::"r"(taddr),
      "r"(0u)
      : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&v)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]), "=r"(v[8]),
        "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// Exact integer value of a float holding an integer below 2^23.
__device__ __forceinline__ uint32_t f2u_small(uint32_t fbits) {
  return __float_as_uint(__uint_as_float(fbits) + 8388608.0f) - 0x4B000000u;
}

// Limb li (bits 8li..8li+7) of x0 and of x1 as a packed pair of fp16 values
// (x0's in the low half): bytes placed at 0 and 2, exponent bits of 1024
// or-ed in (half 1024 + v, exact for v < 1024), then 1024 subtracted.
template <int li>
__device__ __forceinline__ uint32_t limb_pair_f16(uint32_t x0, uint32_t x1) {
  constexpr uint32_t sel = (uint32_t)li | ((uint32_t)(4 + li) << 8);
  const uint32_t t = (__byte_perm(x0, x1, sel) & 0x00FF00FFu) | 0x64006400u;
  uint32_t r;
  asm("sub.rn.f16x2 %0, %1, %2;" : "=r"(r) : "r"(t), "r"(0x64006400u));
  return r;
}

// ---- the kernel ------------------------------------------------------------

// Byte offset of element (row r, k-index q) of a K-major limb tile whose core
// matrices are 8 rows x 8 elements: core (r/8, q/8) at (r/8)*SBO + (q/8)*128,
// element at (r%8)*16 + (q%8)*2; SBO = (kChunkK/8)*128 = 1024.
__device__ __forceinline__ uint32_t kmajor_off(uint32_t r, uint32_t q) {
  return (r >> 3) * 1024u + (q >> 3) * 128u + (r & 7u) * 16u + (q & 7u) * 2u;
}

// Stage chunk k0 of A's 128 rows and B's 32 rows as 8-bit limbs (bf16).
// 1024 (row, 8-q group) pairs of A and 256 of B are shared by the 256 threads:
// every thread first issues all 40 of its loads, then converts and stores.
__device__ __forceinline__ void stage_chunk(uint8_t* sA, uint8_t* sB, const uint32_t* A, const uint32_t* B, uint32_t M,
                                            uint32_t N, uint32_t m0, uint32_t n0, uint32_t k0, uint32_t tid) {
  uint32_t x[5][8];
#pragma unroll
  for (int it = 0; it < 5; it++) {
    const uint32_t job = tid + it * kThreads;  // 0..1023: A, 1024..1279: B (warp-uniform per it)
    const bool isA = it < 4;
    const uint32_t jj = isA ? job : job - 1024;
    const uint32_t r = isA ? (jj & 127u) : (jj & 31u);
    const uint32_t q8 = isA ? (jj >> 7) * 8u : (jj >> 5) * 8u;
    const uint32_t* src = isA ? A + m0 + r : B + n0 + r;
    const uint32_t ld = isA ? M : N;
#pragma unroll
    for (int e = 0; e < 8; e++) x[it][e] = src[(uint64_t)(k0 + q8 + e) * ld];
  }
#pragma unroll
  for (int it = 0; it < 5; it++) {
    const uint32_t job = tid + it * kThreads;
    const bool isA = it < 4;
    const uint32_t jj = isA ? job : job - 1024;
    const uint32_t r = isA ? (jj & 127u) : (jj & 31u);
    const uint32_t q8 = isA ? (jj >> 7) * 8u : (jj >> 5) * 8u;
    uint8_t* base = isA ? sA : sB;
    const uint32_t lbytes = isA ? kALimbBytes : kBLimbBytes;
    const uint32_t off = kmajor_off(r, q8);
    const uint32_t* v = x[it];
    *reinterpret_cast<uint4*>(base + 0 * lbytes + off) =
        make_uint4(limb_pair_f16<0>(v[0], v[1]), limb_pair_f16<0>(v[2], v[3]), limb_pair_f16<0>(v[4], v[5]),
                   limb_pair_f16<0>(v[6], v[7]));
    *reinterpret_cast<uint4*>(base + 1 * lbytes + off) =
        make_uint4(limb_pair_f16<1>(v[0], v[1]), limb_pair_f16<1>(v[2], v[3]), limb_pair_f16<1>(v[4], v[5]),
                   limb_pair_f16<1>(v[6], v[7]));
    *reinterpret_cast<uint4*>(base + 2 * lbytes + off) =
        make_uint4(limb_pair_f16<2>(v[0], v[1]), limb_pair_f16<2>(v[2], v[3]), limb_pair_f16<2>(v[4], v[5]),
                   limb_pair_f16<2>(v[6], v[7]));
    *reinterpret_cast<uint4*>(base + 3 * lbytes + off) =
        make_uint4(limb_pair_f16<3>(v[0], v[1]), limb_pair_f16<3>(v[2], v[3]), limb_pair_f16<3>(v[4], v[5]),
                   limb_pair_f16<3>(v[6], v[7]));
  }
}

// B's four limb tiles are contiguous with the same core-matrix strides, so
// together they are one K-major operand of 4 x 32 = 128 rows (row = 32 lj + n).
// One MMA of 128 x 128 x 16 per A limb li then yields A_li B_lj for all lj;
// written at column offset 32 li, the product of limbs (li, lj) lands in the
// columns of accumulator s = li + lj.  Columns 0..127 are overwritten by the
// first MMA of the chunk; 128..223 are zeroed beforehand.
__device__ __forceinline__ void issue_chunk(uint32_t acc_col, uint32_t sA, uint32_t sB) {
  constexpr uint32_t idesc = make_idesc(kTileM, 4 * kTileN);
  const uint64_t a0 = make_desc(sA, 128u, 1024u), b0 = make_desc(sB, 128u, 1024u);
#pragma unroll
  for (int li = 0; li < 4; li++)
#pragma unroll
    for (int ks = 0; ks < kChunkK / 16; ks++) {
      // +16 bytes per unit of the descriptor's start-address field
      const uint64_t ad = a0 + (uint64_t)((li * kALimbBytes + ks * 256u) >> 4);
      const uint64_t bd = b0 + (uint64_t)((ks * 256u) >> 4);
      mma_f16(acc_col + (uint32_t)li * kTileN, ad, bd, idesc, (li | ks) ? 1u : 0u);
    }
}

__global__ void __launch_bounds__(kThreads, 1) tc_step_kernel(const TcStep* __restrict__ g, uint32_t* arena,
                                                             uint32_t* part, uint32_t* err) {
  extern __shared__ __align__(1024) uint8_t smem[];
  __shared__ uint64_t mbar_storage[2];
  __shared__ uint32_t tmem_base_s;
  const uint32_t tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const uint32_t quarter = warp & 3u, half = warp >> 2;
  const uint32_t M = 1u << g->fa, N = 1u << g->fb, K = 1u << g->k;
  const uint32_t tiles_m = M / kTileM;
  const uint32_t split = blockIdx.x & ((1u << g->log_split) - 1u), tile = blockIdx.x >> g->log_split;
  const uint32_t tm = tile % tiles_m, tn = tile / tiles_m;
  const uint32_t kbeg = split * (K >> g->log_split);
  const uint32_t n_chunks = (K >> g->log_split) / kChunkK;
  const uint32_t m0 = tm * kTileM, n0 = tn * kTileN;
  // stage b: A limbs at smem + b*kStageBytes, B limbs right after them
#define TC_SA(b) (smem + (b) * kStageBytes)
#define TC_SB(b) (smem + (b) * kStageBytes + 4 * kALimbBytes)
  const uint32_t mbar0 = smem_u32(&mbar_storage[0]), mbar1 = smem_u32(&mbar_storage[1]);

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base_s)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    mbar_init(mbar0, 1);
    mbar_init(mbar1, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  const uint32_t* A = arena + g->a_off;
  const uint32_t* B = arena + g->b_off;
  stage_chunk(TC_SA(0), TC_SB(0), A, B, M, N, m0, n0, kbeg, tid);
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_base_s;
  // zero accumulators s = 4..6 (columns 128..223) of both buffers; each warp
  // owns one lane quarter and one 16-column half of every accumulator
#pragma unroll
  for (uint32_t bb = 0; bb < 2; bb++)
#pragma unroll
    for (uint32_t ss = 4; ss < 7; ss++)
      tmem_zero16(tmem + ((quarter * 32u) << 16) + bb * kAccStride + ss * kTileN + half * 16u);
  asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (tid == 0) {
    issue_chunk(tmem, smem_u32(TC_SA(0)), smem_u32(TC_SB(0)));
    mma_commit(mbar0);
  }

  const uint32_t p = g->p;
  const uint64_t mu = g->mu;
  uint64_t lo[16], hi[16];
#pragma unroll
  for (int j = 0; j < 16; j++) lo[j] = hi[j] = 0;
  bool ok = true;
  for (uint32_t c = 0; c < n_chunks; c++) {
    const uint32_t b = c & 1u;
    if (c + 1 < n_chunks)  // the buffer of chunk c-1 is free: its MMAs completed in the previous iteration
      stage_chunk(TC_SA(b ^ 1u), TC_SB(b ^ 1u), A, B, M, N, m0, n0, kbeg + (c + 1) * kChunkK, tid);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    const int waited = mbar_wait(b ? mbar1 : mbar0, (c >> 1) & 1u) ? 1 : 0;
    ok = __syncthreads_and(waited) != 0;  // also: every thread has staged chunk c+1
    if (!ok) break;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (c + 1 < n_chunks && tid == 0) {
      issue_chunk(tmem + (b ^ 1u) * kAccStride, smem_u32(TC_SA(b ^ 1u)), smem_u32(TC_SB(b ^ 1u)));
      mma_commit(b ? mbar0 : mbar1);
    }
    // fold the 7 accumulators of chunk c (this thread: one row, 16 columns):
    // lo += C0 + C1 2^8 + ... + C4 2^32 (< 2^57 per chunk), hi += C5 + C6 2^8
    // (< 2^31 per chunk); count = lo + hi 2^40.  lo and hi are reduced mod p
    // every 64 chunks (64 * 2^57 = 2^63) and at the end.  Accumulators with
    // at most 2 limb pairs are below 2^23 and convert by a float add
    // (x + 2^23 has x in its low mantissa bits); the others by F2I.
    const uint32_t tl = tmem + ((quarter * 32u) << 16) + b * kAccStride + half * 16u;
    {
      uint32_t v0[16], v1[16];
      tmem_ld16(tl + 0 * kTileN, v0);
      tmem_ld16(tl + 1 * kTileN, v1);
#pragma unroll
      for (int j = 0; j < 16; j++)
        lo[j] += (uint64_t)(f2u_small(v0[j]) + (f2u_small(v1[j]) << 8));
    }
#pragma unroll
    for (int ss = 2; ss < 5; ss++) {
      uint32_t v[16];
      tmem_ld16(tl + (uint32_t)ss * kTileN, v);
#pragma unroll
      for (int j = 0; j < 16; j++) lo[j] += (uint64_t)__float2uint_rn(__uint_as_float(v[j])) << (8 * ss);
    }
    {
      uint32_t v5[16], v6[16];
      tmem_ld16(tl + 5 * kTileN, v5);
      tmem_ld16(tl + 6 * kTileN, v6);
#pragma unroll
      for (int j = 0; j < 16; j++) hi[j] += f2u_small(v5[j]) + (f2u_small(v6[j]) << 8);
    }
    if ((c & 63u) == 63u) {
#pragma unroll
      for (int j = 0; j < 16; j++) {
        lo[j] = tnc_dev::mod_reduce(lo[j], p, mu);
        hi[j] = tnc_dev::mod_reduce(hi[j], p, mu);
      }
    }
    // the columns this warp just read of accumulators 4..6 start the chunk
    // after next at zero
#pragma unroll
    for (uint32_t ss = 4; ss < 7; ss++) tmem_zero16(tl + ss * kTileN);
    asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  }
  if (!ok && tid == 0) atomicExch(err, 1u);

  uint32_t res[16];
  {
    const uint32_t w40 = g->w256[5];  // 2^40 mod p
#pragma unroll
    for (int j = 0; j < 16; j++)
      res[j] = tnc_dev::mod_reduce(tnc_dev::mod_reduce(lo[j], p, mu) +
                                       (uint64_t)tnc_dev::mod_reduce(hi[j], p, mu) * w40,
                                   p, mu);
  }
  if (ok) {
    // C[o(m, n)]: o = sum of the output weights of m's and n's bits
    const uint32_t m = m0 + quarter * 32u + lane;
    uint64_t om = 0;
    for (uint32_t j = 0; j < g->fa; j++)
      if ((m >> j) & 1u) om += g->wm[j];
    uint32_t* C = g->log_split ? part + ((uint64_t)split << (g->fa + g->fb)) : arena + g->c_off;
    const uint32_t nb = n0 + half * 16u;  // columns nb .. nb+15: bits 0..3 vary
    uint64_t on0 = 0;
    for (uint32_t j = 4; j < g->fb; j++)
      if ((nb >> j) & 1u) on0 += g->wn[j];
#pragma unroll
    for (int jn = 0; jn < 16; jn++) {
      uint64_t on = on0;
#pragma unroll
      for (int j = 0; j < 4; j++)
        if ((jn >> j) & 1) on += g->wn[j];
      C[om + on] = res[jn];
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
#undef TC_SA
#undef TC_SB
}

// Sum of the K-split partials of a dense step: C[o] = sum_j part[j][o] mod p.
__global__ void tc_split_final_kernel(const TcStep* __restrict__ g, uint32_t* arena, const uint32_t* __restrict__ part) {
  const uint64_t n = 1ull << (g->fa + g->fb);
  uint32_t* C = arena + g->c_off;
  for (uint64_t o = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; o < n; o += (uint64_t)gridDim.x * blockDim.x) {
    uint64_t s = 0;
    for (uint32_t j = 0; j < (1u << g->log_split); j++) s += part[((uint64_t)j << (g->fa + g->fb)) + o];
    C[o] = tnc_dev::mod_reduce(s, g->p, g->mu);
  }
}

}  // namespace tnc_tc

namespace tnc {

// Can this step run on the tensor cores (possibly with A and B exchanged)?
bool tc_eligible(const StepDesc& d) {
  const int fa = d.ka, fb = d.kb;
  return d.k >= 6 && ((fa >= 7 && fb >= 5) || (fb >= 7 && fa >= 5));
}

size_t tc_step_bytes() { return sizeof(tnc_tc::TcStep); }

// K split of a dense step: double it while the tiles x splits stay below two
// CTAs per SM of a 152-SM GPU, each split keeps >= 2 chunks of 64, and the
// partials (2^c entries per split) stay within tc_part_entries().
uint64_t tc_part_entries() { return 1ull << 24; }
uint32_t tc_split_log(const StepDesc& d) {
  const bool swap = !(d.ka >= 7 && d.kb >= 5);
  const uint32_t fa = swap ? d.kb : d.ka, fb = swap ? d.ka : d.kb;
  const uint64_t tiles = (1ull << (fa - 7)) << (fb - 5);
  uint32_t ls = 0;
  while ((tiles << ls) < 304 && d.k - ls > 7 && (1ull << (d.c + ls + 1)) <= tc_part_entries()) ls++;
  return ls;
}

// Host-side descriptor for one dense step and residue prime p.
void tc_make_step(const StepDesc& d, uint32_t p, void* out) {
  using tnc_tc::TcStep;
  TcStep t;
  std::memset(&t, 0, sizeof(t));
  int op[64] = {0}, dst[64] = {0};
  if (d.nra != TNC_BITMAP) {
    for (int i = 0; i < d.nra; i++)
      for (int q = 0; q < d.map.runs.ra[i].len; q++) {
        op[d.map.runs.ra[i].src + q] = 0;
        dst[d.map.runs.ra[i].src + q] = d.map.runs.ra[i].dst + q;
      }
    for (int i = 0; i < d.nrb; i++)
      for (int q = 0; q < d.map.runs.rb[i].len; q++) {
        op[d.map.runs.rb[i].src + q] = 1;
        dst[d.map.runs.rb[i].src + q] = d.map.runs.rb[i].dst + q;
      }
  } else {
    for (int j = 0; j < d.c; j++) {
      op[j] = d.map.bit[j] >> 7;
      dst[j] = d.map.bit[j] & 63;
    }
  }
  // row operand = the one with >= 7 free bits (A unless only B qualifies)
  const bool swap = !(d.ka >= 7 && d.kb >= 5);
  const int row_op = swap ? 1 : 0;
  t.a_off = swap ? d.b_off : d.a_off;
  t.b_off = swap ? d.a_off : d.b_off;
  t.c_off = d.c_off;
  t.fa = swap ? d.kb : d.ka;
  t.fb = swap ? d.ka : d.kb;
  t.k = d.k;
  t.log_split = tc_split_log(d);
  for (int j = 0; j < d.c; j++) {
    if (op[j] == row_op) t.wm[dst[j]] = 1ull << j;
    else t.wn[dst[j]] = 1ull << j;
  }
  t.p = p;
  t.mu = ~0ull / p;
  uint64_t w = 1;
  for (int s = 0; s < 7; s++) {
    t.w256[s] = (uint32_t)w;
    w = w * 256 % p;
  }
  std::memcpy(out, &t, sizeof(t));
}

int tc_launch(const void* dev_step, const StepDesc& d, uint32_t* arena, uint32_t* part, uint32_t* dev_err,
              void* stream) {
  cudaStream_t st = (cudaStream_t)stream;
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(tnc_tc::tc_step_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)tnc_tc::kSmemBytes);
    if (e != cudaSuccess) return set_error(TNC_ERR_CUDA, std::string("tc attribute: ") + cudaGetErrorString(e));
    attr_set = true;
  }
  const bool swap = !(d.ka >= 7 && d.kb >= 5);
  const uint32_t fa = swap ? d.kb : d.ka, fb = swap ? d.ka : d.kb;
  const uint32_t ls = tc_split_log(d);
  const uint64_t tiles = ((1ull << (fa - 7)) * (1ull << (fb - 5))) << ls;
  if (tiles >= (1ull << 31)) return set_error(TNC_ERR_TOO_LARGE, "dense step has too many tiles");
  tnc_tc::tc_step_kernel<<<(unsigned)tiles, tnc_tc::kThreads, tnc_tc::kSmemBytes, st>>>(
      (const tnc_tc::TcStep*)dev_step, arena, part, dev_err);
  launch_counts().tc_gemm++;
  if (ls) launch_counts().tc_split++;
  if (ls) {
    const uint64_t n = 1ull << (fa + fb);
    tnc_tc::tc_split_final_kernel<<<(unsigned)std::min<uint64_t>((n + 255) / 256, 8192), 256, 0, st>>>(
        (const tnc_tc::TcStep*)dev_step, arena, part);
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return set_error(TNC_ERR_CUDA, std::string("tc launch: ") + cudaGetErrorString(e));
  return TNC_OK;
}

}  // namespace tnc
