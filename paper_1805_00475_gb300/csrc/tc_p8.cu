// Dense pairwise steps on the 5th-generation tensor cores with residues
// modulo primes below 2^8 (the TNC_PATH_TC_P8 arithmetic).
//
// A step C[m,n] = sum_q A[m,q] B[n,q] mod p (Sec. 2.1: the two tensors
// permuted and reshaped to matrices over their shared bonds) with p <= 251.
// Residues are taken balanced, |a|, |b| <= (p-1)/2 <= 125, and are exact as
// fp16; a product is at most 125^2 = 15625, so 1024 of them plus a residue
// left from an earlier reduction stay below 2^24 in magnitude, where every
// fp32 partial sum is an exact integer.  The fp32 tensor-core accumulator
// therefore takes K in chunks of 1024 exactly; after each chunk the epilogue
// warps read it from TMEM, reduce it modulo p (in fp32, exactly) and write the
// residue back, and the next chunk accumulates on top.  One residue is one
// 8-bit limb: one fp16 MMA per residue instead of the 16 limb pairs of a
// 30-bit residue (about 7.8 bits of the count per MMA against 1.9).
//
// Data path: tensors on this path hold one byte per residue (an entry is the
// RG residues of its pass side by side: 4 bytes for RG = 4).  A pack kernel
// turns the operands of a step that are still in entry form (the lowering's
// column-major layout: row index low, shared index high; all residues of the
// pass at once) into balanced fp16 planes, one per residue: in the entries'
// own order (rows contiguous) where the GEMM reads the operand MN-major
// (at least 64 shared values), else transposed so that the shared index is
// contiguous (K-major).  TMA moves boxes of 128-byte lines (64 shared values
// of a tile's rows, K-major; or 64 rows of 64 shared values, MN-major) into
// shared memory with the 128-byte swizzle, the canonical SWIZZLE_128B layouts
// of the MMA operand descriptors.
// An output that feeds another dense step is written straight as that
// step's fp16 planes (representatives of magnitude at most (p+1)/2, which
// keep its chunk sums exact).
// Persistent CTAs (one per SM, 576 threads) run three warp roles:
//   warp 0, lane 0: TMA producer over a ring of 3 to 8 shared-memory stages;
//   warp 1, lane 0: MMA issuer (kind::f16, 128 x TN x 16, fp32 in TMEM);
//   warps 2..17: epilogue (TMEM lane quarter = warp % 4, column group =
//   (warp - 2) / 4, a quarter of the tile's columns, at least 16).
// A work item is an output tile of 128 rows x TN columns (TN <= 256) and a K
// slice; NA = min(RG, 512 / TN) residues accumulate at once, one TMEM
// accumulator each, so one residue's reduction overlaps the next residue's
// MMAs.  256-wide tiles run on CTA pairs (clusters of two, one per SM): an
// item is then 256 rows x 256 columns, the leader CTA issues one
// cta_group::2 MMA (M = 256) over both CTAs' shared memory, each CTA staging
// its own 128 A rows and half of the B tile (32 KiB per stage instead of 48,
// four stages in flight instead of three) and reducing its own 128 TMEM
// lanes.  Items run K slice by K slice.  Every wait is bounded (about 2 s);
// on timeout the kernel records an error word, drains its own copies and
// MMAs, frees its TMEM and returns.
#include <cuda.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstring>
#include <string>
#include <type_traits>
#include <utility>
#include <vector>

#include "tnc_internal.h"

namespace tnc_p8 {

constexpr uint32_t kTileM = 128;
constexpr uint32_t kStageK = 64;
constexpr uint32_t kChunkK = 1024;
constexpr uint32_t kEpiWarps = 16;  // 4 per TMEM lane quarter, each a quarter of the columns
constexpr uint32_t kThreads = 64 + 32 * kEpiWarps;  // 2 role warps + the epilogue warps
constexpr uint32_t kEpiThreads = 32 * kEpiWarps;
constexpr uint32_t kABytes = kTileM * kStageK * 2;  // 16 KiB
// Staged entries per column of the output tile: at least the tile's 128 rows,
// padded so that a column's stride is an odd number of 32-bit words (entries
// of NA bytes: 132, 130 and 129 for NA = 1, 2, 4), which keeps both the
// staging writes (lanes along rows) and the reads (lanes along rows or
// along columns) free of bank conflicts.
__host__ __device__ constexpr uint32_t stage_pitch(uint32_t na) { return na == 4 ? 129u : (na == 2 ? 130u : 132u); }

// Shared-memory plan of a tile width: NA = min(RG, 512 / TN) residues
// accumulate together (NA TMEM accumulators of TN fp32 columns), in RG / NA
// rounds per tile; stages of A (16 KiB) + B (TN x 64 fp16), 1 KiB aligned for
// the 128-byte swizzle; the output staging holds NA bytes per entry of the
// tile; as many stages (up to 8) as fit next to it in 220 KiB (3 for
// TN = 256, 4 for TN = 128, more for narrow tiles, whose steps stream a tall
// operand and need more bytes in flight).
// PAIR (TN = 256 only): a CTA pair shares one M = 256 MMA and each CTA stages
// half of the B tile, so a stage is 16 + 16 KiB instead of 16 + 32 KiB and
// four stages fit instead of three.
template <uint32_t TN, uint32_t RG, bool PAIR = false>
struct Cfg {
  static constexpr uint32_t NA = RG * TN <= 512 ? RG : 512 / TN;
  static constexpr uint32_t kRounds = RG / NA;
  static constexpr uint32_t kRowsB = PAIR ? TN / 2 : TN;  // B rows (tile columns) staged by this CTA
  static constexpr uint32_t kStageBytes = (kABytes + kRowsB * kStageK * 2 + 1023u) / 1024u * 1024u;
  static constexpr uint32_t kStagePitch = stage_pitch(NA);
  static constexpr uint32_t kStagingBytes = (TN * kStagePitch * NA + 15u) / 16u * 16u;
  static constexpr uint32_t kFit = (220u * 1024u - kStagingBytes) / kStageBytes;
  static constexpr uint32_t kStages = kFit > 8 ? 8 : kFit;
  static constexpr uint32_t kSmemBytes = kStages * kStageBytes + kStagingBytes + 1024;
};
// the NA-byte word of a staged entry
template <uint32_t NA>
using StageWord = std::conditional_t<NA == 4, uint32_t, std::conditional_t<NA == 2, uint16_t, uint8_t>>;
constexpr uint64_t kWaitNs = 2000000000ull;

struct P8Args {
  uint32_t fa, fb, k, log_split;  // rows 2^fa, columns 2^fb, shared 2^k, K split 2^log_split
  uint32_t n_items, tiles_m;      // work items (tiles x splits); row tiles
  uint32_t rg, gm_log;            // residues per entry (1, 2 or 4), computed together; row tiles per raster group (log2)
  uint32_t p[4];
  float pf[4], invp[4];
  uint64_t wm[32], wn[32];  // output address weight of row bit j / column bit j
  uint8_t ebit[16];         // the tile's row and column bits by output weight, lightest first
                            // (column bit j: 0x80 | j; row bit j: j); bits 0..4 go to lanes
  uint32_t n_ebits, pad3;
  uint32_t a_mn, b_mn;      // operand planes row-contiguous (MN-major) instead of K-contiguous
  uint32_t direct;          // output as rg balanced fp16 planes, plane i at out + i 2^(fa+fb) halves
  uint32_t pairs;           // row bit 0 has output weight 1: entries written two at a time (TN >= 32)
  uint8_t* out;             // C (entry o at out[o * rg]), or the split partials [split][2^(fa+fb) * rg]
};

// ---- PTX helpers -----------------------------------------------------------

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t gtimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void mbar_init(uint32_t mbar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(mbar), "r"(count) : "memory");
}

__device__ __forceinline__ bool mbar_try(uint32_t mbar, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.b32 %0, 1, 0, p;\n\t}\n"
      : "=r"(done)
      : "r"(mbar), "r"(parity)
      : "memory");
  return done != 0;
}

// Bounded wait for the phase of parity `parity`; false after ~2 s (or 2^26
// polls if the timer were not to advance).
__device__ __noinline__ bool mbar_wait(uint32_t mbar, uint32_t parity) {
  if (mbar_try(mbar, parity)) return true;
  const uint64_t t0 = gtimer();
  for (uint32_t i = 0; i < (1u << 26); i++) {
    if (mbar_try(mbar, parity)) return true;
    if ((i & 63u) == 63u && gtimer() - t0 > kWaitNs) return false;
  }
  return false;
}

__device__ __forceinline__ void mbar_arrive(uint32_t mbar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(mbar) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t mbar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mbar), "r"(bytes) : "memory");
}

// ---- CTA pairs (clusters of two CTAs sharing one tcgen05 MMA) --------------

__device__ __forceinline__ uint32_t cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}

// Every thread of both CTAs of the cluster (release / acquire).
__device__ __forceinline__ void cluster_sync() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// The shared::cluster address of the same shared-memory offset in the CTA
// of cluster rank `rank`.
__device__ __forceinline__ uint32_t mapa_cluster(uint32_t saddr, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(saddr), "r"(rank));
  return r;
}

// try_wait with cluster-scope acquire: the phase was completed by arrivals
// of both CTAs of the pair (their tcgen05 stores are then visible).
__device__ __forceinline__ bool mbar_try_cl(uint32_t mbar, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.b32 %0, 1, 0, p;\n\t}\n"
      : "=r"(done)
      : "r"(mbar), "r"(parity)
      : "memory");
  return done != 0;
}

// Bounded cluster-scope wait, as mbar_wait.
__device__ __noinline__ bool mbar_wait_cl(uint32_t mbar, uint32_t parity) {
  if (mbar_try_cl(mbar, parity)) return true;
  const uint64_t t0 = gtimer();
  for (uint32_t i = 0; i < (1u << 26); i++) {
    if (mbar_try_cl(mbar, parity)) return true;
    if ((i & 63u) == 63u && gtimer() - t0 > kWaitNs) return false;
  }
  return false;
}

// One arrival on the mbarrier at the shared::cluster address `cmbar` (this
// CTA's or the peer's).  Default semantics (release at CTA scope): the
// arrival follows the thread's completed tcgen05 loads and stores (waited for
// and fenced before it); a cluster-scope release would also wait for the
// thread's global stores in flight, which the MMA never reads.
__device__ __forceinline__ void mbar_arrive_cluster(uint32_t cmbar) {
  asm volatile("mbarrier.arrive.shared::cluster.b64 _, [%0];" ::"r"(cmbar) : "memory");
}

// 3-D tiled TMA load of the box at (x, y, z) into shared memory, completing
// on mbar with its byte count.
__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap* map, int32_t x, int32_t y, int32_t z,
                                            uint32_t mbar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::
          "r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(mbar)
      : "memory");
}

// The same load into this CTA's shared memory, completing on the mbarrier at
// the shared::cluster address `cmbar`, which may lie in the peer CTA of the
// pair (the pair's leader counts both CTAs' bytes on one barrier).
__device__ __forceinline__ void tma_load_3d_pair(uint32_t dst, const CUtensorMap* map, int32_t x, int32_t y, int32_t z,
                                                 uint32_t cmbar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.cta_group::2.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(cmbar)
      : "memory");
}

// 2-D tiled TMA load of the box at (x, y) into shared memory, completing on
// mbar with its byte count.
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int32_t x, int32_t y,
                                            uint32_t mbar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(mbar)
      : "memory");
}

// Shared-memory matrix descriptor of a K-major operand in the 128-byte
// swizzle layout: rows of 64 fp16 (128 bytes), 8-row atoms of 1024 bytes
// (SBO = 1024; LBO unused for this layout, set to 16 bytes); version 1;
// layout type 2 (SWIZZLE_128B).  The tile base is 1024-byte aligned; the
// K-th group of 16 values starts 32 K bytes further (the swizzle applies to
// the address bits, so the start simply advances within the atom).
__device__ __forceinline__ uint64_t make_desc_sw128(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)1 << 16;
  d |= (uint64_t)(1024u >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;
  return d;
}

// The same for an MN-major operand (rows contiguous): each 128-byte line
// holds 64 consecutive rows at one shared value, 8 lines (shared values) form
// a 1024-byte swizzle atom; the tile's atoms run along K at 1024 bytes (the
// stride byte offset) and along the rows at 8192 bytes (the leading byte
// offset: one TMA box of 64 rows x 64 shared values).  The ks-th group of 16
// shared values starts 2048 ks bytes further.
__device__ __forceinline__ uint64_t make_desc_mn_sw128(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)(8192u >> 4) << 16;
  d |= (uint64_t)(1024u >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;
  return d;
}

// Instruction descriptor, kind::f16: D = F32, A = B = F16, K-major unless
// the transpose bit of A (15) or B (16) marks it MN-major, N >> 3 at bits
// 17-22, M >> 4 at bits 24-28.
__host__ __device__ constexpr uint32_t make_idesc(uint32_t M, uint32_t N, uint32_t a_mn = 0, uint32_t b_mn = 0) {
  return (1u << 4) | (a_mn << 15) | (b_mn << 16) | ((N >> 3) << 17) | ((M >> 4) << 24);
}

// PAIR: one MMA of the CTA pair (cta_group::2), M = 256 rows, A's rows and
// B's rows (tile columns) split between the two CTAs' shared memory at the
// same offsets, the accumulator in both CTAs' TMEM (128 lanes each).
template <bool PAIR>
__device__ __forceinline__ void mma_f16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                        uint32_t accumulate) {
  if constexpr (PAIR)
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate));
  else
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate));
}

// One arrival on this CTA's mbarrier once the MMAs issued so far are done.
template <bool PAIR>
__device__ __forceinline__ void mma_commit(uint32_t mbar) {
  if constexpr (PAIR)
    asm volatile("tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
                 : "memory");
  else
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
                 : "memory");
}

// PAIR: the same arrival on the mbarrier at offset mbar of both CTAs.
__device__ __forceinline__ void mma_commit_both(uint32_t mbar) {
  asm volatile(
      "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;" ::"r"(mbar),
      "h"((uint16_t)3)
      : "memory");
}

template <bool PAIR>
__device__ __forceinline__ void tmem_alloc(uint32_t dst_smem, uint32_t cols) {
  if constexpr (PAIR) {
    asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(dst_smem), "r"(cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
  } else {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(dst_smem), "r"(cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
}

template <bool PAIR>
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t cols) {
  if constexpr (PAIR)
    asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(cols) : "memory");
  else
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(cols) : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&v)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]), "=r"(v[8]),
        "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
      : "r"(taddr));
}

__device__ __forceinline__ void tmem_st16(uint32_t taddr, const uint32_t (&v)[16]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};" ::"r"(
          taddr),
      "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7]), "r"(v[8]), "r"(v[9]),
      "r"(v[10]), "r"(v[11]), "r"(v[12]), "r"(v[13]), "r"(v[14]), "r"(v[15])
      : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// x (an exact integer, as fp32) reduced modulo p to a representative of
// magnitude at most (p+1)/2: q is x (1/p) rounded to nearest, and the fma is
// exact.  Operands are representatives of magnitude at most (p+1)/2 <= 126
// (balanced residues, or this function's own outputs), so an accumulator
// holds at most 1024 126^2 + 126 < 2^24 in magnitude (one chunk of products
// on top of a reduced remainder), where fp32 sums are exact, and
// |x| / p < 2^16, so x (1/p) is within 2^-8 of x / p: q is off by one only
// next to a half, and then |r| <= p/2 + p 2^-8 < p/2 + 1.  The rounding adds
// 1.5 2^23 inside the fma (the spacing of floats there is 1) and takes it off
// again: no float-to-integer conversion.
constexpr float kMagic = 12582912.0f;     // 1.5 * 2^23
constexpr float kMagic128 = 12583040.0f;  // 1.5 * 2^23 + 128
__device__ __forceinline__ float reduce_p(float x, float pf, float invp) {
  const float q = fmaf(x, invp, kMagic) - kMagic;
  return fmaf(-q, pf, x);
}

// The canonical residue v in [0, p) of such a representative r (magnitude
// below p), as the low byte of a float's bits: r + 1.5 2^23 (plus p when r
// is negative) is the float 1.5 2^23 + v, exact (the spacing there is 1),
// whose bits are 0x4B400000 + v.  pm = 1.5 2^23 + p.  No float-to-integer
// conversion.
__device__ __forceinline__ uint32_t canonical_bits(float r, float pm) {
  return __float_as_uint(r + (r < 0.0f ? pm : kMagic));
}

// The representative r itself (|r| <= (p+1)/2 <= 126), offset by 128, as the
// low byte of a float's bits: r + 128 + 1.5 2^23 is exact, with bits
// 0x4B400000 + r + 128 (2 <= r + 128 <= 254).  Outputs that a dense step reads
// as fp16 planes are staged this way: any representative of magnitude at most
// (p+1)/2 keeps that step's chunk sums exact (reduce_p).
__device__ __forceinline__ uint32_t offset_bits(float r) { return __float_as_uint(r + kMagic128); }

// fp16 values of such staged bytes b: the half with bits 0x6400 | b is
// 1024 + b exactly, and one packed add of -1152 leaves r = b - 128 (exact).
// staged_half2: byte ra of the entries o (in w0) and o + 1 (in w1 when the
// staged word holds 4 residues, else in w0 above o's NA bytes) as a half2.
__device__ __forceinline__ uint32_t add_m1152(uint32_t h2) {  // both halves minus 1152 (0xE480)
  uint32_t r;
  asm("add.rn.f16x2 %0, %1, %2;" : "=r"(r) : "r"(h2), "r"(0xE480E480u));
  return r;
}
template <uint32_t NA>
__device__ __forceinline__ uint32_t staged_half2(uint32_t w0, uint32_t w1, uint32_t ra) {
  uint32_t t;
  if constexpr (NA == 4) {
    t = (__byte_perm(w0, w1, ra | ((4u + ra) << 8)) & 0x00FF00FFu) | 0x64006400u;
  } else {
    t = __byte_perm(w0, 0x64646464u, ra | (4u << 4) | ((NA + ra) << 8) | (4u << 12));
  }
  return add_m1152(t);
}
// bytes ra and ra + 1 of one entry's staged word as a half2 (low: residue ra)
__device__ __forceinline__ uint32_t staged_half2_res(uint32_t w, uint32_t ra) {
  uint32_t t = __byte_perm(w, 0x64646464u, ra | (4u << 4) | ((ra + 1u) << 8) | (4u << 12));
  return add_m1152(t);
}

// ---- operand packing ------------------------------------------------------

// X: the operand's residues in [0, p_i), one byte each, entry q * R + r at
// X + (q * R + r) * RG (R = 2^f >= 16 rows, K = 2^k shared values, RG
// residues per entry); Y_i (i < RG, Y_i = Y + i * R * Kp): balanced fp16
// residues mod p_i.  K-contiguous planes (mode 1): Y_i[r * Kp + q] with rows
// padded to Kp = max(K, 64) values by zeros; a block transposes tiles of 64
// rows x 64 shared values through shared memory: a thread reads the entries
// of 4 consecutive rows at shared values q and q + 1 (4 RG bytes each,
// coalesced along r) and builds, for each row and residue, the half2
// (Y_i[r][q], Y_i[r][q+1]); 16-byte writes are coalesced along q.
// Row-contiguous planes (mode 2, K >= 64): Y_i[q * R + r], the entries' own
// order, converted in place of the transpose (8-byte writes along r).
struct PackPrimes {
  uint32_t p[4];
};

// half2 of the balanced residues (a, b) given as bytes ia of wa and ib of wb:
// 0x64XX is the half 1024 + XX exactly, so one subtraction gives a, b as
// halves, and v - p [v > (p-1)/2] is exact in fp16 (|v| <= 250).
__device__ __forceinline__ uint32_t p8_half2(uint32_t wa, uint32_t ia, uint32_t wb, uint32_t ib, __half2 hp2,
                                             __half2 np2) {
  uint32_t t = __byte_perm(wa, wb, ia | ((4u + ib) << 8));
  t = (t & 0x00FF00FFu) | 0x64006400u;  // byte 0 -> low half, byte 1 -> high half
  __half2 h;
  *reinterpret_cast<uint32_t*>(&h) = t;
  h = __hsub2(h, __halves2half2(__ushort_as_half(0x6400), __ushort_as_half(0x6400)));
  h = __hfma2(__hgt2(h, hp2), np2, h);
  return *reinterpret_cast<uint32_t*>(&h);
}

// One operand of a dense step to pack: X its byte entries, Y its RG planes,
// 2^f rows; mode 0: nothing to do (the producing step wrote the planes),
// 1: K-contiguous planes (the transpose above), 2: row-contiguous planes,
// Y_i[q * R + r] (no transpose: the entries' own order, K >= 64).
struct PackOperand {
  const uint8_t* X;
  __half* Y;
  uint32_t f, mode;
};

// Both operands of a step in one launch: the tiles of A, then those of B.
template <int RG>
__global__ void __launch_bounds__(256) p8_pack_kernel(PackOperand opA, PackOperand opB, uint32_t k, uint32_t kp,
                                                      PackPrimes pp) {
  // [residue][row][pair of shared values] half2 words; a row is 32 words + 1
  // of padding, so both phases are free of bank conflicts (phase 1: lanes =
  // 8 row quads x 4 pairs; phase 2: lanes = 8 chunks x 4 rows)
  __shared__ uint32_t tile[RG][64][33];
  const uint32_t K = 1u << k, Kp = 1u << kp;
  const uint64_t tiles_a = opA.mode ? (uint64_t)(((1u << opA.f) + 63u) / 64u) << (kp - 6) : 0;
  const uint64_t n_tiles = tiles_a + (opB.mode ? (uint64_t)(((1u << opB.f) + 63u) / 64u) << (kp - 6) : 0);
  const uint32_t t = threadIdx.x, lane = t & 31u, warp = t >> 5;
  __half2 hp2[RG], np2[RG];
#pragma unroll
  for (int i = 0; i < RG; i++) {
    hp2[i] = __float2half2_rn((float)((pp.p[i] - 1) / 2));
    np2[i] = __float2half2_rn(-(float)pp.p[i]);
  }
  for (uint64_t bt = blockIdx.x; bt < n_tiles; bt += gridDim.x) {
    const bool isA = bt < tiles_a;  // uniform over the block
    const uint8_t* __restrict__ X = isA ? opA.X : opB.X;
    __half* __restrict__ Y = isA ? opA.Y : opB.Y;
    const uint32_t R = 1u << (isA ? opA.f : opB.f);
    const uint32_t tiles_r = (R + 63) / 64;
    const uint64_t b = isA ? bt : bt - tiles_a;
    const uint32_t r0 = (uint32_t)(b % tiles_r) * 64u, q0 = (uint32_t)(b / tiles_r) * 64u;
    if ((isA ? opA.mode : opB.mode) == 2) {  // row-contiguous: 64 shared values x 16 quads of rows
#pragma unroll
      for (int it = 0; it < 4; it++) {
        const uint32_t id = t + 256u * it;
        const uint32_t r = r0 + 4u * (id & 15u), q = q0 + (id >> 4);
        if (r < R) {
          const uint8_t* src = X + ((uint64_t)q * R + r) * RG;
          uint32_t w[RG];  // 4 rows x RG bytes
          if constexpr (RG == 4) {
            const uint4 v = *reinterpret_cast<const uint4*>(src);
            w[0] = v.x; w[1] = v.y; w[2] = v.z; w[3] = v.w;
          } else if constexpr (RG == 2) {
            const uint2 v = *reinterpret_cast<const uint2*>(src);
            w[0] = v.x; w[1] = v.y;
          } else {
            w[0] = *reinterpret_cast<const uint32_t*>(src);
          }
#pragma unroll
          for (int i = 0; i < RG; i++) {
            const uint32_t b0 = (uint32_t)i, b1 = (uint32_t)(RG + i), b2 = (uint32_t)(2 * RG + i),
                           b3 = (uint32_t)(3 * RG + i);  // byte of row j, residue i
            uint2 h;
            h.x = p8_half2(w[b0 >> 2], b0 & 3u, w[b1 >> 2], b1 & 3u, hp2[i], np2[i]);
            h.y = p8_half2(w[b2 >> 2], b2 & 3u, w[b3 >> 2], b3 & 3u, hp2[i], np2[i]);
            *reinterpret_cast<uint2*>(Y + (uint64_t)i * R * Kp + (uint64_t)q * R + r) = h;
          }
        }
      }
      continue;
    }
#pragma unroll
    for (int it = 0; it < 2; it++) {
      const uint32_t rq = (lane & 7u) + 8u * (warp & 1u);                // row quad 0..15
      const uint32_t qp = (lane >> 3) + 4u * ((warp >> 1) + 4u * it);   // pair 0..31
      const uint32_t r = r0 + 4u * rq, q = q0 + 2u * qp;
      if (r < R) {  // R is a multiple of 16: a quad is wholly in or out
        uint32_t w0[RG], w1[RG];  // 4 rows x RG bytes at q and at q + 1
#pragma unroll
        for (int h = 0; h < 2; h++) {
          uint32_t* w = h ? w1 : w0;
          if (q + h < K) {
            const uint8_t* src = X + ((uint64_t)(q + h) * R + r) * RG;
            if constexpr (RG == 4) {
              const uint4 v = *reinterpret_cast<const uint4*>(src);
              w[0] = v.x; w[1] = v.y; w[2] = v.z; w[3] = v.w;
            } else if constexpr (RG == 2) {
              const uint2 v = *reinterpret_cast<const uint2*>(src);
              w[0] = v.x; w[1] = v.y;
            } else {
              w[0] = *reinterpret_cast<const uint32_t*>(src);
            }
          } else {
#pragma unroll
            for (int i = 0; i < RG; i++) w[i] = 0;
          }
        }
#pragma unroll
        for (int j = 0; j < 4; j++)
#pragma unroll
          for (int i = 0; i < RG; i++) {
            const uint32_t idx = (uint32_t)(j * RG + i);  // byte of row j, residue i in the quad
            tile[i][4u * rq + j][qp] = p8_half2(w0[idx >> 2], idx & 3u, w1[idx >> 2], idx & 3u, hp2[i], np2[i]);
          }
      }
    }
    __syncthreads();
#pragma unroll
    for (int it = 0; it < 2 * RG; it++) {  // RG planes x 64 rows x 8 chunks of 16 bytes
      const uint32_t id = t + 256u * it;
      const uint32_t c = id & 7u, row = (id >> 3) & 63u, i = id >> 9;
      if (r0 + row < R) {
        const uint32_t* src = &tile[i][row][4u * c];
        uint4 w;
        w.x = src[0];
        w.y = src[1];
        w.z = src[2];
        w.w = src[3];
        *reinterpret_cast<uint4*>(Y + (uint64_t)i * R * Kp + (uint64_t)(r0 + row) * Kp + q0 + 8u * c) = w;
      }
    }
    __syncthreads();
  }
}

// Sum of the K-split partials: C[i] = sum_j part[j][i] mod p_(i mod rg) for
// the n = 2^c * rg residues (bytes) of the step's output.
__global__ void p8_split_final_kernel(const uint8_t* __restrict__ part, uint8_t* __restrict__ C, uint32_t c,
                                      uint32_t log_split, uint32_t rg, uint4 primes) {
  const uint64_t n = (uint64_t)rg << c;
  const uint32_t pr[4] = {primes.x, primes.y, primes.z, primes.w};
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
    uint32_t s = 0;
    for (uint32_t j = 0; j < (1u << log_split); j++) s += part[(uint64_t)j * n + i];
    C[i] = (uint8_t)(s % pr[i % rg]);
  }
}

// ---- the GEMM -------------------------------------------------------------

// Origin of output tile `tile`: the tiles are taken in groups of 2^gm_log
// row tiles, column tiles outermost within a group, row tiles fastest, so
// that the CTAs running at one time share the operand rows of a few row tiles
// and of a few column tiles.
// Row tiles are 128 rows (PAIR: 256, the pair's two 128-row halves).
template <uint32_t TN, bool PAIR>
__device__ __forceinline__ void tile_origin(uint32_t tile, const P8Args& g, uint32_t& m0, uint32_t& n0) {
  const uint32_t gm = g.gm_log, per_group = (g.n_items >> g.log_split) >> (31 - __clz(g.tiles_m) - gm);
  const uint32_t grp = tile / per_group, w = tile - grp * per_group;
  m0 = ((grp << gm) + (w & ((1u << gm) - 1u))) * (PAIR ? 2u * kTileM : kTileM);
  n0 = (w >> gm) * TN;
}

__device__ __forceinline__ void epi_bar() { asm volatile("bar.sync 1, %0;" ::"n"(kEpiThreads) : "memory"); }

// One CTA per SM.  Work item = (output tile of 128 rows x TN columns, K
// slice); for each item, each round of NA residues, each K chunk and each
// residue r of the round (in that order) the MMA warp accumulates chunk c of
// C_r = A_r B_r^T into TMEM accumulator r mod NA (columns (r mod NA) TN ..).
// The epilogue reduces an accumulator in place after every chunk but the
// last; after the last it turns it into canonical residues, staged in shared
// memory as one byte per residue of each entry, and frees the accumulator at
// once, so the next MMAs start while the staged bytes are written out (NA
// residue bytes of each entry per round, the pass's layout: RG bytes per
// entry).
//
// PAIR: clusters of two CTAs take work items of 256 rows x TN columns; CTA
// rank q holds rows 128 q .. 128 q + 127 of the item (its A rows, its TMEM
// lanes, its epilogue) and tile columns (TN / 2) q .. of the B tile.  The
// leader (rank 0) issues the pair's M = 256 MMAs (cta_group::2); both
// producers' copies complete on the leader's stage barrier (expecting both
// CTAs' bytes), the leader's commits arrive on both CTAs' stage-free and
// accumulator-full barriers, and one lane of each epilogue warp of both CTAs
// arrives on the leader's accumulator-free barrier.
template <uint32_t TN, uint32_t RG, bool PAIR>
__global__ void __launch_bounds__(kThreads, 1)
    p8_gemm_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                   const __grid_constant__ P8Args g, uint32_t* err) {
  static_assert(!PAIR || TN == 256, "CTA pairs for 256-wide tiles");
  using C = Cfg<TN, RG, PAIR>;
  constexpr uint32_t kStages = C::kStages, kStageBytes = C::kStageBytes, NA = C::NA, kRounds = C::kRounds;
  using SW = StageWord<NA>;
  constexpr uint32_t kStagePitch = C::kStagePitch;
  extern __shared__ uint8_t smem_raw[];
  __shared__ __align__(8) uint64_t bars[2 * kStages + 2 * NA + 1];
  __shared__ uint32_t tmem_base_s;
  // per index h of the entry bits above the lane bits: their part of the
  // entry's output offset (x) and of its staging index (y)
  __shared__ uint2 ho_tab[kTileM * TN / 32];
  uint8_t* smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
  SW* staging = reinterpret_cast<SW*>(smem + kStages * kStageBytes);  // [col][kStagePitch] entries of NA bytes
  const uint32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31u;
  const uint32_t full0 = smem_u32(&bars[0]), empty0 = smem_u32(&bars[kStages]);
  const uint32_t accf0 = smem_u32(&bars[2 * kStages]), acce0 = smem_u32(&bars[2 * kStages + NA]);
  const uint32_t drain = smem_u32(&bars[2 * kStages + 2 * NA]);
  constexpr uint32_t kCols = NA * TN < 32 ? 32 : NA * TN;  // NA accumulators of TN columns
  if (threadIdx.x == 0) {
    for (uint32_t s = 0; s < kStages; s++) {
      mbar_init(full0 + 8 * s, 1);
      mbar_init(empty0 + 8 * s, 1);
    }
    for (uint32_t r = 0; r < NA; r++) {
      mbar_init(accf0 + 8 * r, 1);
      mbar_init(acce0 + 8 * r, PAIR ? 2 * kEpiWarps : kEpiThreads);
    }
    mbar_init(drain, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) tmem_alloc<PAIR>(smem_u32(&tmem_base_s), kCols);  // PAIR: both CTAs' warp 1 together
  tc_fence_before();
  __syncthreads();
  if constexpr (PAIR) cluster_sync();  // the peer's barriers exist before any copy, commit or arrival reaches them
  tc_fence_after();
  const uint32_t tmem = tmem_base_s;
  const uint32_t crank = PAIR ? cluster_rank() : 0u;
  const bool leader = crank == 0;

  const uint32_t G = gridDim.x / (PAIR ? 2u : 1u), bid = blockIdx.x / (PAIR ? 2u : 1u);
  const uint32_t T = g.n_items > bid ? (g.n_items - bid + G - 1) / G : 0;
  const uint32_t Ks = (1u << g.k) >> g.log_split;
  const uint32_t chunk = Ks < kChunkK ? Ks : kChunkK;
  const uint32_t n_chunks = Ks / chunk;
  const uint32_t spc = chunk / kStageK;  // stages per chunk
  // items run K slice by K slice (split-major): the items of one wave share
  // their slice's operand rows in L2
  const uint32_t tile_bits = 31u - __clz(g.n_items >> g.log_split), tile_mask = (1u << tile_bits) - 1u;
  // row-contiguous operands (a tile of TN < 64 columns always reads B K-contiguous)
  const bool a_mn = g.a_mn != 0, b_mn = TN >= 64 && g.b_mn != 0;
  bool ok = true;

  if (warp == 0) {
    if (lane == 0) {  // TMA producer
      uint32_t s = 0, ph = 0, issued = 0;
      for (uint32_t t = 0; t < T && ok; t++) {
        const uint32_t item = bid + t * G;
        const uint32_t split = item >> tile_bits, tile = item & tile_mask;
        uint32_t m0, n0;
        tile_origin<TN, PAIR>(tile, g, m0, n0);
        m0 += crank * kTileM;                  // this CTA's rows
        n0 += crank * C::kRowsB;               // this CTA's part of the B tile
        for (uint32_t rd = 0; rd < kRounds && ok; rd++)
        for (uint32_t c = 0; c < n_chunks && ok; c++)
          for (uint32_t ra = 0; ra < NA && ok; ra++) {
            const uint32_t r = rd * NA + ra;
            const uint32_t q0 = split * Ks + c * chunk;
            for (uint32_t j = 0; j < spc; j++) {
              if (!mbar_try(empty0 + 8 * s, ph ^ 1u) && !mbar_wait(empty0 + 8 * s, ph ^ 1u)) {
                ok = false;
                break;
              }
              const uint32_t sa = smem_u32(smem + s * kStageBytes);
              const int32_t x = (int32_t)(q0 + j * kStageK);
              // PAIR: the stage's copies of both CTAs complete on the leader's barrier
              const uint32_t fb = PAIR ? mapa_cluster(full0 + 8 * s, 0) : full0 + 8 * s;
              if (leader) mbar_expect_tx(full0 + 8 * s, (PAIR ? 2u : 1u) * (kTileM + C::kRowsB) * kStageK * 2u);
              auto load = [&](uint32_t dst, const CUtensorMap* map, int32_t cx, int32_t cy) {
                if constexpr (PAIR) tma_load_3d_pair(dst, map, cx, cy, (int32_t)r, fb);
                else tma_load_3d(dst, map, cx, cy, (int32_t)r, fb);
              };
              // K-contiguous planes: one box of rows x 64 shared values;
              // row-contiguous: boxes of 64 rows x 64 shared values, 8 KiB apart
              if (a_mn) {
                load(sa, &tmA, (int32_t)m0, x);
                load(sa + 8192u, &tmA, (int32_t)m0 + 64, x);
              } else {
                load(sa, &tmA, x, (int32_t)m0);
              }
              if (b_mn) {
                for (uint32_t h = 0; 64u * h < C::kRowsB; h++)
                  load(sa + kABytes + 8192u * h, &tmB, (int32_t)(n0 + 64u * h), x);
              } else {
                load(sa + kABytes, &tmB, x, (int32_t)n0);
              }
              issued++;
              if (++s == kStages) {
                s = 0;
                ph ^= 1u;
              }
            }
          }
      }
      // every copy issued has landed before the CTA can exit (PAIR: the
      // leader's barriers count the peer's copies too; the peer stays until
      // the leader reaches the final cluster barrier)
      for (uint32_t s2 = 0; s2 < kStages && s2 < issued && leader; s2++) {
        const uint32_t uses = issued / kStages + (s2 < issued % kStages ? 1u : 0u);
        if (!mbar_wait(full0 + 8 * s2, (uses - 1u) & 1u)) ok = false;
      }
      if (!ok) atomicExch(err, 1u);
      // PAIR, after a failed wait: copies this CTA issued may not have been
      // consumed, and their barrier is the leader's, which this thread cannot
      // wait on; about 1 ms for them to land before the CTAs can exit
      if (PAIR && !ok)
        for (int i = 0; i < 1000; i++) __nanosleep(1000);
    }
  } else if (warp == 1) {
    if (lane == 0 && leader) {  // MMA issuer (PAIR: the leader's, for both CTAs)
      const uint32_t idesc = make_idesc(PAIR ? 2u * kTileM : kTileM, TN, a_mn ? 1u : 0u, b_mn ? 1u : 0u);
      const uint32_t a_ks = a_mn ? 2048u >> 4 : 32u >> 4, b_ks = b_mn ? 2048u >> 4 : 32u >> 4;
      uint32_t s = 0, ph = 0, par = 0;  // bit r: phase parity of accumulator r
      for (uint32_t t = 0; t < T && ok; t++)
        for (uint32_t rd = 0; rd < kRounds && ok; rd++)
        for (uint32_t c = 0; c < n_chunks && ok; c++)
          for (uint32_t r = 0; r < NA && ok; r++) {
            // the epilogue (PAIR: both CTAs' epilogues) is done with accumulator r
            const uint32_t pr = ((par >> r) & 1u) ^ 1u;
            if (!(PAIR ? mbar_wait_cl(acce0 + 8 * r, pr) : mbar_wait(acce0 + 8 * r, pr))) {
              ok = false;
              break;
            }
            tc_fence_after();
            const uint32_t d = tmem + r * TN;
            for (uint32_t j = 0; j < spc; j++) {
              if (!mbar_try(full0 + 8 * s, ph) && !mbar_wait(full0 + 8 * s, ph)) {
                ok = false;
                break;
              }
              tc_fence_after();
              const uint32_t sa = smem_u32(smem + s * kStageBytes), sb = sa + kABytes;
              const uint64_t ad = a_mn ? make_desc_mn_sw128(sa) : make_desc_sw128(sa);
              const uint64_t bd = b_mn ? make_desc_mn_sw128(sb) : make_desc_sw128(sb);
#pragma unroll
              for (uint32_t ks = 0; ks < kStageK / 16; ks++)  // the ks-th 16 K values
                mma_f16<PAIR>(d, ad + a_ks * ks, bd + b_ks * ks, idesc, (c | j | ks) ? 1u : 0u);
              // the stage (PAIR: in both CTAs) is free once these MMAs are done
              if constexpr (PAIR) mma_commit_both(empty0 + 8 * s);
              else mma_commit<false>(empty0 + 8 * s);
              if (++s == kStages) {
                s = 0;
                ph ^= 1u;
              }
            }
            if (!ok) break;
            if constexpr (PAIR) mma_commit_both(accf0 + 8 * r);
            else mma_commit<false>(accf0 + 8 * r);
            par ^= 1u << r;
          }
      // every MMA issued has completed before the TMEM is freed
      mma_commit<PAIR>(drain);
      if (!mbar_wait(drain, 0)) ok = false;
      if (!ok) atomicExch(err, 1u);
    }
  } else {
    // epilogue: warps 2..17; TMEM lanes 32 (warp % 4) .., column group (warp - 2) / 4.
    // Every epilogue thread runs the same loop trips and named barriers; a
    // failed wait only turns the thread's work off.
    const uint32_t et = threadIdx.x - 64u;
    const uint32_t quarter = warp & 3u;
    const uint32_t row = quarter * 32u + lane;
    // columns per epilogue warp: the tile's columns shared by the warps of a
    // lane quarter, at least 16 per warp (the rest of the warps idle)
    constexpr uint32_t kGroups = kEpiWarps / 4 < TN / 16 ? kEpiWarps / 4 : TN / 16;
    constexpr uint32_t kHalf = TN / kGroups;
    constexpr uint32_t kBatch = kHalf >= 32 ? 32 : 16;  // columns per TMEM load batch
    const uint32_t cbeg = ((warp - 2u) >> 2) * kHalf;
    const bool idle = cbeg >= TN;
    uint8_t* stage8 = reinterpret_cast<uint8_t*>(staging);
    // write order of a tile's entries: entry index e has the tile's row and
    // column bits ordered by output weight, so consecutive e are as close in C
    // as the step's bit map allows (lane bits: the five lightest).  An
    // entry's output offset is a sum of one weight per set row or column bit,
    // so it splits into the tile's base (the bits of m0 and n0), the lane
    // bits' part and the part of the bits above them (ho_tab, the same for
    // every tile: below 2^c <= 2^32); its staging index splits the same way.
    // With pairs, entry bit 0 is row bit 0 (output weight 1): a thread takes
    // the two entries o, o + 1, adjacent in the staging and in C, and the
    // lane and table bits start one higher.
    const uint32_t pv = (TN >= 32 && g.pairs) ? 1u : 0u;
    uint32_t lane_off = 0, lane_sid = 0;
    for (uint32_t i = 0; i < 5; i++) {
      if (!((lane >> i) & 1u)) continue;
      const uint32_t b = g.ebit[pv + i];
      if (b & 0x80u) {
        lane_off += (uint32_t)g.wn[b & 31u];
        lane_sid += kStagePitch << (b & 31u);
      } else {
        lane_off += (uint32_t)g.wm[b];
        lane_sid += 1u << b;
      }
    }
    for (uint32_t h = et; h < (kTileM * TN / 32) >> pv; h += kEpiThreads) {
      uint32_t off = 0, sid = 0;
      for (uint32_t i = 5 + pv; i < g.n_ebits; i++) {
        if (!((h >> (i - 5 - pv)) & 1u)) continue;
        const uint32_t b = g.ebit[i];
        if (b & 0x80u) {
          off += (uint32_t)g.wn[b & 31u];
          sid += kStagePitch << (b & 31u);
        } else {
          off += (uint32_t)g.wm[b];
          sid += 1u << b;
        }
      }
      ho_tab[h] = make_uint2(off, sid);
    }
    constexpr uint32_t kLogTN = TN == 256 ? 8 : TN == 128 ? 7 : TN == 64 ? 6 : TN == 32 ? 5 : 4;
    uint32_t par = 0;  // bit ra: phase parity of accumulator ra
    for (uint32_t t = 0; t < T; t++) {
      const uint32_t item = bid + t * G;
      const uint32_t split = item >> tile_bits, tile = item & tile_mask;
      uint32_t m0, n0;
      tile_origin<TN, PAIR>(tile, g, m0, n0);
      m0 += crank * kTileM;  // PAIR: this CTA's 128 rows of the item (its TMEM lanes)
      uint64_t tile_base = lane_off;  // output offset of the tile's origin + the lane bits' part
      for (uint32_t j = 7; j < g.fa; j++)
        if ((m0 >> j) & 1u) tile_base += g.wm[j];
      for (uint32_t j = kLogTN; j < g.fb; j++)
        if ((n0 >> j) & 1u) tile_base += g.wn[j];
      for (uint32_t rd = 0; rd < kRounds; rd++) {
        for (uint32_t c = 0; c < n_chunks; c++) {
          const bool last = c + 1 == n_chunks;
          if (last) epi_bar();  // the previous round's bytes are out: the staging is free
          for (uint32_t ra = 0; ra < NA; ra++) {
            const uint32_t r = rd * NA + ra;
            if (ok && !mbar_wait(accf0 + 8 * ra, (par >> ra) & 1u)) ok = false;
            tc_fence_after();
            const uint32_t tb = tmem + ((quarter * 32u) << 16) + ra * TN + cbeg;
            if (ok && !idle) {
              const float pf = g.pf[r], invp = g.invp[r], pm = kMagic + pf;
#pragma unroll 1
              for (uint32_t col = 0; col < kHalf; col += kBatch) {
                uint32_t v[kBatch / 16][16];
#pragma unroll
                for (uint32_t b = 0; b < kBatch / 16; b++) tmem_ld16(tb + col + 16 * b, v[b]);
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                if (!last) {  // reduce in place; the next chunk accumulates on top
#pragma unroll
                  for (uint32_t b = 0; b < kBatch / 16; b++) {
#pragma unroll
                    for (int jj = 0; jj < 16; jj++)
                      v[b][jj] = __float_as_uint(reduce_p(__uint_as_float(v[b][jj]), pf, invp));
                    tmem_st16(tb + col + 16 * b, v[b]);
                  }
                } else if (g.direct) {  // r + 128, one byte per residue of the round in the staged entry
#pragma unroll
                  for (uint32_t b = 0; b < kBatch / 16; b++)
#pragma unroll
                    for (uint32_t jj = 0; jj < 16; jj++)
                      stage8[((cbeg + col + 16 * b + jj) * kStagePitch + row) * NA + ra] =
                          (uint8_t)offset_bits(reduce_p(__uint_as_float(v[b][jj]), pf, invp));
                } else {  // canonical residue, one byte per residue of the round in the staged entry
#pragma unroll
                  for (uint32_t b = 0; b < kBatch / 16; b++)
#pragma unroll
                    for (uint32_t jj = 0; jj < 16; jj++)
                      stage8[((cbeg + col + 16 * b + jj) * kStagePitch + row) * NA + ra] =
                          (uint8_t)canonical_bits(reduce_p(__uint_as_float(v[b][jj]), pf, invp), pm);
                }
              }
              if (!last) asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
            }
            tc_fence_before();
            // the accumulator is free (its values are in registers or staged);
            // PAIR: one arrival per warp of either CTA, on the leader's barrier
            if constexpr (PAIR) {
              __syncwarp();
              if (lane == 0) mbar_arrive_cluster(mapa_cluster(acce0 + 8 * ra, 0));
            } else {
              mbar_arrive(acce0 + 8 * ra);
            }
            par ^= 1u << ra;
          }
        }
        epi_bar();  // every residue of the round is staged
        const SW* sp = staging + lane_sid;
        if (ok && pv && g.direct) {
          // pairs of entries: one staging load, one half2 store per residue
          __half* planes = reinterpret_cast<__half*>(g.out) + ((uint64_t)(rd * NA) << (g.fa + g.fb)) + tile_base;
          for (uint32_t e0 = et; e0 < (kTileM * TN) / 2; e0 += 4 * kEpiThreads) {
            uint32_t adr[4], w0[4], w1[4];  // the pair's staged bytes: entry o in w0, o + 1 in w1 (NA = 4) or both in w0
#pragma unroll
            for (uint32_t u = 0; u < 4; u++) {
              const uint2 t = ho_tab[(e0 + u * kEpiThreads) >> 5];
              adr[u] = t.x;
              if constexpr (NA == 4) {
                w0[u] = reinterpret_cast<const uint32_t*>(sp)[t.y];
                w1[u] = reinterpret_cast<const uint32_t*>(sp)[t.y + 1];
              } else if constexpr (NA == 2) {
                w0[u] = *reinterpret_cast<const uint32_t*>(sp + t.y);
                w1[u] = w0[u];
              } else {
                w0[u] = *reinterpret_cast<const uint16_t*>(sp + t.y);
                w1[u] = w0[u];
              }
            }
#pragma unroll
            for (uint32_t ra = 0; ra < NA; ra++) {
              __half* pl = planes + ((uint64_t)ra << (g.fa + g.fb));
#pragma unroll
              for (uint32_t u = 0; u < 4; u++) {
                *reinterpret_cast<uint32_t*>(pl + adr[u]) = staged_half2<NA>(w0[u], w1[u], ra);
              }
            }
          }
        } else if (ok && g.direct) {
          // fp16 planes of the next dense step's operand (representatives of
          // magnitude at most (p+1)/2), the entries' own order: plane of
          // residue rd NA + ra at out + (rd NA + ra) 2^(fa+fb) halves
          __half* planes = reinterpret_cast<__half*>(g.out) + ((uint64_t)(rd * NA) << (g.fa + g.fb)) + tile_base;
          for (uint32_t e0 = et; e0 < kTileM * TN; e0 += 4 * kEpiThreads) {
            uint32_t adr[4];
            SW val[4];
#pragma unroll
            for (uint32_t u = 0; u < 4; u++) {
              const uint2 t = ho_tab[(e0 + u * kEpiThreads) >> 5];
              adr[u] = t.x;
              val[u] = sp[t.y];
            }
#pragma unroll
            for (uint32_t ra = 0; ra < NA; ra += 2) {  // two residues per half2
              __half* pl = planes + ((uint64_t)ra << (g.fa + g.fb));
#pragma unroll
              for (uint32_t u = 0; u < 4; u++) {
                const uint32_t h2 = staged_half2_res((uint32_t)val[u], ra);
                pl[adr[u]] = __ushort_as_half((unsigned short)(h2 & 0xFFFFu));
                if (ra + 1 < NA) pl[((uint64_t)1 << (g.fa + g.fb)) + adr[u]] = __ushort_as_half((unsigned short)(h2 >> 16));
              }
            }
          }
        } else if (ok) {
          uint8_t* outp = g.out + (g.log_split ? ((uint64_t)split << (g.fa + g.fb)) * RG : 0ull) + rd * NA +
                          tile_base * RG;
          // four entries (or pairs) per trip, their loads issued before their stores
          static_assert((kTileM * TN) % (4 * kEpiThreads) == 0, "whole trips of four");
          static_assert(TN < 32 || (kTileM * TN / 2) % (4 * kEpiThreads) == 0, "whole trips of four pairs");
          if (pv) {
            for (uint32_t e0 = et; e0 < (kTileM * TN) / 2; e0 += 4 * kEpiThreads) {
              uint8_t* adr[4];
              SW v0[4], v1[4];
#pragma unroll
              for (uint32_t u = 0; u < 4; u++) {
                const uint2 t = ho_tab[(e0 + u * kEpiThreads) >> 5];
                adr[u] = outp + (uint64_t)t.x * RG;
                v0[u] = sp[t.y];
                v1[u] = sp[t.y + 1];
              }
#pragma unroll
              for (uint32_t u = 0; u < 4; u++) {
                if constexpr (NA == RG) {  // the pair's entries are contiguous in C
                  if constexpr (NA == 4) {
                    *reinterpret_cast<uint2*>(adr[u]) = make_uint2(v0[u], v1[u]);
                  } else if constexpr (NA == 2) {
                    *reinterpret_cast<uint32_t*>(adr[u]) = (uint32_t)v0[u] | ((uint32_t)v1[u] << 16);
                  } else {
                    *reinterpret_cast<uint16_t*>(adr[u]) = (uint16_t)((uint32_t)v0[u] | ((uint32_t)v1[u] << 8));
                  }
                } else {
                  *reinterpret_cast<SW*>(adr[u]) = v0[u];
                  *reinterpret_cast<SW*>(adr[u] + RG) = v1[u];
                }
              }
            }
          } else
          for (uint32_t e0 = et; e0 < kTileM * TN; e0 += 4 * kEpiThreads) {
            uint8_t* adr[4];
            SW val[4];
#pragma unroll
            for (uint32_t u = 0; u < 4; u++) {
              const uint2 t = ho_tab[(e0 + u * kEpiThreads) >> 5];
              adr[u] = outp + (uint64_t)t.x * RG;
              val[u] = sp[t.y];
            }
#pragma unroll
            for (uint32_t u = 0; u < 4; u++) *reinterpret_cast<SW*>(adr[u]) = val[u];
          }
        }
      }
    }
    if (!ok) atomicExch(err, 1u);
  }
  tc_fence_before();
  __syncthreads();
  if constexpr (PAIR) cluster_sync();  // no copy, commit or arrival of the peer still targets this CTA
  tc_fence_after();
  if (warp == 1) tmem_dealloc<PAIR>(tmem, kCols);
}

}  // namespace tnc_p8

namespace tnc {

namespace {

using EncodeTiled = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                 const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// The driver's tensor-map encoder, fetched once through the runtime (no
// link-time dependency on the driver library).
EncodeTiled encoder() {
  static EncodeTiled fn = [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q{};
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      p = nullptr;
    return reinterpret_cast<EncodeTiled>(p);
  }();
  return fn;
}

// Tensor map of the packed operand planes (rg planes of rows x K fp16,
// row-major) with boxes of box_rows x 64 values (128-byte lines) of one plane,
// 128-byte swizzle.
int make_map(CUtensorMap* m, void* base, uint64_t rows, uint64_t K, uint32_t rg, uint32_t box_rows) {
  EncodeTiled fn = encoder();
  if (!fn) return set_error(TNC_ERR_CUDA, "cuTensorMapEncodeTiled is not available");
  const cuuint64_t dims[3] = {K, rows, rg};
  const cuuint64_t strides[2] = {K * 2, rows * K * 2};
  const cuuint32_t box[3] = {64, box_rows, 1};
  const cuuint32_t es[3] = {1, 1, 1};
  const CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 3, base, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                        CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return set_error(TNC_ERR_CUDA, "cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")");
  return TNC_OK;
}

// Row-contiguous planes (rg planes of K x rows fp16, a shared value's rows
// contiguous) with boxes of 64 rows x 64 shared values of one plane.
int make_map_mn(CUtensorMap* m, void* base, uint64_t rows, uint64_t K, uint32_t rg) {
  EncodeTiled fn = encoder();
  if (!fn) return set_error(TNC_ERR_CUDA, "cuTensorMapEncodeTiled is not available");
  const cuuint64_t dims[3] = {rows, K, rg};
  const cuuint64_t strides[2] = {rows * 2, rows * K * 2};
  const cuuint32_t box[3] = {64, 64, 1};
  const cuuint32_t es[3] = {1, 1, 1};
  const CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 3, base, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                        CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return set_error(TNC_ERR_CUDA, "cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")");
  return TNC_OK;
}

struct Shape {
  bool swap;                   // rows come from B
  bool pair;                   // 256-wide tiles on CTA pairs (an even number of row tiles)
  uint32_t fa, fb, k, kp, tn;  // row bits, column bits, shared bits (padded to >= 6), columns per tile
  uint64_t tiles;              // tiles of 128 rows x tn columns
};

constexpr uint64_t kP8WideTiles = 456;
constexpr uint64_t kP8Sms = 152;  // SMs of the GPU this path is laid out for

Shape shape_of(const StepDesc& d) {
  Shape s;
  s.swap = !(d.ka >= 7 && d.kb >= 4);
  s.fa = s.swap ? d.kb : d.ka;
  s.fb = s.swap ? d.ka : d.kb;
  s.k = d.k;
  s.kp = std::max<uint32_t>(d.k, 6);
  // 256 columns per tile (two residues at a time in TMEM, a quarter fewer
  // operand bytes per product than 128) where that still leaves at least three
  // tiles per SM; otherwise at most 128
  const uint64_t tiles_m = (1ull << s.fa) / tnc_p8::kTileM;
  s.tn = std::min<uint32_t>(1u << s.fb, 128);
  if (s.fb >= 8 && tiles_m * ((1ull << s.fb) / 256) >= kP8WideTiles) s.tn = 256;
  // long-K steps with fewer 256-wide tiles take CTA pairs too: their K split
  // (p8_split_log) supplies the work items
  if (s.fb >= 8 && tiles_m % 2 == 0 && s.k >= 11) s.tn = 256;
  // steps with less than a wave of tiles: narrower tiles (down to 32 columns)
  // while they stay within one wave, so that more SMs share the epilogue
  while (s.tn > 32 && s.tn < 256 && tiles_m * ((2ull << s.fb) / s.tn) <= kP8Sms) s.tn /= 2;
  s.tiles = tiles_m * ((1ull << s.fb) / s.tn);
  s.pair = s.tn == 256 && tiles_m % 2 == 0;
  return s;
}

// One CTA per SM for the g.n_items work items (at most `sms` CTAs); PAIR:
// clusters of two CTAs, as many as fit at once (at most one item each).
template <uint32_t TN, uint32_t RG, bool PAIR>
int launch_gemm(const CUtensorMap& ma, const CUtensorMap& mb, const tnc_p8::P8Args& g, int sms, uint32_t* err,
                cudaStream_t st) {
  auto kern = tnc_p8::p8_gemm_kernel<TN, RG, PAIR>;
  constexpr uint32_t smem = tnc_p8::Cfg<TN, RG, PAIR>::kSmemBytes;
  static int max_units = -1;  // CTAs (PAIR: clusters) resident at once
  if (max_units < 0) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return set_error(TNC_ERR_CUDA, std::string("p8 attribute: ") + cudaGetErrorString(e));
    int units = sms;
    if (PAIR) {
      cudaLaunchConfig_t cfg{};
      cudaLaunchAttribute at[1];
      at[0].id = cudaLaunchAttributeClusterDimension;
      at[0].val.clusterDim.x = 2;
      at[0].val.clusterDim.y = 1;
      at[0].val.clusterDim.z = 1;
      cfg.gridDim = dim3(2u * (unsigned)std::max(1, sms / 2));
      cfg.blockDim = dim3(tnc_p8::kThreads);
      cfg.dynamicSmemBytes = smem;
      cfg.attrs = at;
      cfg.numAttrs = 1;
      units = 0;
      e = cudaOccupancyMaxActiveClusters(&units, kern, &cfg);
      if (e != cudaSuccess)
        return set_error(TNC_ERR_CUDA, std::string("p8 cluster occupancy: ") + cudaGetErrorString(e));
      if (units <= 0) return set_error(TNC_ERR_CUDA, "no cluster of two CTAs fits the p8 GEMM");
    }
    max_units = units;
  }
  const unsigned units = (unsigned)std::min<uint64_t>(g.n_items, (uint64_t)std::min(max_units, sms));
  if (!PAIR) {
    kern<<<units, tnc_p8::kThreads, smem, st>>>(ma, mb, g, err);
    return TNC_OK;
  }
  cudaLaunchConfig_t cfg{};
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = 2;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.gridDim = dim3(2u * units);
  cfg.blockDim = dim3(tnc_p8::kThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  const cudaError_t e = cudaLaunchKernelEx(&cfg, kern, ma, mb, g, err);
  if (e != cudaSuccess) return set_error(TNC_ERR_CUDA, std::string("p8 cluster launch: ") + cudaGetErrorString(e));
  return TNC_OK;
}

template <uint32_t RG>
int launch_gemm_rg(uint32_t tn, bool pair, const CUtensorMap& ma, const CUtensorMap& mb, const tnc_p8::P8Args& g,
                   int sms, uint32_t* err, cudaStream_t st) {
  switch (tn) {
    case 16: return launch_gemm<16, RG, false>(ma, mb, g, sms, err, st);
    case 32: return launch_gemm<32, RG, false>(ma, mb, g, sms, err, st);
    case 64: return launch_gemm<64, RG, false>(ma, mb, g, sms, err, st);
    case 128: return launch_gemm<128, RG, false>(ma, mb, g, sms, err, st);
    default:
      return pair ? launch_gemm<256, RG, true>(ma, mb, g, sms, err, st)
                  : launch_gemm<256, RG, false>(ma, mb, g, sms, err, st);
  }
}

}  // namespace

bool p8_eligible(const StepDesc& d) {
  return d.k >= 4 && ((d.ka >= 7 && d.kb >= 4) || (d.kb >= 7 && d.ka >= 4));
}

// K split of a dense step: double it while the work items stay below
// kP8SplitTarget, each split keeps a whole chunk of 1024, and the partials
// (2^c entries per split, each of up to 4 residues) stay within 2^26 entries.
constexpr uint64_t kP8SplitTarget = 160;
// Raster groups of a dense step's tiles: as many row tiles as keep their
// operand rows (all residues of the pass) within 32 MiB, so that the CTAs of
// one wave re-read rows and columns that are still in L2 (32 and 64 MiB
// measured 2 % faster on C4 than all row tiles in one group, 8 MiB and
// 128 MiB no better).
constexpr uint64_t kP8GroupBytes = 32ull << 20;
// CTA-pair steps with fewer than three work items (pairs of tiles) per pair
// of SMs: the split whose waves of items take the least time (waves x K per
// item), the smallest within 5 % of it (fewer partial sums).
uint32_t p8_split_log(const StepDesc& d) {
  const Shape s = shape_of(d);
  uint32_t ls = 0;
  if (s.pair) {
    if (s.tiles >= kP8WideTiles) return 0;
    uint32_t max_ls = 0;
    while (s.k - max_ls - 1 >= 10 && (1ull << (d.c + max_ls + 1)) <= (1ull << 26)) max_ls++;
    double t[32], best = 1e300;
    for (uint32_t l = 0; l <= max_ls; l++) {
      const uint64_t items = (s.tiles / 2) << l, units = kP8Sms / 2;
      t[l] = (double)((items + units - 1) / units) / (double)(1u << l);
      best = std::min(best, t[l]);
    }
    while (t[ls] > 1.05 * best) ls++;
    return ls;
  }
  while ((s.tiles << ls) < kP8SplitTarget && s.k - ls - 1 >= 10 && (1ull << (d.c + ls + 1)) <= (1ull << 26)) ls++;
  return ls;
}

uint32_t p8_tile_width(const StepDesc& d) { return shape_of(d).tn; }

// Operand `side` (0: A, 1: B) of a dense step is read row-contiguous when it
// has at least 64 shared values and its tile side has at least 64 rows (the
// row tile always; the column tile when 64 or more wide).
bool p8_operand_mn(const StepDesc& d, int side) {
  const Shape s = shape_of(d);
  if (s.k < 6) return false;
  const bool row_side = (side == 1) == s.swap;
  return row_side || s.tn >= 64;
}

uint64_t p8_scratch_bytes(const StepDesc& d, int rg) {
  const uint32_t kp = std::max<uint32_t>(d.k, 6);
  return 2ull * (uint64_t)rg * ((1ull << (d.ka + kp)) + (1ull << (d.kb + kp)));
}

uint64_t p8_part_bytes(const StepDesc& d, int rg) {
  const uint32_t ls = p8_split_log(d);
  return ls ? (uint64_t)rg << (d.c + ls) : 0;
}

int p8_launch(const StepDesc& d, const uint32_t* primes, uint32_t rg, uint8_t* arena, uint64_t arena_bytes,
              uint32_t flags, void* scratch, uint8_t* part, uint32_t* dev_err, int sms, void* stream) {
  cudaStream_t st = (cudaStream_t)stream;
  if (rg != 1 && rg != 2 && rg != 4) return set_error(TNC_ERR_INVALID, "internal: residues per pass must be 1, 2 or 4");
  tnc_p8::PackPrimes pp{};
  for (uint32_t i = 0; i < 4; i++) pp.p[i] = primes[i < rg ? i : 0];
  for (uint32_t i = 0; i < rg; i++)
    if (primes[i] < 3 || primes[i] > 251) return set_error(TNC_ERR_INVALID, "tensor-core p8 steps need primes in [3, 251]");
  const Shape s = shape_of(d);
  const uint32_t ls = p8_split_log(d);
  const uint64_t a_elems = 1ull << (s.fa + s.kp);
  __half* a16 = (__half*)scratch;    // rg planes of a_elems
  __half* b16 = a16 + rg * a_elems;  // rg planes of b_elems
  const uint64_t a_off = s.swap ? d.b_off : d.a_off, b_off = s.swap ? d.a_off : d.b_off;
  // operands by tile side (row side = A unless swapped): read row-contiguous
  // (mn), and taken straight from the planes their producing dense step
  // wrote (direct), which occupy twice the entries' bytes
  const int side_a = s.swap ? 1 : 0, side_b = 1 - side_a;
  const bool mn_a = p8_operand_mn(d, side_a), mn_b = p8_operand_mn(d, side_b);
  const bool dir_a = (flags & (side_a ? kP8DirectB : kP8DirectA)) != 0;
  const bool dir_b = (flags & (side_b ? kP8DirectB : kP8DirectA)) != 0;
  const bool dir_out = (flags & kP8DirectOut) != 0;
  if ((dir_a && !mn_a) || (dir_b && !mn_b) || (dir_out && ls))
    return set_error(TNC_ERR_INVALID, "internal: direct fp16 planes for an operand read K-contiguous");
  {  // every range the launch touches lies inside the arena
    const uint64_t ea = (1ull << (s.fa + s.k)) * rg * (dir_a ? 2 : 1), eb = (1ull << (s.fb + s.k)) * rg * (dir_b ? 2 : 1);
    const uint64_t ec = (1ull << d.c) * rg * (dir_out ? 2 : 1);
    if (a_off * rg + ea > arena_bytes || b_off * rg + eb > arena_bytes || d.c_off * rg + ec > arena_bytes)
      return set_error(TNC_ERR_INVALID, "internal: dense step range outside the arena");
  }
  __half* pa = dir_a ? reinterpret_cast<__half*>(arena + a_off * rg) : a16;
  __half* pb = dir_b ? reinterpret_cast<__half*>(arena + b_off * rg) : b16;
  if (((uintptr_t)pa | (uintptr_t)pb) & 15u)
    return set_error(TNC_ERR_INVALID, "internal: fp16 operand planes not 16-byte aligned");
  if (!dir_a || !dir_b) {  // the operands still in entry form, packed by one launch
    const tnc_p8::PackOperand oa{arena + a_off * rg, a16, s.fa, dir_a ? 0u : (mn_a ? 2u : 1u)};
    const tnc_p8::PackOperand ob{arena + b_off * rg, b16, s.fb, dir_b ? 0u : (mn_b ? 2u : 1u)};
    const uint64_t n = ((dir_a ? 0 : (uint64_t)((1u << s.fa) + 63u) / 64u) +
                        (dir_b ? 0 : (uint64_t)((1u << s.fb) + 63u) / 64u))
                       << (s.kp - 6);
    const unsigned blocks = (unsigned)std::min<uint64_t>(n, (uint64_t)sms * 16);
    if (rg == 4) tnc_p8::p8_pack_kernel<4><<<blocks, 256, 0, st>>>(oa, ob, s.k, s.kp, pp);
    else if (rg == 2) tnc_p8::p8_pack_kernel<2><<<blocks, 256, 0, st>>>(oa, ob, s.k, s.kp, pp);
    else tnc_p8::p8_pack_kernel<1><<<blocks, 256, 0, st>>>(oa, ob, s.k, s.kp, pp);
    launch_counts().p8_pack++;
  }
  CUtensorMap ma, mb;
  int rc = mn_a ? make_map_mn(&ma, pa, 1ull << s.fa, 1ull << s.k, rg)
                : make_map(&ma, pa, 1ull << s.fa, 1ull << s.kp, rg, tnc_p8::kTileM);
  if (!rc)
    rc = mn_b ? make_map_mn(&mb, pb, 1ull << s.fb, 1ull << s.k, rg)
              : make_map(&mb, pb, 1ull << s.fb, 1ull << s.kp, rg, s.pair ? s.tn / 2 : s.tn);
  if (rc) return rc;
  tnc_p8::P8Args g;
  std::memset(&g, 0, sizeof(g));
  g.fa = s.fa;
  g.fb = s.fb;
  g.k = s.kp;  // zero-padded shared values contribute nothing
  g.log_split = ls;
  const uint32_t tile_rows = tnc_p8::kTileM * (s.pair ? 2u : 1u);  // rows per work item
  g.tiles_m = (1u << s.fa) / tile_rows;
  {  // raster groups of 2^gm_log row tiles
    uint32_t gm = 0;
    while ((2u << gm) <= g.tiles_m && (uint64_t)(2u << gm) * tile_rows * (2ull << s.kp) * rg <= kP8GroupBytes) gm++;
    g.gm_log = gm;
  }
  if ((s.tiles << ls) >= (1ull << 31)) return set_error(TNC_ERR_TOO_LARGE, "dense step has too many tiles");
  g.n_items = (uint32_t)((s.pair ? s.tiles / 2 : s.tiles) << ls);
  g.rg = rg;
  g.a_mn = mn_a ? 1u : 0u;
  g.b_mn = mn_b ? 1u : 0u;
  g.direct = dir_out ? 1u : 0u;
  for (uint32_t i = 0; i < 4; i++) {
    g.p[i] = pp.p[i];
    g.pf[i] = (float)pp.p[i];
    g.invp[i] = 1.0f / (float)pp.p[i];
  }
  // output address weights (the output bit j comes from one operand's free bit)
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
  const int row_op = s.swap ? 1 : 0;
  for (int j = 0; j < d.c; j++) {
    if (op[j] == row_op) g.wm[dst[j]] = 1ull << j;
    else g.wn[dst[j]] = 1ull << j;
  }
  // the tile's bits by output weight (ties cannot occur: distinct bits)
  {
    std::vector<std::pair<uint64_t, uint8_t>> bits;
    for (uint32_t j = 0; j < 7; j++) bits.push_back({g.wm[j], (uint8_t)j});
    for (uint32_t j = 0; (1u << j) < s.tn; j++) bits.push_back({g.wn[j], (uint8_t)(0x80u | j)});
    std::sort(bits.begin(), bits.end());
    g.n_ebits = (uint32_t)bits.size();
    for (size_t i = 0; i < bits.size(); i++) g.ebit[i] = bits[i].second;
  }
  g.pairs = (s.tn >= 32 && g.wm[0] == 1) ? 1u : 0u;  // output bit 0 is row bit 0
  g.out = ls ? part : arena + d.c_off * rg;  // direct: the planes, same place (twice the bytes)
  if (rg == 4) rc = launch_gemm_rg<4>(s.tn, s.pair, ma, mb, g, sms, dev_err, st);
  else if (rg == 2) rc = launch_gemm_rg<2>(s.tn, s.pair, ma, mb, g, sms, dev_err, st);
  else rc = launch_gemm_rg<1>(s.tn, s.pair, ma, mb, g, sms, dev_err, st);
  if (rc) return rc;
  {
    tnc_launch_counts& lc = launch_counts();
    lc.p8_gemm++;
    if (ls) lc.p8_split++;
    int w = 0;
    while ((16u << w) < s.tn) w++;
    lc.p8_tile_n[w]++;
    const int32_t chunks = (int32_t)std::max<uint64_t>(1, ((1ull << s.kp) >> ls) / tnc_p8::kChunkK);
    lc.p8_max_chunks = std::max(lc.p8_max_chunks, chunks);
    if (s.swap) lc.p8_swapped++;
    if (s.kp > s.k) lc.p8_padded++;
    if (dir_out) lc.p8_direct_out++;
    lc.p8_direct_in += (dir_a ? 1 : 0) + (dir_b ? 1 : 0);
    lc.p8_mn += (mn_a ? 1 : 0) + (mn_b ? 1 : 0);
    if (g.pairs) lc.p8_pairs++;
    if (s.pair) lc.p8_cta_pair++;
  }
  if (ls) {
    const uint64_t n = (uint64_t)rg << d.c;
    tnc_p8::p8_split_final_kernel<<<(unsigned)std::min<uint64_t>((n + 255) / 256, (uint64_t)sms * 8), 256, 0, st>>>(
        part, arena + d.c_off * rg, d.c, ls, rg, make_uint4(pp.p[0], pp.p[1], pp.p[2], pp.p[3]));
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return set_error(TNC_ERR_CUDA, std::string("p8 launch: ") + cudaGetErrorString(e));
  return TNC_OK;
}

}  // namespace tnc
