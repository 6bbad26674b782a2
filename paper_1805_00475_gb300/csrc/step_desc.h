// Device-visible descriptors of one pairwise contraction step and one leaf.
// Shared by the host lowering and the CUDA kernels of libtnc.
#pragma once

#include <cstdint>

// Maximum number of bit runs that map an output index to an operand address.
#define TNC_MAXRUN 8

// Output bits [src, src+len) of the step land on operand bits [dst, dst+len).
struct TncRun {
  uint8_t src, dst, len, pad;
};

// C[o] = sum_{q < 2^k} A[mapA(o) + (q << ka)] * B[mapB(o) + (q << kb)]  (mod p)
// for every output index o < 2^c.  All tensors of a plan have dimension 2 on
// every bond, so a permute of a tensor is a permutation of its index bits and
// the "reshape to a matrix over the shared bonds" of a step is exactly this
// pair of bit maps.  Offsets count entries; an entry holds one u32 residue per
// prime of the residue group, interleaved.
//
// mapA/mapB are given either as up to TNC_MAXRUN runs per operand
// (nra, nrb <= TNC_MAXRUN) or, when nra == TNC_BITMAP, bit by bit:
// bit[j] = (operand << 7) | destination bit, operand 0 = A, 1 = B.
#define TNC_BITMAP 0xFF

struct alignas(16) StepDesc {
  uint64_t a_off, b_off, c_off;
  uint32_t work_lo;  // level schedule: first work item of this step in its level
  uint8_t c, k, ka, kb;
  uint8_t nra, nrb, a_rank, b_rank;
  union {
    struct {
      TncRun ra[TNC_MAXRUN];
      TncRun rb[TNC_MAXRUN];
    } runs;
    uint8_t bit[64];
  } map;
};

// Leaf tensor to materialise: COPY (kind 4) or one of the clause kinds 0..3.
struct alignas(16) LeafDesc {
  uint64_t off;        // arena entry offset
  uint32_t table_off;  // TABLE: offset of its 2^rank weights (already in layout order)
  uint8_t kind, rank, pad0, pad1;
};
