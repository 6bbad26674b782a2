// Internal host-side structures of libtnc (not part of the C ABI).
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "tnc.h"
#include "step_desc.h"

namespace tnc {

// Leaf tensor kinds: the four clause kinds of tnc.h plus the variable COPY.
enum LeafKind : uint8_t { LK_1IN3 = 0, LK_OR = 1, LK_NAND = 2, LK_TABLE = 3, LK_COPY = 4 };

struct Leaf {
  uint8_t kind = LK_COPY;
  std::vector<int> bonds;       // bond ids; bit j of an entry index = value on bonds[j]
  std::vector<uint32_t> table;  // TABLE only: 2^rank weights in `bonds` order
  int rank() const { return (int)bonds.size(); }
};

// A formula's tensor network (Sec. 2.1): clause c -> leaf c, variable v ->
// leaf n_cons + v.  Bond b joins leaves bond_end[b][0] and bond_end[b][1]
// (-1 for the free end of an open bond).
struct Network {
  int n_vars = 0, n_cons = 0;
  std::vector<int> open_vars;
  std::vector<Leaf> leaves;
  int n_bonds = 0;
  std::vector<int> bond_end0, bond_end1;
  int first_open_bond = 0;  // open bond of open_vars[i] = first_open_bond + i
  int n_components = 0;
  double log2_bound = 0.0;  // certified log2 upper bound on any count entry
  int n_leaves() const { return (int)leaves.size(); }
};

// Binary contraction tree.  Leaves 0..L-1, internal nodes L..2L-2 created in
// an order where children precede parents (so ascending id = a valid
// execution order).
struct Node {
  int left = -1, right = -1;
  std::vector<int> bonds;  // sorted bond ids of this tensor
};

struct Tree {
  std::vector<Node> nodes;
  int n_leaves = 0;
  int root = -1;
};

struct TreeCost {
  int max_rank = 0;
  int depth = 0;
  double macs = 0.0;
  double entries = 0.0;
};

// A lowered plan.
struct Lowered {
  std::vector<std::vector<int>> layout;  // node -> bond ids in bit order
  // sequential (one launch per step) schedule
  std::vector<StepDesc> seq_steps;  // internal nodes ascending
  std::vector<uint64_t> seq_leaf_off;
  uint64_t seq_arena_entries = 0;
  uint64_t seq_root_off = 0;
  // level-synchronous schedule (persistent batch kernel)
  std::vector<StepDesc> lvl_steps;  // sorted by level, work_lo filled
  std::vector<uint32_t> lvl_start;  // n_levels + 1
  std::vector<uint64_t> lvl_leaf_off;
  uint64_t lvl_arena_entries = 0;
  uint64_t lvl_root_off = 0;
  std::vector<int32_t> lvl_src_a, lvl_src_b;  // producing step of each operand (-1: a leaf)
  std::vector<int32_t> lvl_dst;               // consuming step of each output (-1: the root)
  // the level schedule as TNC_PATH_TC_P8 runs it: a dense step's output that
  // the consuming dense step reads row-contiguous is written as fp16 planes
  // (p8_direct), twice the entries, so the arena is laid out again
  std::vector<uint8_t> p8_direct;
  std::vector<StepDesc> p8_steps;  // lvl_steps with the offsets of this layout
  std::vector<uint64_t> p8_leaf_off;
  uint64_t p8_arena_entries = 0;
  uint64_t p8_root_off = 0;
  // leaves
  std::vector<LeafDesc> leaves;          // offsets filled per schedule at pack time
  std::vector<uint32_t> leaf_tables;     // TABLE entries permuted to leaf layouts
  std::vector<uint8_t> root_perm;        // root bit j -> open variable index
  int max_runs = 0;
  int n_bitmap_steps = 0;
  bool lvl_fits = false;  // level schedule validated (work offsets fit 32 bits)
};

}  // namespace tnc

struct tnc_network_s {
  tnc::Network net;
};

struct tnc_plan_s {
  tnc::Network net;  // own copy: a plan outlives its network handle
  tnc::Tree tree;
  tnc::TreeCost cost;
  tnc::Lowered low;
  tnc_plan_stats stats{};
};

namespace tnc {

// thread-local error reporting
int set_error(int code, const std::string& msg);
void clear_error();

// Kernel launches of the calling thread's current (or last) contraction
// (tnc_last_launch_counts); contract.cu resets it per call.
tnc_launch_counts& launch_counts();

// Fault injection (inject.cpp): true if an armed failure of this kind fires
// at this call site (tnc_inject_failure).
bool inject_hit(int kind);

// network.cpp
int build_network(const tnc_formula* f, Network& out);

// planner.cpp
int plan_tree(const Network& net, const tnc_plan_opts& opts, Tree& out);
TreeCost tree_cost(const Tree& t);
void tree_from_merges(const Network& net, const std::vector<std::pair<int, int>>& merges, Tree& t);
int plan_greedy(const Network& net, Tree& t);
int plan_bisect(const Network& net, int tries, uint64_t seed, Tree& t);
int plan_gn(const Network& net, Tree& t);

// learned.cpp: TNC_PLAN_COARSEN (tensor-greedy coarsening finished by
// TNC_PLAN_BEST; fewest MACs within the rank cap)
int plan_coarsen(const Network& net, const tnc_plan_opts& opts, Tree& out);

// lower.cpp
int lower_plan(const Network& net, const Tree& tree, Lowered& low);
int validate_lowered(const Network& net, const Tree& tree, Lowered& low);

// primes.cpp
// Default primes: the largest below 2^30, so that 16 residue products fit a
// 64-bit accumulator between reductions (4 for primes near 2^31).
constexpr uint32_t kDefaultPrimeBound = 1u << 30;
std::vector<uint32_t> default_primes(int n);
// Largest prime of the TNC_PATH_TC_P8 arithmetic, and its default primes.
constexpr uint32_t kP8PrimeMax = 251;
constexpr int kP8MaxResidues = 53;  // odd primes in [3, 251]
std::vector<uint32_t> default_primes_p8(int n);
bool is_prime_u32(uint32_t n);

// tc.cu: dense steps on the tensor cores (exact 8-bit-limb GEMMs)
bool tc_eligible(const StepDesc& d);
// TNC_PATH_TC_P8 dense steps (tc_p8.cu).
bool p8_eligible(const StepDesc& d);
uint32_t p8_split_log(const StepDesc& d);
uint32_t p8_tile_width(const StepDesc& d);
uint64_t p8_scratch_bytes(const StepDesc& d, int rg);
uint64_t p8_part_bytes(const StepDesc& d, int rg);
// Operand `side` (0: A, 1: B) of a dense step read row-contiguous (MN-major).
bool p8_operand_mn(const StepDesc& d, int side);
// Direct fp16 planes: the step's output goes straight to the planes of the
// consuming dense step's operand (kP8DirectOut), and operand A / B is read
// from planes its producer wrote (kP8DirectA / kP8DirectB); such a tensor
// takes twice its entries' bytes in the arena.
constexpr uint32_t kP8DirectOut = 1, kP8DirectA = 2, kP8DirectB = 4;
// One dense step for all rg residues (primes[0..rg)) of a pass whose entries
// hold rg residues of one byte each: the operands not already in fp16 planes
// packed by one launch, then one GEMM launch that computes every residue of
// each output tile and writes whole entries (or planes).  arena_bytes bounds
// every range the step touches (checked before any launch).
int p8_launch(const StepDesc& d, const uint32_t* primes, uint32_t rg, uint8_t* arena, uint64_t arena_bytes,
              uint32_t flags, void* scratch, uint8_t* part, uint32_t* dev_err, int sms, void* stream);
size_t tc_step_bytes();
void tc_make_step(const StepDesc& d, uint32_t p, void* out);
uint32_t tc_split_log(const StepDesc& d);
uint64_t tc_part_entries();
int tc_launch(const void* dev_step, const StepDesc& d, uint32_t* arena, uint32_t* part, uint32_t* dev_err,
              void* stream);

}  // namespace tnc
