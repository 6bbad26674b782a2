/*
 * tnc.h -- C ABI of libtnc: exact model counting by tensor-network contraction
 * on one GB300 GPU (sm_103a).
 *
 * Method: Kourtis, Chamon, Mucciolo, Ruckenstein, "Fast counting with tensor
 * networks".  A #CSP formula becomes a network with one COPY tensor per
 * variable (Eq. var) and one clause tensor per clause (Eq. or, Eq. 1in3, ...),
 * every occurrence of a variable in a clause being one bond of dimension 2
 * (Sec. 2.1).  Its full contraction (Eq. z at beta -> infinity) is the number
 * of satisfying assignments.  The contraction is a sequence of pairwise steps,
 * each merging two tensors over all the bonds they share (edge contraction of
 * Sec. 2.2), along an order from the paper's graph heuristics (tensor-greedy,
 * tensor-METIS-style recursive bisection, tensor-GN; Sec. 3.1.1).
 *
 * Exactness: counts exceed 2^64, so every tensor entry is kept as residues
 * modulo R primes below 2^31 and the final count is rebuilt as a big integer
 * by the Chinese remainder theorem (Garner's mixed radix).  The paper counts
 * in floating point and notes its rounding errors from about 100 vertices
 * (Sec. 3.2); this library is exact whenever the count is below the product
 * of the primes, and flags results for which it cannot certify that.
 *
 * Conventions for every entry point:
 *   - return 0 (TNC_OK) on success, a negative TNC_ERR_* code otherwise;
 *     tnc_last_error() then describes the failure (thread-local string);
 *   - no C++ exception crosses this boundary;
 *   - pointers documented "host" must be host memory, "device" device memory
 *     of the current CUDA device; sizes are in bytes unless stated;
 *   - objects returned through `T** out` are owned by the library and freed
 *     with the matching tnc_free_* call; all caller buffers stay owned by the
 *     caller and are not retained after the call returns (except where a
 *     batch documents otherwise);
 *   - `cuda_stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Device work is enqueued on it.
 */
#ifndef TNC_H
#define TNC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- error codes ---------------------------------------------------------- */
#define TNC_OK 0
#define TNC_ERR_INVALID (-1)   /* malformed argument or formula */
#define TNC_ERR_TOO_LARGE (-2) /* rank cap or memory bound exceeded (found at plan time) */
#define TNC_ERR_CUDA (-3)      /* a CUDA call failed; see tnc_last_error() */
#define TNC_ERR_BUFFER (-4)    /* caller buffer too small; needed size reported */
#define TNC_ERR_TIMEOUT (-5)   /* a bounded device-side wait gave up */
#define TNC_ERR_NOMEM (-6)     /* host allocation failed */

/* ---- clause kinds (clause tensor definitions, Sec. 2.1 and Sec. 3.2) ----- */
#define TNC_1IN3 0  /* 1 iff exactly one index is 1 (Eq. 1in3; any arity)       */
#define TNC_OR 1    /* 0 iff all indices are 0 (Eq. or)                          */
#define TNC_NAND 2  /* 0 iff all indices are 1 (independent-set edge)           */
#define TNC_TABLE 3 /* explicit 2^arity non-negative weights, index bit j =
                       value of the clause's j-th variable                       */

/* ---- planners (Sec. 3.1.1) ----------------------------------------------- */
#define TNC_PLAN_GREEDY 0   /* tensor-greedy: smallest result rank first          */
#define TNC_PLAN_BISECT 1   /* tensor-METIS reading: recursive min-cut bisection,
                               best of `tries` per split                          */
#define TNC_PLAN_GN 2       /* tensor-GN: Girvan-Newman community dendrogram      */
#define TNC_PLAN_EXPLICIT 3 /* caller-given pairwise order                        */
#define TNC_PLAN_BEST 4     /* run GREEDY, BISECT and GN; keep the cheapest       */
#define TNC_PLAN_PORTFOLIO 5 /* GREEDY, GN and BISECT with 8 seeds; the cheapest   */
#define TNC_PLAN_COARSEN 6  /* two levels: tensor-greedy merges coarsen the network,
                               BEST finishes it at 10, 20, .., 80 % of the merges;
                               with GREEDY, BISECT and GN on the whole network, the
                               plan with the fewest MACs within rank_cap is kept   */

/* ---- arithmetic paths ---------------------------------------------------- */
#define TNC_PATH_INT64 0 /* CUDA cores: u32 residues, 64-bit multiply-accumulate */
#define TNC_PATH_TC 1    /* dense steps (k >= 6 shared bonds, one side >= 2^7 and the
                            other >= 2^5 free entries) as exact 8-bit-limb GEMMs on the
                            tcgen05 tensor cores (fp16 limbs, fp32 accumulation below
                            2^24, K chunks of 64); other steps as TNC_PATH_INT64; one
                            pass per residue.  tnc_contract only. */
#define TNC_PATH_TC_P8 2 /* residues modulo primes p <= 251 (Sec. 3.2's exact counts
                            from more, smaller residues): each residue is one 8-bit
                            limb, taken balanced (|r| <= 125) and exact in fp16.
                            Tensors hold one byte per residue, passes of up to 4
                            residues.  Dense steps (k >= 4, one side >= 2^7 and the
                            other >= 2^4 free entries) run as fp16 GEMMs on tcgen05,
                            operand tiles by TMA, fp32 accumulation in TMEM reduced
                            mod p in place every 1024 shared values (1024 * 125^2 +
                            125 < 2^24: exact); other steps on CUDA cores with 32-bit
                            multiply-accumulate.  Workspace: tnc_workspace_bytes_opts.
                            tnc_contract only. */

/* ---- result flags -------------------------------------------------------- */
#define TNC_MAYBE_WRAPPED 1u /* the certified bound on the count is not below the
                                product of the primes: the CRT value may be the
                                count reduced modulo that product               */

typedef struct tnc_network_s tnc_network_t;
typedef struct tnc_plan_s tnc_plan_t;
typedef struct tnc_batch_s tnc_batch_t;

/* A formula.  All arrays are host memory owned by the caller and copied in.
 *   var_of   : concatenation of each clause's variable list (sum of arity);
 *              variables within one clause must be distinct;
 *   kind     : one TNC_* clause kind per clause;
 *   table    : for TABLE clauses only, 2^arity weights each, concatenated in
 *              clause order (may be NULL when no clause is TABLE);
 *   open_vars: variables whose COPY tensor keeps one extra, uncontracted bond;
 *              the result is then a tensor of 2^n_open counts, entry index bit
 *              i = value of open_vars[i] (the open network of the worked
 *              example, Sec. 2.1).  n_open <= 20. */
typedef struct {
  int32_t n_vars;
  int32_t n_cons;
  const int32_t* arity;
  const int32_t* var_of;
  const uint8_t* kind;
  const uint32_t* table;
  int32_t n_open;
  const int32_t* open_vars;
} tnc_formula;

typedef struct {
  int32_t heuristic;     /* TNC_PLAN_*                                              */
  int32_t rank_cap;      /* refuse plans whose largest tensor has a higher rank
                            (<= 0: default 32)                                      */
  int32_t tries;         /* bisections per split, best kept (<= 0: 2, Sec. 3.1.1)   */
  uint64_t seed;         /* seed of the randomised planners                         */
  const int32_t* order;  /* EXPLICIT: n_order pairs (a, b) of live tensor ids; ids:
                            clause c -> c, variable v -> n_cons + v, result of the
                            i-th pair -> n_cons + n_vars + i.  Tensors left over
                            are finished by tensor-greedy.                          */
  int32_t n_order;
} tnc_plan_opts;

/* Exact cost of a plan, predicted before any tensor is touched (the "lazy"
 * evaluation of Sec. 4).  MACs count one multiply-accumulate per residue-free
 * scalar: sum over steps of 2^(a+b-k) for ranks a, b sharing k bonds. */
typedef struct {
  int32_t max_rank;       /* largest tensor rank along the plan                   */
  int32_t n_steps;        /* pairwise contractions                                */
  int32_t n_leaves;       /* tensors of the network                               */
  int32_t depth;          /* longest root-to-leaf path of the contraction tree    */
  double total_macs;      /* sum of 2^(a+b-k)                                     */
  double total_entries;   /* sum of 2^a + 2^b + 2^(a+b-2k): entries moved          */
  double log2_bound;      /* log2 of the certified upper bound on every count      */
  uint64_t arena_entries; /* peak live entries, one launch per step (x residues per
                             pass x 4 bytes, 1 byte on TNC_PATH_TC_P8 = the tensor
                             arena of tnc_contract)                                */
  uint64_t batch_arena_entries; /* same for the level-by-level batch schedule     */
  int32_t n_dense_steps;  /* steps TNC_PATH_TC runs on the tensor cores            */
  double dense_macs;      /* their share of total_macs                             */
  int32_t n_dense_steps_p8; /* steps TNC_PATH_TC_P8 runs on the tensor cores       */
  double dense_macs_p8;     /* their share of total_macs                           */
  int32_t n_direct_p8;      /* of those, steps whose output goes straight to the fp16
                               operand planes of the next dense step (no packing)  */
  uint64_t p8_arena_entries; /* arena of TNC_PATH_TC_P8 (such outputs take twice
                               their entries)                                      */
} tnc_plan_stats;

typedef struct {
  int32_t path;          /* TNC_PATH_*                                           */
  int32_t n_residues;    /* R, 1..16 (TNC_PATH_TC_P8: 1..53)                     */
  const uint32_t* primes;/* host, R distinct primes in (2^29, 2^31); NULL = the R
                            largest primes below 2^30 (16 residue products fit a
                            64-bit accumulator between reductions; 4 near 2^31).
                            TNC_PATH_TC_P8: R distinct primes in [3, 251]; NULL =
                            the R largest (tnc_default_primes_p8)                */
} tnc_contract_opts;

/* One formula's result.  Caller-allocated host buffers.
 *   residues : [n_out][R]   count mod primes[r];
 *   limbs    : [n_out][cap_limbs] little-endian u32 limbs of the CRT value;
 *   n_out    : out, 2^n_open;
 *   n_limbs  : out, limbs needed per entry (if > cap_limbs: TNC_ERR_BUFFER and
 *              nothing written to limbs);
 *   flags    : out, TNC_MAYBE_WRAPPED or 0. */
typedef struct {
  uint32_t* residues;
  uint32_t* limbs;
  int32_t cap_out;
  int32_t cap_limbs;
  int32_t n_out;
  int32_t n_limbs;
  uint32_t flags;
} tnc_count;

/* ---- library ------------------------------------------------------------- */
const char* tnc_version(void);
/* Last error message of the calling thread ("" if none). */
const char* tnc_last_error(void);
/* The default primes: the n largest below 2^30, descending (deterministic
 * Miller-Rabin). */
int tnc_default_primes(int32_t n, uint32_t* out /* host, n */);
/* The default primes of TNC_PATH_TC_P8: the n (<= 53) largest primes <= 251,
 * descending. */
int tnc_default_primes_p8(int32_t n, uint32_t* out /* host, n */);

/* ---- network (Sec. 2.1): formula -> COPY + clause tensors, bonds --------- */
int tnc_build_network(const tnc_formula* f, tnc_network_t** out);
/* Counts of the network: tensors, bonds (incl. open), connected components. */
int tnc_network_info(const tnc_network_t* net, int32_t* n_tensors, int32_t* n_bonds,
                     int32_t* n_components);
void tnc_free_network(tnc_network_t* net);

/* ---- planning (Sec. 2.2, Sec. 3.1.1, Sec. 4) ----------------------------- */
/* Builds the contraction tree and lowers it (layouts, arena offsets).
 * stats may be NULL.  TNC_ERR_TOO_LARGE if max_rank > rank_cap. */
int tnc_plan(const tnc_network_t* net, const tnc_plan_opts* opts, tnc_plan_t** out,
             tnc_plan_stats* stats);
/* Plans n networks in parallel on the host cores (OpenMP).  out[i] and, if
 * stats is not NULL, stats[i] receive formula i's plan.  All or nothing: on
 * any failure every out[i] is NULL and the first failing formula is named in
 * tnc_last_error(). */
int tnc_plan_many(const tnc_network_t* const* nets, int32_t n, const tnc_plan_opts* opts,
                  tnc_plan_t** out, tnc_plan_stats* stats);
/* Bond slicing (memory is the method's bottleneck, Sec. 4): chooses s
 * variables of the network (not open ones) and plans the 2^s slices, the
 * networks with those variables fixed (Eq. z's trace split by their values;
 * the fixed COPY tensors leave, the clause tensors on their bonds become
 * tables over their other bonds).  Variables are added one at a time: each
 * round scores the variables on the tensors of largest rank of the current
 * plan by the exact cost of their slices (max rank, then total MACs; the
 * lazy evaluation of Sec. 4), each planned by `opts` and by the current plan
 * restricted to the slice, the cheaper kept (so the max rank never grows with
 * s).  Slice j fixes vars_out[i] = bit i of j; all slices share one tree.
 *   out: host array of 2^s plan handles (freed with tnc_free_plan);
 *   vars_out: s variables; stats: 2^s entries or NULL.
 * All or nothing on failure.  The count is the sum of the slices' counts
 * (tnc_contract_sliced). */
int tnc_plan_sliced(const tnc_network_t* net, int32_t s, const tnc_plan_opts* opts, tnc_plan_t** out,
                    int32_t* vars_out, tnc_plan_stats* stats);
/* The network of one slice: variables vars[i] fixed to bit i of `bits` (the
 * restriction tnc_plan_sliced applies; for inspection and for callers that
 * plan slices themselves).  Fixed variables leave and the others are
 * renumbered in order.  Open variables cannot be fixed (TNC_ERR_INVALID). */
int tnc_slice_network(const tnc_network_t* net, int32_t s, const int32_t* vars, uint32_t bits,
                      tnc_network_t** out);
/* The formula a network encodes (clause kinds as built: a clause restricted
 * by slicing is a TABLE).  Call once with the array pointers NULL for the
 * sizes (clauses, occurrences = sum of arities, table entries, open
 * variables), then with arrays of those sizes. */
int tnc_network_formula(const tnc_network_t* net, int32_t* n_vars, int32_t* n_cons, int32_t* n_occ,
                        int32_t* n_table, int32_t* n_open, int32_t* arity, int32_t* var_of, uint8_t* kind,
                        uint32_t* table, int32_t* open_vars);
/* Contraction tree as pairs: for step i, the tensor ids it merges (ids as in
 * tnc_plan_opts.order).  left/right: host arrays of n_steps entries. */
int tnc_plan_steps(const tnc_plan_t* plan, int32_t* left, int32_t* right, int32_t cap);
void tnc_free_plan(tnc_plan_t* plan);

/* ---- single formula (Sec. 2.1 contraction; one launch per step) --------- */
/* Device workspace needed by tnc_contract for R residues on TNC_PATH_INT64 or
 * TNC_PATH_TC. */
size_t tnc_workspace_bytes(const tnc_plan_t* plan, int32_t n_residues);
/* Device workspace needed by tnc_contract with these options (any path; adds
 * TNC_PATH_TC_P8's packed fp16 operands and K-split partials); 0 if the options
 * are invalid. */
size_t tnc_workspace_bytes_opts(const tnc_plan_t* plan, const tnc_contract_opts* opts);
/* Sliced contraction (bond slicing: fixing s variables of a formula splits its
 * count into 2^s counts of smaller networks, each with at most the original
 * ranks; the paper leaves memory as the bottleneck of its method, Sec. 4).
 * plans[i] are the networks of the slices (same open variables); the result
 * is the sum of their counts, exact: each slice's residues are added on the
 * device modulo the primes, then one CRT.  As many slices at a time as the
 * workspace holds beyond tnc_workspace_bytes_sliced's minimum run with their
 * tree levels merged (as tnc_contract_many).  `flags` certifies the sum (the sum
 * of the slices' bounds).  dev_ws: tnc_workspace_bytes_sliced bytes, 256-byte
 * aligned.  Synchronises `cuda_stream`. */
size_t tnc_workspace_bytes_sliced(const tnc_plan_t* const* plans, int32_t n, const tnc_contract_opts* opts);
int tnc_contract_sliced(const tnc_plan_t* const* plans, int32_t n, const tnc_contract_opts* opts, void* dev_ws,
                        size_t ws_bytes, void* cuda_stream, tnc_count* out);
/* Many formulas in one call: independent contractions (Sec. 2.1) whose tree
 * levels are merged, so that one launch covers the small steps of level l of
 * every formula of a group, and the group's big, split-K and dense steps
 * follow one another on the stream.  A group is as many consecutive plans as
 * the workspace holds (each plan alone must fit: TNC_ERR_BUFFER otherwise).
 * Any path; outs: n counts, as tnc_contract would give them one by one.
 * tnc_workspace_bytes_many gives the bytes that hold groups of `group`
 * consecutive plans (group = 1: the least that works).  dev_ws 256-byte
 * aligned; synchronises `cuda_stream`. */
size_t tnc_workspace_bytes_many(const tnc_plan_t* const* plans, int32_t n, const tnc_contract_opts* opts,
                                int32_t group);
int tnc_contract_many(const tnc_plan_t* const* plans, int32_t n, const tnc_contract_opts* opts, void* dev_ws,
                      size_t ws_bytes, void* cuda_stream, tnc_count* outs);
/* Measurement aid (calling thread only; off by default): with on != 0, every
 * later tnc_contract brackets each dense (tensor-core) step with CUDA events
 * on its stream, and tnc_last_dense_time returns the summed device time (ms)
 * and the number of dense step launches of the last tnc_contract. */
void tnc_set_step_timing(int32_t on);
int tnc_last_dense_time(double* ms, int32_t* n_steps);
/* Same mode, step by step: the device time of every dense step launch of the
 * last contraction (operand packing + GEMM + split sum, in launch order) and
 * its shape, for per-step roofline fractions (flops = 2 * macs * residues). */
typedef struct {
  double ms;         /* CUDA-event time of the launch                           */
  double macs;       /* 2^(a+b-k): multiply-accumulates per residue              */
  int32_t rows_log2; /* free bits of the two operands (before any exchange)      */
  int32_t cols_log2;
  int32_t k_log2;    /* shared bonds                                              */
  int32_t residues;  /* residues computed by the launch                           */
  int32_t tile_n;    /* columns per tile                                          */
  int32_t log_split; /* K split                                                   */
} tnc_dense_step_time;
int tnc_last_dense_steps(tnc_dense_step_time* out, int32_t cap, int32_t* n);
/* Same mode: device time (ms) of the last tnc_contract's kernels, from its
 * first launch to its CRT (host work and the final copies excluded). */
int tnc_last_contract_time(double* device_ms);
/* The device kernels the calling thread's last tnc_contract,
 * tnc_contract_sliced or tnc_contract_noalloc enqueued, by kind: a record of
 * which branches of the pairwise step (Sec. 2.1) actually ran.  Always
 * recorded (host counters, no device work); a sliced call sums its slices. */
typedef struct {
  int32_t leaf_fill;      /* leaf tensors (Eq. var, Eq. or, Eq. 1in3, ...)           */
  int32_t level;          /* one launch for all small steps of a tree level           */
  int32_t grid_step;      /* one large step over the whole GPU                       */
  int32_t splitk;         /* split-K steps on CUDA cores (a partial + final pair)    */
  int32_t tc_gemm;        /* TNC_PATH_TC dense steps (tcgen05 limb GEMM launches)     */
  int32_t tc_split;       /*   of which split over K (partials summed after)          */
  int32_t p8_pack;        /* TNC_PATH_TC_P8 operand packing launches                  */
  int32_t p8_gemm;        /* TNC_PATH_TC_P8 dense steps (tcgen05 GEMM launches)       */
  int32_t p8_split;       /*   of which split over K                                 */
  int32_t p8_tile_n[5];   /*   by tile width: 16, 32, 64, 128, 256 columns            */
  int32_t p8_max_chunks;  /* most 1024-value chunks one tile accumulates in TMEM per
                             residue (each reduced mod p in place before the next)   */
  int32_t p8_swapped;     /*   with the row operand taken from B (A too narrow)       */
  int32_t p8_padded;      /*   with fewer than 64 shared values, zero-padded to 64     */
  int32_t extract;        /* root tensor -> result residues                          */
  int32_t crt;            /* Chinese remaindering                                     */
  int32_t p8_direct_out;  /* TNC_PATH_TC_P8 dense steps whose output went straight to
                             the fp16 planes the consuming dense step reads           */
  int32_t p8_direct_in;   /* dense-step operands read from such planes (not packed)   */
  int32_t p8_mn;          /* dense-step operands read row-contiguous (MN-major)       */
  int32_t p8_pairs;       /* dense steps whose epilogue writes two entries at a time
                             (output bit 0 is row bit 0)                              */
  int32_t outer;          /* big steps with one small operand (at most 16 free rows,
                             8 shared values), staged in shared memory               */
  int32_t p8_cta_pair;    /* TNC_PATH_TC_P8 dense steps on CTA pairs: 256 x 256 tiles,
                             one cta_group::2 MMA over two SMs' shared memory         */
} tnc_launch_counts;
int tnc_last_launch_counts(tnc_launch_counts* out);
/* Bytes the calling thread's last tnc_contract or tnc_contract_sliced copied
 * host -> device (descriptors, weight tables) and device -> host (residues,
 * CRT limbs, status word). */
int tnc_last_io_bytes(uint64_t* h2d_bytes, uint64_t* d2h_bytes);
/* Contracts the plan on the GPU and returns the count(s) in `out` (host).
 * dev_ws: device buffer of at least tnc_workspace_bytes_opts(plan, opts) bytes
 * (= tnc_workspace_bytes(plan, R) on TNC_PATH_INT64 and TNC_PATH_TC), 256-byte
 * aligned, owned by the caller, free for the library's use during the call.
 * Synchronises `cuda_stream` before returning. */
int tnc_contract(const tnc_plan_t* plan, const tnc_contract_opts* opts, void* dev_ws,
                 size_t ws_bytes, void* cuda_stream, tnc_count* out);

/* ---- host combine of residues from several processes ---------------------
 * A count can be shared out over processes (one GPU each) without any device
 * collective: each process counts modulo its own subset of the primes (the
 * residues are independent), or contracts its own subset of the slices of a
 * sliced network; the small residue arrays are gathered to one host, which
 * adds the slices' residues and rebuilds the exact count (Sec. 3.2: exact
 * counts need more than machine words; the paper leaves distributed
 * contraction as a prospect, Sec. 4).  Host memory only, no device work. */
/* Garner's mixed-radix CRT: residues [n][R] (entry e's residue mod primes[r]
 * at e R + r) -> little-endian u32 limbs [n][cap_limbs] of the value in
 * [0, prod p).  *n_limbs (may be NULL) receives the limbs needed;
 * TNC_ERR_BUFFER if cap_limbs is smaller.  Primes: distinct odd primes below
 * 2^31, any order. */
int tnc_crt_host(const uint32_t* primes, int32_t R, const uint32_t* residues, int64_t n, uint32_t* limbs,
                 int32_t cap_limbs, int32_t* n_limbs);
/* acc[e R + r] = (acc[e R + r] + src[e R + r]) mod primes[r] for n entries
 * (the sum of slices' counts, residue by residue). */
int tnc_residue_add_host(const uint32_t* primes, int32_t R, uint32_t* acc, const uint32_t* src, int64_t n);

/* ---- batches: many formulas in one persistent launch -------------------- */
/* Packs the plans into compact descriptors in pinned host memory and picks a
 * default launch shape for the current device.  The plans must outlive the
 * batch.  Batch formulas need plan rank <= 24 (TNC_ERR_TOO_LARGE otherwise). */
int tnc_batch_create(const tnc_plan_t* const* plans, int32_t n, const tnc_contract_opts* opts,
                     tnc_batch_t** out);
size_t tnc_batch_workspace_bytes(const tnc_batch_t* b);
/* Sizes of a batch: bytes uploaded by tnc_batch_upload (h2d), bytes read back
 * by tnc_batch_download (d2h), result entries, device kernels per launch.
 * Any pointer may be NULL. */
int tnc_batch_info(const tnc_batch_t* b, size_t* h2d_bytes, size_t* d2h_bytes, uint64_t* n_entries,
                   int32_t* kernels_per_launch);
/* Host -> device copy of the packed descriptors into dev_ws (async on stream). */
int tnc_batch_upload(tnc_batch_t* b, void* dev_ws, size_t ws_bytes, void* cuda_stream);
/* Device-only work: all contractions + CRT of the batch, results left in dev_ws.
 * Requires a prior tnc_batch_upload to the same dev_ws.  The launch sequence is
 * captured once into a CUDA graph per (dev_ws, stream) and replayed. */
int tnc_batch_launch(tnc_batch_t* b, void* dev_ws, void* cuda_stream);
/* Autotuner: times the batch's launch for every CTA size in {64, 128, 256},
 * shared-memory arena capacity in {0, 16, 32, 48, 64, 96, 128, 192} KiB
 * (capped at the largest formula's arena) and cap on CTAs per SM in {as many
 * as fit, 2, 1} (fewer CTAs leave more of the SM's memory to L1), keeps the
 * fastest and reports it.  Needs a prior tnc_batch_upload to dev_ws; leaves
 * the results of the last trial in dev_ws; synchronises the stream.  Any out
 * pointer may be NULL. */
int tnc_batch_autotune(tnc_batch_t* b, void* dev_ws, void* cuda_stream, int32_t* threads_out,
                       int32_t* smem_bytes_out, int32_t* ctas_per_sm_out);
/* Sets the launch shape without timing (threads per CTA in {64, 128, 256},
 * shared-memory arena bytes per CTA, CTAs per SM cap, 0 = as many as
 * fit; e.g. a shape an earlier autotune chose).  TNC_ERR_INVALID for another
 * CTA size, TNC_ERR_TOO_LARGE if the CTA does not fit on an SM.  Host only: no
 * device work is queued. */
int tnc_batch_set_launch(tnc_batch_t* b, int32_t threads, int32_t smem_bytes, int32_t ctas_per_sm);
/* The current launch shape (after tnc_batch_autotune: the one it chose), to be
 * kept by the caller and given back with tnc_batch_set_launch.  Any out pointer
 * may be NULL. */
int tnc_batch_get_launch(const tnc_batch_t* b, int32_t* threads, int32_t* smem_bytes, int32_t* ctas_per_sm);
/* Device -> host copy of the results; synchronises the stream.  outs: n counts. */
int tnc_batch_download(tnc_batch_t* b, const void* dev_ws, void* cuda_stream, tnc_count* outs);
/* Bulk form of tnc_batch_download: residues [E][R] and CRT limbs
 * [E][ceil(31R/32)] of all E result entries (formula after formula, 2^n_open
 * entries each, in the order the plans were given), and one TNC_* flag word
 * per formula.  Host buffers; any may be NULL; synchronises the stream. */
int tnc_batch_download_flat(tnc_batch_t* b, const void* dev_ws, void* cuda_stream, uint32_t* residues,
                            uint32_t* limbs, uint32_t* flags);
/* Status word of the last launch (0, or TNC_ERR_TIMEOUT if a bounded device
 * wait gave up); synchronises the stream. */
int tnc_batch_status(tnc_batch_t* b, const void* dev_ws, void* cuda_stream);
void tnc_free_batch(tnc_batch_t* b);

/* Upload + launch + download in one call. */
int tnc_contract_batch(const tnc_plan_t* const* plans, int32_t n, const tnc_contract_opts* opts,
                       void* dev_ws, size_t ws_bytes, void* cuda_stream, tnc_count* outs);

/* ---- learned ordering ----------------------------------------------------
 * A 3-layer perceptron scores candidate merges of a greedy contraction (the
 * edge-contraction step of Sec. 2.2); it is trained on the exact plan cost
 * the method itself predicts before contracting (the "lazy" evaluation of
 * Sec. 4), and the paper's heuristics (Sec. 3.1.1) stay the fallback and the
 * judge: a learned plan is kept only if its (max rank, MACs) is not worse.
 * Parameters: fp32, flat, W1[F][H], b1[H], W2[H][H], b2[H], w3[H], b3. */
#define TNC_MLP_FEATURES 16
#define TNC_MLP_HIDDEN 128
#define TNC_MLP_PARAMS (TNC_MLP_FEATURES * TNC_MLP_HIDDEN + TNC_MLP_HIDDEN + TNC_MLP_HIDDEN * TNC_MLP_HIDDEN + \
                        TNC_MLP_HIDDEN + TNC_MLP_HIDDEN + 1)
#define TNC_LEARNED_CANDIDATES 8 /* candidates scored per formula and merge: the cheapest
                                      by result rank (then MACs), greedy's choice first */

/* He-initialised parameters (host, TNC_MLP_PARAMS floats). */
int tnc_mlp_init(uint64_t seed, float* params);
/* Trained parameters to and from a file (host fp32, TNC_MLP_PARAMS floats):
 * magic, layout (features, hidden width, count) and a checksum are written
 * and checked; a file of another layout or a damaged one is refused
 * (TNC_ERR_INVALID) and params is left untouched. */
int tnc_learned_save(const char* path, const float* params);
int tnc_learned_load(const char* path, float* params);
/* Training rows: at `states` random points of an exploring tensor-greedy
 * trajectory of every network, each of its (at most `cands`) cheapest
 * candidate merges gets 16 features (x, host [rows][16]) and its regret
 * (t, host [rows]): log2 of the total MACs of the plan that merges it and
 * finishes by tensor-greedy, minus the least such value at that state.
 * OpenMP over networks; deterministic for a seed.  TNC_ERR_BUFFER if
 * cap_rows is too small (needed rows in *n_rows; x, t may be NULL to ask). */
int tnc_learned_dataset(const tnc_network_t* const* nets, int32_t n, int32_t states, int32_t cands,
                        uint64_t seed, float* x, float* t, int64_t cap_rows, int64_t* n_rows);
/* As tnc_learned_dataset, but the trajectories follow the learned planner's
 * own choices (scorer d_params_bf16, TNC_LEARNED_CANDIDATES candidates), so
 * that a second round of training sees the states the planner visits.
 * d_ws: tnc_plan_learned_workspace_bytes(n) device bytes. */
int tnc_learned_dataset_on_policy(const tnc_network_t* const* nets, int32_t n, const void* d_params_bf16,
                                  void* d_ws, size_t ws_bytes, void* cuda_stream, int32_t states, uint64_t seed,
                                  float* x, float* t, int64_t cap_rows, int64_t* n_rows);
/* fp32 forward over `rows` rows of x (device [rows][16]) into y (device
 * [rows]); h1, h2 (device [rows][128] each) receive the post-ReLU
 * activations for the backward pass, or may be NULL. */
int tnc_mlp_forward(const float* d_params, const float* d_x, int64_t rows, float* d_y, float* d_h1, float* d_h2,
                    void* cuda_stream);
/* Gradient of the mean squared error (1/rows) sum (y - t)^2 with respect to
 * the parameters (d_grads, overwritten), from a forward pass's y, h1, h2.
 * d_scratch: device, tnc_mlp_backward_scratch_floats(rows) floats. */
size_t tnc_mlp_backward_scratch_floats(int64_t rows);
int tnc_mlp_backward(const float* d_params, const float* d_x, const float* d_h1, const float* d_h2, const float* d_y,
                     const float* d_t, int64_t rows, float* d_scratch, float* d_grads, void* cuda_stream);
/* One Adam step (beta 0.9 / 0.999, eps 1e-8) on all parameters; step >= 1. */
int tnc_mlp_adam(float* d_params, const float* d_grads, float* d_m, float* d_v, int32_t step, float lr,
                 void* cuda_stream);
/* Whole training: `epochs` passes over the rows (already shuffled by the
 * caller) in mini-batches of `batch`, Adam with rate lr; per-epoch mean loss
 * into loss_out[epochs] (host, may be NULL).  Synchronises the stream. */
size_t tnc_mlp_train_workspace_bytes(int32_t batch);
int tnc_mlp_train(float* d_params, const float* d_x, const float* d_t, int64_t rows, int32_t epochs, int32_t batch,
                  float lr, void* d_ws, size_t ws_bytes, void* cuda_stream, float* loss_out);
/* bf16 copy of the parameters (device, TNC_MLP_PARAMS bf16) and the bf16
 * inference forward used by the learned planner. */
int tnc_mlp_to_bf16(const float* d_params, void* d_params_bf16, void* cuda_stream);
int tnc_mlp_forward_bf16(const void* d_params_bf16, const float* d_x, int64_t rows, float* d_y, void* cuda_stream);
/* Learned plans for n networks: all formulas advance in lockstep, every round
 * scoring the TNC_LEARNED_CANDIDATES cheapest candidates of each in one bf16
 * inference launch and merging each formula's lowest predicted regret.
 * Each learned plan is then compared with the heuristic plan of `fallback`
 * (NULL: TNC_PLAN_BEST); the one with the smaller (max rank, MACs) is kept.
 * chose_learned[i] = 1 if the learned plan was kept; learned_macs[i] = its
 * MACs either way (both may be NULL).  d_ws: device,
 * tnc_plan_learned_workspace_bytes(n) bytes.  All or nothing on failure. */
size_t tnc_plan_learned_workspace_bytes(int32_t n);
int tnc_plan_learned_many(const tnc_network_t* const* nets, int32_t n, const void* d_params_bf16,
                          const tnc_plan_opts* fallback, void* d_ws, size_t ws_bytes, void* cuda_stream,
                          tnc_plan_t** out, tnc_plan_stats* stats, int32_t* chose_learned, double* learned_macs);

/* Learned coarsening with heuristic completion.  The learned merges (the
 * scorer's lowest predicted regret among the TNC_LEARNED_CANDIDATES cheapest
 * merges, as above) coarsen the network; after checkpoints[j] % of a
 * formula's merges the partial contraction is finished by `completion`, one
 * of the paper's heuristics, planned on the network of the live tensors, and
 * the cheapest of these plans is the learned plan, kept only if it is not
 * worse than `fallback` on the whole network (the paper's heuristic as judge).
 * Training rows for this mode label a candidate merge by the cost of the plan
 * that makes it and is then finished by `completion` (the lazy cost of
 * Sec. 4), at states drawn among the first max_pct % of the merges. */
typedef struct {
  int32_t states;         /* dataset: states sampled per formula                     */
  int32_t cands;          /* dataset: candidates labelled per state                  */
  int32_t completion;     /* TNC_PLAN_*; TNC_PLAN_GREEDY with no checkpoints: the
                             learned merges go to the end (tnc_plan_learned_many)    */
  int32_t n_checkpoints;  /* 0..8                                                     */
  int32_t checkpoints[8]; /* percent of a formula's merges                           */
  int32_t max_pct;        /* dataset: states among the first max_pct % (<= 0: 100)   */
  uint64_t seed;          /* dataset sampling; seed of the randomised completion      */
} tnc_learned_opts;
/* d_params_bf16 NULL: the merges follow tensor-greedy's choice (the same
 * coarsening without the scorer, for comparison); no device work then. */
int tnc_plan_learned_opts(const tnc_network_t* const* nets, int32_t n, const void* d_params_bf16,
                          const tnc_learned_opts* o, const tnc_plan_opts* fallback, void* d_ws, size_t ws_bytes,
                          void* cuda_stream, tnc_plan_t** out, tnc_plan_stats* stats, int32_t* chose_learned,
                          double* learned_macs);
/* Rows for this mode; d_params_bf16 NULL: exploring tensor-greedy
 * trajectories, else the learned planner's own. */
int tnc_learned_dataset_opts(const tnc_network_t* const* nets, int32_t n, const tnc_learned_opts* o,
                             const void* d_params_bf16, void* d_ws, size_t ws_bytes, void* cuda_stream, float* x,
                             float* t, int64_t cap_rows, int64_t* n_rows);

/* ---- diagnostics --------------------------------------------------------- */
/* Measured rate of the modular multiply-accumulate primitive of the step
 * kernels (4 residues per thread, 64-bit accumulation, reduced after every
 * 16th product by the two-fold reduction the step kernels use for the default
 * primes just below 2^30), operands in registers, all SMs busy: a ceiling for
 * steps bound by the integer pipes.  `iters` loop trips per thread (16 MACs each).
 * Allocates an 8-byte device counter with cudaMallocAsync; synchronises. */
int tnc_probe_modmac(void* cuda_stream, int32_t iters, double* macs_per_s);

/* ---- fault injection (host side; the paper has no counterpart) ----------
 * Arms one failure: the (after+1)-th later call site of the given kind, in
 * any thread, fails as described, and the injection disarms itself.  No
 * device fault is ever made: LAUNCH fails before the call's first device
 * call, TIMEOUT after the call's device work has completed (the status word a
 * bounded device wait would have set).  TNC_INJECT_NONE disarms. */
#define TNC_INJECT_NONE 0
#define TNC_INJECT_NOMEM 1   /* tnc_build_network / tnc_plan / tnc_batch_create:
                                host allocation fails -> TNC_ERR_NOMEM            */
#define TNC_INJECT_PLAN 2    /* tnc_plan (also inside tnc_plan_many) -> TNC_ERR_TOO_LARGE */
#define TNC_INJECT_LAUNCH 3  /* tnc_contract / _sliced / _noalloc / tnc_batch_launch
                                -> TNC_ERR_CUDA, nothing enqueued                  */
#define TNC_INJECT_TIMEOUT 4 /* tnc_contract / _sliced: the device status reads as a
                                timed-out wait -> TNC_ERR_TIMEOUT                  */
int tnc_inject_failure(int32_t kind, int32_t after);

/* ---- allocation-free variant (the paper has no counterpart) --------------
 * The counts of tnc_contract on TNC_PATH_INT64 (the only path it takes: other
 * paths fail with TNC_ERR_INVALID), for callers that cannot allocate device
 * memory themselves: a host application whose device memory is owned entirely by
 * another allocator (a framework's caching pool that forbids raw cudaMalloc),
 * or a latency-bound loop that cannot afford cudaMalloc/cudaFree, which may
 * synchronise the whole device.  It calls no cudaMalloc, cudaFree or other
 * allocating routine; its device scratch is one fixed array of
 * TNC_NOALLOC_SCRATCH_BYTES inside libtnc, held on every GPU that loads the
 * library until the process exits.  The caller still passes the plan (input)
 * and the host result buffers of `out` (output).
 *   - The first call on each device looks up that array's device address
 *     (cudaGetSymbolAddress) with the device current; make that first call
 *     before any stream capture.  The address is kept with the device's
 *     context; if the context changes (after cudaDeviceReset) the next call
 *     looks it up again.
 *   - Every call shares the one array: calls that overlap on the GPU (other
 *     streams, other host threads, same device) race and corrupt each other's
 *     results.  Serialise them.  Nothing in the array needs to start zeroed,
 *     so the previous call's contents do no harm.
 *   - A plan whose scratch (tnc_workspace_bytes for the same R) exceeds the
 *     array fails with TNC_ERR_TOO_LARGE and a message giving both sizes.
 *   - Synchronises `cuda_stream` before returning. */
#define TNC_NOALLOC_SCRATCH_BYTES (32u << 20)
int tnc_contract_noalloc(const tnc_plan_t* plan, const tnc_contract_opts* opts, void* cuda_stream,
                         tnc_count* out);

#ifdef __cplusplus
}
#endif
#endif /* TNC_H */
