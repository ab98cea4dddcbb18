/*
 * lsyn.h — C ABI of the GB300 (sm_103a) library for bottom-up semantic
 * enumeration of LTLf formulae from positive and negative example traces.
 *
 * The method is the one of "GPU accelerated program synthesis: Enumerate
 * semantics, not syntax!" (arXiv 2504.18943):
 *
 *  - A specification (P, N) is a pair of finite sets of finite traces over the
 *    powerset of the propositions p0..p{n-1}; a formula separates (P, N) when it
 *    holds at position 0 of every trace of P and of no trace of N (section
 *    "Synthesising linear temporal logic formulae from examples").
 *  - Formulae: atoms, not (!), and (&), or (|), next (X), future (F),
 *    globally (G, read as "not F not"), until (U). Size = number of syntax-tree
 *    nodes. Satisfaction is over finite traces; nothing holds at or beyond the
 *    end of a trace.
 *  - A formula is represented only by its characteristic matrix (CM): one word
 *    per trace whose bit t says whether the formula holds at position t
 *    (section "Parallel enumeration of LTLf formulae on GPUs", characteristic
 *    sequence and matrix). Two formulae with equal CMs are observationally
 *    equivalent and only the first one found is kept.
 *  - Level k (all new CMs of size k) is built from levels < k by bitwise
 *    operators (paragraph "Logical operations as bitwise operations"), every
 *    candidate is checked against the specification, and new CMs go into a
 *    device-resident language cache (the listing of paragraph "A generic program
 *    synthesiser", section "Program synthesis"). The first level that holds a
 *    separating CM gives a minimal-size formula.
 *
 * Conventions for every call:
 *  - Return value: an lsyn_status. Negative values are errors; no C++
 *    exception crosses this boundary. lsyn_last_error() gives a message.
 *  - Pointers documented as "host" point to ordinary CPU memory; the library
 *    copies what it needs before returning (inputs) or writes results there
 *    before returning (outputs). The caller keeps ownership.
 *  - Device memory is owned by the context and released by lsyn_destroy().
 *  - One context is used by one host thread at a time. All device work of a
 *    context is issued on the stream given in lsyn_config, except the clear of
 *    a large hash table after lsyn_reset, which runs on a stream of the
 *    context's own, ordered by events (see lsyn_reset).
 *  - Formula text: prefix, fully parenthesised, atoms p0..p{n-1}, e.g.
 *    "(U (! p1) (& p0 (X p1)))". Unary: "(! f)", "(X f)", "(F f)", "(G f)";
 *    binary: "(& f g)", "(| f g)", "(U f g)".
 */
#ifndef LSYN_H_
#define LSYN_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  LSYN_OK = 0,
  LSYN_NOT_FOUND = 1,       /* no separating formula up to the requested size */
  LSYN_PENDING = 2,         /* (serving) the request is not finished yet */
  LSYN_E_INVAL = -1,        /* an argument is out of range or inconsistent */
  LSYN_E_NOMEM = -2,        /* a device allocation failed */
  LSYN_E_CUDA = -3,         /* a CUDA runtime call failed */
  LSYN_E_UNSUPPORTED = -4,  /* a valid request the library does not handle (CMs above 64 KiB) */
  LSYN_E_CACHE_FULL = -5,   /* the language cache ran out of space: deeper levels cannot be built */
  LSYN_E_TIMEOUT = -6,      /* a deadline passed between levels */
  LSYN_E_STATE = -7         /* call out of order, or an internal consistency check failed */
} lsyn_status;

/* Operator mask bits (lsyn_config.op_mask). */
#define LSYN_OP_NOT 0x01u
#define LSYN_OP_AND 0x02u
#define LSYN_OP_OR 0x04u
#define LSYN_OP_X 0x08u
#define LSYN_OP_F 0x10u
#define LSYN_OP_G 0x20u
#define LSYN_OP_U 0x40u
#define LSYN_OPS_ALL 0x7Fu
/* The grammar printed in the paper: atoms, not, and, X, F, U. */
#define LSYN_OPS_PAPER (LSYN_OP_NOT | LSYN_OP_AND | LSYN_OP_X | LSYN_OP_F | LSYN_OP_U)

/*
 * A specification (P, N), positives first (section "Synthesising linear
 * temporal logic formulae from examples"; the fixed total order on P ∪ N of the
 * characteristic matrix, section "Parallel enumeration of LTLf formulae on
 * GPUs").
 *   n_props     number of atomic propositions, 1..32.
 *   n_pos       |P| >= 0;  n_neg = |N| >= 0;  n_pos + n_neg >= 1.
 *   word_bits   32 or 64: bits per characteristic-sequence word. A trace
 *               longer than a word takes W = ceil(longest trace / word_bits)
 *               words (at most 16; the paper's one word per trace when W = 1).
 *   lengths     host, int32[n_pos + n_neg]: trace lengths, each
 *               1..16 x word_bits.
 *   atom_words  host, [n_props][n_pos + n_neg][W] words of word_bits bits
 *               (uint32_t or uint64_t), row-major. Bit t of word (p, i, w) is 1
 *               iff p holds at position w x word_bits + t of trace i. Bits at
 *               positions >= lengths[i] are ignored.
 */
typedef struct {
  int32_t n_props;
  int32_t n_pos;
  int32_t n_neg;
  int32_t word_bits;
  const int32_t* lengths;
  const void* atom_words;
} lsyn_problem;

/* Device allocator hooks: return a device pointer (NULL on failure) / free it. */
typedef void* (*lsyn_alloc_fn)(size_t bytes, void* user);
typedef void (*lsyn_free_fn)(void* ptr, void* user);

/*
 * Context configuration. A zero-filled struct selects every default.
 *   op_mask      operators to enumerate (LSYN_OP_*); 0 = LSYN_OPS_ALL.
 *   cache_bytes  device bytes for the language cache: CM arena, provenance and
 *                hash table together; 0 = 1 GiB.
 *   table_load   maximum load factor of the hash table in (0, 0.9]; 0 = 0.5.
 *   full_levels  0: a level stops at its first separating candidate (the early
 *                return of the listing); 1: every level is built completely even
 *                when it holds a solution (used to compare whole levels).
 *   timing       1 records CUDA events around each kernel launch and fills the
 *                kernel_ms fields of lsyn_level_stats.
 *   alloc, free, alloc_user   device allocator (e.g. the PyTorch caching
 *                allocator); NULL = cudaMalloc / cudaFree.
 *   stream       cudaStream_t for all device work; NULL = the legacy default stream.
 *   device       CUDA device ordinal; -1 or 0..n-1 (the current device if -1).
 *                One process drives one device: the kernels' shared-memory
 *                attributes are set once per process, on the device that
 *                first launches them, so contexts, batches or servers of one
 *                process on a second device fail their launches (LSYN_E_CUDA).
 *                Run one process per GPU (as bench.py does).
 *   tile_rows    0: automatic; 8, 16 or 32: rows of each side of the block
 *                tiles of the binary launch for 512-byte CMs (k_binary_c),
 *                kept at every level. By default a tile starts at 32 rows and
 *                is halved (to 16, then 8) while the level gives fewer than
 *                two tiles per resident block. The tile changes only the order
 *                in which pairs are visited, never a level's set of CMs; the
 *                field exists so that each tile size can be checked at any
 *                level. Other values: LSYN_E_INVAL.
 *   defer_cap    entries of each of the two deferred-candidate lists; 0 =
 *                automatic (cache entries / 16, within 2^16..2^23). A level
 *                that defers more candidates than this fails with
 *                LSYN_E_STATE ("deferred list overflow").
 *   hole_cap     entries of the hole log (id ranges warps reserved and left
 *                unused, closed after each level); 0 = 2^16. A level that
 *                logs more fails with LSYN_E_STATE. After either failure the
 *                context must be reset (lsyn_reset) before it is used again.
 *   time_limit_ms  0: none. Otherwise lsyn_solve checks, before building each
 *                level after the first one it builds, whether this much time
 *                has passed since it was called, and if so stops with
 *                LSYN_E_TIMEOUT; the levels built so far stay complete and a
 *                later lsyn_solve continues from them. A later level (not the
 *                first the call builds, which always runs to its end) that is
 *                running when the limit passes is stopped by its kernels at their next
 *                poll (every few warp batches; once per tile), and lsyn_solve
 *                returns LSYN_E_TIMEOUT with out->levels_done complete levels;
 *                the interrupted level's entries are in the cache, so the
 *                context answers LSYN_E_STATE until it is reset (lsyn_reset).
 *                lsyn_enumerate_level on its own keeps no time limit.
 * The fields after `device` were added later; a zero-filled struct keeps every
 * default.
 */
typedef struct {
  uint32_t op_mask;
  uint64_t cache_bytes;
  float table_load;
  int32_t full_levels;
  int32_t timing;
  lsyn_alloc_fn alloc;
  lsyn_free_fn free;
  void* alloc_user;
  void* stream;
  int32_t device;
  int32_t tile_rows;
  uint32_t defer_cap;
  uint32_t hole_cap;
  double time_limit_ms;
} lsyn_config;

/* Per-level statistics (filled by lsyn_enumerate_level). */
typedef struct {
  int32_t level;          /* k */
  int32_t solved;         /* 1 if a candidate of this level separates (P, N) */
  int32_t cache_full;     /* 1 if an insert failed for lack of space: the level is incomplete */
  int32_t early_exit;     /* 1 if the level stopped at a solution before building every candidate */
  int64_t candidates;     /* candidate formulae built at this level (and/or once per unordered pair) */
  int64_t unique;         /* new characteristic matrices added to the cache: |L_k| */
  int64_t total;          /* entries in the cache after this level */
  int64_t deferred;       /* candidates re-examined after meeting an unpublished slot */
  double ms;              /* wall time of the level (host clock, includes the final sync) */
  double kernel_ms[4];    /* with timing=1: device time of the unary, binary, resolve and other launches */
  double bytes_alg;       /* algorithmic bytes of the level (operand reads, probes, compares, inserts) */
  double bytes_binary;    /* the part of bytes_alg moved by the binary-operator launch */
  double bytes_unary;     /* the part of bytes_alg moved by the unary-operator launch */
  int32_t launches;       /* kernel launches issued for this level */
  int32_t reserved;
} lsyn_level_stats;

/*
 * Result of lsyn_solve.
 *   formula / formula_cap  caller-owned host buffer for the formula text
 *                          (LSYN_E_INVAL if too small).
 *   level_stats / level_stats_cap  optional caller-owned host array: entry
 *                          k - 1 receives the statistics of level k when this
 *                          call builds level k and k <= level_stats_cap.
 */
typedef struct {
  int32_t found;          /* 1 if a separating formula was found */
  int32_t size;           /* its size (syntax-tree nodes) */
  int32_t exact;          /* 1 if minimal: every smaller level was complete */
  int32_t levels_done;    /* levels built so far */
  int64_t constructed;    /* candidates built over all levels, atoms included */
  int64_t unique;         /* entries in the language cache */
  double ms;              /* wall time of the call */
  int32_t launches;       /* kernel launches issued by this call */
  int32_t level_stats_cap;
  lsyn_level_stats* level_stats;
  char* formula;
  size_t formula_cap;
} lsyn_result;

typedef struct lsyn_ctx lsyn_ctx;

/*
 * Create a context for one specification: validates the problem, allocates the
 * language cache and scratch on the device, copies the traces there and builds
 * nothing yet. *out receives the context, or NULL on error (then
 * lsyn_last_error(NULL) explains). Errors: LSYN_E_INVAL (bad sizes, lengths out
 * of 1..16 x word_bits, more than 2^30 - 2 cache entries requested),
 * LSYN_E_UNSUPPORTED (a CM above 64 KiB), LSYN_E_NOMEM, LSYN_E_CUDA.
 */
lsyn_status lsyn_create(const lsyn_problem* problem, const lsyn_config* config, lsyn_ctx** out);

/* Release every device buffer of the context (after its stream's work is done). NULL is allowed. */
void lsyn_destroy(lsyn_ctx* ctx);

/* Message of the last error on this context; with NULL, of the last failed lsyn_create on this thread. */
const char* lsyn_last_error(const lsyn_ctx* ctx);

/*
 * Forget every level (keeps the traces and the memory); the next level to
 * build is 1. Asynchronous on the context's stream. A context whose hash table
 * has at least 2^23 slots builds its first levels in a small 8 MiB table and
 * clears the large one meanwhile on a stream of its own (ordered after the
 * work queued on the context's stream before this call); the level that first
 * needs the large table waits for that clear, a solve that returns earlier
 * joins it into the context's stream, and lsyn_destroy waits for it.
 * Errors: LSYN_E_INVAL (NULL), LSYN_E_STATE (a batch or server problem),
 * LSYN_E_CUDA.
 */
lsyn_status lsyn_reset(lsyn_ctx* ctx);

/*
 * Build level k = levels_done + 1 (the listing of "A generic program
 * synthesiser": every operator, every split of k-1 into child sizes, every
 * pair of cached programs; level 1 is the distinct atoms). Every candidate is
 * checked against the specification; new CMs are inserted into the cache.
 * out (host, may be NULL) receives the level's statistics.
 * Errors: LSYN_E_STATE if k is not the next level, or the previous level is
 * incomplete (cache full or stopped early); LSYN_E_CACHE_FULL is NOT returned
 * here (see out->cache_full); LSYN_E_CUDA.
 */
lsyn_status lsyn_enumerate_level(lsyn_ctx* ctx, int32_t k, lsyn_level_stats* out);

/*
 * Build levels until one holds a separating formula, or max_size (1..64) is
 * passed. On LSYN_OK out->formula holds a separating formula of minimal size
 * out->size (minimal when out->exact is 1). Returns LSYN_NOT_FOUND when no
 * formula up to max_size separates, LSYN_E_CACHE_FULL when the cache filled up
 * before a solution was found (levels up to out->levels_done are exact), and
 * LSYN_E_TIMEOUT when config->time_limit_ms passed before a level could start
 * (out->levels_done complete levels are kept; calling again continues).
 */
lsyn_status lsyn_solve(lsyn_ctx* ctx, int32_t max_size, lsyn_result* out);

/* Number of entries of level k (1 <= k <= levels_done) in *n_out. */
lsyn_status lsyn_level_count(const lsyn_ctx* ctx, int32_t k, int64_t* n_out);

/*
 * Copy the CMs of entries [first, first + count) of level k into dst (host):
 * count rows of (n_pos + n_neg) x W words of word_bits bits (W words per trace
 * as in lsyn_problem), positives first, the rows in the cache's (unspecified,
 * run-dependent) order. cap = bytes of dst.
 */
lsyn_status lsyn_export_level(lsyn_ctx* ctx, int32_t k, int64_t first, int64_t count,
                              void* dst, size_t cap);

/* Formula text of entry `index` of level k (host buffer of cap bytes). */
lsyn_status lsyn_entry_formula(lsyn_ctx* ctx, int32_t k, int64_t index, char* buf, size_t cap);

/*
 * Evaluate a formula on every trace of a problem (the bitwise operators on the
 * device). dst (host) receives (n_pos + n_neg) x W words of word_bits bits
 * (W words per trace as in lsyn_problem): the formula's CM. config may be NULL
 * (defaults). Errors: LSYN_E_INVAL on a parse error, an atom >= n_props or more
 * than 4096 nodes.
 */
lsyn_status lsyn_eval(const lsyn_problem* problem, const char* formula, void* dst,
                      const lsyn_config* config);

/*
 * Multi-problem scheduling (batches and the server). The paper enumerates one
 * specification at a time; this library also advances many at once, each at
 * its own level, in one persistent launch per step over a packed work list of
 * every admitted problem (the listing of "A generic program synthesiser"
 * applied to each problem).
 *
 * Two lanes share the GPU: small levels of every admitted problem advance in
 * batch steps (one persistent launch each) on a high-priority stream, while a
 * level with more than solo_candidates candidates runs in the large-level lane
 * (the one-problem kernels on streams of their own, on all but light_sms SMs;
 * up to `lanes` problems' levels at once, taken in admission order). A step
 * never waits for a large level, so small problems are not held up by large
 * ones.
 *
 * Memory: per-problem language caches live in one device memory pool
 * (pool_bytes). A cache starts small and grows before each level to the
 * entries the level is predicted to add, without copying (virtual address
 * ranges backed on demand), up to the same entry limit lsyn_create derives
 * from config->cache_bytes. So each problem's levels, status and answer size
 * are those of lsyn_create + lsyn_solve with the same config, whatever else
 * runs beside it; only which separating formula of the minimal size is
 * returned may differ. A level that outgrows its prediction is undone and run
 * again with room for every candidate. When the pool cannot hold a problem's
 * next level it waits; when nothing can run, the most recently admitted
 * problems are evicted (their caches dropped, restarted later). A problem that
 * does not fit even alone is capped at what the pool gives it and answers
 * LSYN_E_CACHE_FULL (its error text says so).
 */
typedef struct {
  int32_t blocks_per_sm;  /* persistent blocks of 256 threads per SM (0 = 4) */
  int32_t use_graph;      /* 1: replay the step (upload, reset, launch, copy back) from CUDA graphs */
  int32_t max_active;     /* problems admitted at once (0: a batch admits all, a server 256) */
  int32_t predict_pct;    /* a level's predicted new entries: candidates x this percentage of the
                             previous level's unique ratio (0 = 150); lower saves memory, costs redos */
  uint64_t pool_bytes;    /* device memory for every cache together (0: 90% of the free memory) */
  uint64_t solo_candidates; /* a level with more candidates is a large level: it runs in the large-level
                               lane with the one-problem kernels, beside the batch steps (0 = 2^19) */
  int32_t light_sms;      /* SMs the batch steps keep while a large level runs (0 = 1/8 of the SMs) */
  int32_t lanes;          /* large levels of different problems in flight at once (0 = 4) */
  int32_t rows_per_item;  /* formulas per warp: rows of the unary work and pairs of the binary work in
                             one work item of a batch step, each with its 4 operators (2, 4 or 8; 0 = 8) */
  int32_t words_per_thread; /* CMs above 128 bytes: 16-byte vectors a lane loads together in each step
                             of its loops over a CM (1 or 2; 0 = 1) */
  int32_t table_load_pct; /* load, in percent (25..90), up to which a problem's hash table fills before
                             it is rebuilt larger (0 = the config's table_load). Only the table's size
                             follows it: the problem's entry limit stays the one lsyn_create derives
                             from cache_bytes and table_load, so answers do not change. */
} lsyn_batch_tuning;

typedef struct {
  int64_t submitted, completed, active, queued;
  int64_t steps;          /* batch steps run */
  int64_t evictions;      /* problems evicted and restarted for lack of memory */
  int64_t redos;          /* levels undone and run again (outgrew their prediction) */
  int64_t large_levels;   /* levels run in the large-level lane */
  uint64_t pool_bytes, pool_in_use, pool_peak;
} lsyn_sched_stats;

/*
 * One unit of scheduler work (a trace for tuning; the last 4096 are kept):
 * a batch step (lane 0) or one large level (lane 1; times are as the host saw
 * them between steps).
 */
typedef struct {
  int64_t step;           /* batch steps run before it */
  int32_t lane;           /* 0: batch step, 1: large level */
  int32_t active;         /* problems advanced (1 for a large level) */
  int32_t solo;           /* batch step: a large level was in flight beside it */
  int32_t passes;         /* deferred-candidate passes */
  int32_t finished;       /* problems answered */
  int32_t level;          /* large level: its size k */
  double plan_ms;         /* host: predictions, cache growth, table rebuild launches */
  double run_ms;          /* the launches until their counters are back */
  double settle_ms;       /* deferred passes, hole fixups, commits, answers */
  uint64_t candidates;    /* candidates built */
  uint64_t pool_in_use;
} lsyn_step_trace;

/*
 * Batched solving of n independent specifications.
 *   problems   host array of n problem descriptions (32- and 64-bit words may
 *              be mixed); copied during the call.
 *   config     shared by every problem; cache_bytes is each problem's cap.
 *   tuning     NULL = defaults.
 * Errors: as lsyn_create (the first failing problem is named in
 * lsyn_batch_last_error(NULL)); LSYN_E_CUDA if the driver's virtual-memory
 * interface is unavailable.
 */
typedef struct lsyn_batch lsyn_batch;

lsyn_status lsyn_batch_create(const lsyn_problem* problems, int32_t n, const lsyn_config* config,
                              const lsyn_batch_tuning* tuning, lsyn_batch** out);

/*
 * Solve every problem up to max_size (1..17). results (host, n entries, each
 * with its own caller-owned formula buffer) receive what lsyn_solve would
 * return, ms = time from the start of this call to the problem's answer;
 * statuses[i] receives the status lsyn_solve would return for problem i
 * (LSYN_OK, LSYN_NOT_FOUND, LSYN_E_CACHE_FULL; LSYN_E_NOMEM if the pool cannot
 * hold even its constants). Caches of answered problems stay on the device for
 * lsyn_batch_problem until their memory is needed. The call itself returns
 * LSYN_OK unless a CUDA error or a consistency check stops the whole batch.
 */
lsyn_status lsyn_batch_solve(lsyn_batch* batch, int32_t max_size, lsyn_result* results, int32_t* statuses);

/*
 * Autotuner: solves the batch (up to max_size) repeatedly, one parameter at a
 * time over formulas per warp (rows_per_item {2, 4, 8}), words per thread
 * {1, 2}, table sizing (table_load_pct {25, 50, 75}), blocks per SM {2, 4, 8},
 * step graphs {off, on}, solo_candidates {2^17, 2^19, 2^21} and light_sms
 * {1/16, 1/8, 1/4 of the batch's device's SMs}, keeping the fastest value of
 * each (coordinate descent); the result serves later lsyn_batch_solve calls
 * and is written to *out (may be NULL). No tuning point changes an answer.
 */
lsyn_status lsyn_batch_autotune(lsyn_batch* batch, int32_t max_size, lsyn_batch_tuning* out);

/*
 * Problem i of the batch as a context handle owned by the batch (valid until
 * lsyn_batch_destroy; lsyn_destroy ignores it). Read-only calls
 * (lsyn_level_count, lsyn_export_level, lsyn_entry_formula) inspect the levels
 * the last lsyn_batch_solve built for that problem while its cache is
 * resident (otherwise they see no levels); driving calls answer LSYN_E_STATE.
 */
lsyn_status lsyn_batch_problem(lsyn_batch* batch, int32_t i, lsyn_ctx** out);

lsyn_status lsyn_batch_stats(const lsyn_batch* batch, lsyn_sched_stats* out);

/* The step trace of the last lsyn_batch_solve: up to cap entries into out, their count in *n_out. */
lsyn_status lsyn_batch_trace(const lsyn_batch* batch, lsyn_step_trace* out, int32_t cap, int32_t* n_out);

/* Message of the last error of the batch (NULL: of the last failed lsyn_batch_create on this thread). */
const char* lsyn_batch_last_error(const lsyn_batch* batch);

/* Release the batch and every problem's device memory. NULL is allowed. */
void lsyn_batch_destroy(lsyn_batch* batch);

/*
 * Divide-and-conquer (paragraph "Divide-and-conquer"): a specification with no
 * separating formula of size <= max_size that fits its cache is split into
 * four parts (P_i, N_j), i, j = 1, 2 — P_1 the first ceil(|P| / 2) positive
 * traces, P_2 the rest, N_1 and N_2 likewise — the parts are solved
 * recursively and recombined as (phi_11 & phi_12) | (phi_21 & phi_22). A part
 * with a single positive trace splits N only (phi_1 & phi_2); one with a
 * single negative trace splits P only (phi_1 | phi_2). The parts pending at
 * each depth are solved together, as one batch of the scheduler above.
 *   problem    as for lsyn_create (copied); max_size 1..17 for every part.
 *   config     per-part settings (cache_bytes = each part's cap); tuning as
 *              for a batch (NULL = defaults).
 *   out        found / size (nodes of the returned formula) / formula text
 *              (caller's buffer) / ms / constructed and unique (summed over
 *              every part solved); exact = 1 only if no split was needed
 *              (the answer is then minimal; otherwise it separates but need
 *              not be minimal).
 *   stats      may be NULL.
 * Returns LSYN_OK, LSYN_NOT_FOUND if a part of one positive and one negative
 * trace has no separating formula up to max_size (for example two equal
 * traces), LSYN_E_INVAL (bad problem or max_size, or out->formula too small:
 * out->formula_cap is then not changed and the needed length is in
 * stats->formula_len), or an error of the scheduler.
 */
typedef struct {
  int32_t rounds;         /* depths solved */
  int32_t splits;         /* parts that were split */
  int32_t leaves;         /* parts answered directly */
  int32_t depth;          /* deepest part (0 = the whole specification) */
  int64_t parts;          /* parts solved in all */
  int64_t formula_len;    /* length of the combined formula text */
  int64_t reserved[2];
} lsyn_dc_stats;

lsyn_status lsyn_dc_solve(const lsyn_problem* problem, int32_t max_size, const lsyn_config* config,
                          const lsyn_batch_tuning* tuning, lsyn_result* out, lsyn_dc_stats* stats);

/* Message of this thread's last failed lsyn_dc_solve. */
const char* lsyn_dc_last_error(void);

/*
 * Serving: a host thread runs the step loop over the problems submitted so
 * far. A submission joins the loop between steps as soon as a slot and pool
 * memory allow (admission in submission order, by the memory the running
 * problems are predicted to need next plus what the newcomer needs first), so
 * problems arriving while others are on the GPU share their launches
 * (continuous batching). Results are collected by ticket.
 *   config   per-problem settings as for a batch (cache_bytes = each cap).
 *   tuning   NULL = defaults (256 problems at once, 90% of free memory).
 * Thread safety: every lsyn_server_* call, lsyn_submit, lsyn_poll and
 * lsyn_wait may be made from any host thread.
 */
typedef struct lsyn_server lsyn_server;

lsyn_status lsyn_server_create(const lsyn_config* config, const lsyn_batch_tuning* tuning, lsyn_server** out);

/*
 * Queue a problem (copied during the call) to be solved up to max_size
 * (1..17). *ticket names it for lsyn_poll / lsyn_wait. Errors: LSYN_E_INVAL
 * (invalid problem or max_size; nothing is queued), LSYN_E_STATE (the server
 * stopped after an error).
 */
lsyn_status lsyn_submit(lsyn_server* server, const lsyn_problem* problem, int32_t max_size, uint64_t* ticket);

/*
 * LSYN_PENDING while the problem waits or runs. Once it is answered: its
 * status (as lsyn_solve's: LSYN_OK, LSYN_NOT_FOUND, LSYN_E_CACHE_FULL, or an
 * error), with *out filled as lsyn_solve fills it (formula into
 * out->formula / formula_cap; ms = time from submission to the answer, queueing
 * included); the ticket is then retired. LSYN_E_INVAL for an unknown or
 * retired ticket, or if out->formula is too small (the result is kept).
 */
lsyn_status lsyn_poll(lsyn_server* server, uint64_t ticket, lsyn_result* out);

/* As lsyn_poll, but waits up to timeout_ms (< 0: no limit); LSYN_E_TIMEOUT if still pending. */
lsyn_status lsyn_wait(lsyn_server* server, uint64_t ticket, int32_t timeout_ms, lsyn_result* out);

lsyn_status lsyn_server_stats(lsyn_server* server, lsyn_sched_stats* out);

/* The server's most recent steps (oldest first): up to cap entries into out, their count in *n_out. */
lsyn_status lsyn_server_trace(lsyn_server* server, lsyn_step_trace* out, int32_t cap, int32_t* n_out);

/* Message of the server's last error (NULL: of the last failed lsyn_server_create on this thread). */
const char* lsyn_server_last_error(const lsyn_server* server);

/* Stop the loop (running problems are dropped) and release everything. NULL is allowed. */
void lsyn_server_destroy(lsyn_server* server);

/*
 * Formula evaluation that allocates no device memory (the paper has no
 * counterpart; it is a service for callers that cannot call cudaMalloc, such
 * as a process whose memory manager owns every device allocation, or a
 * latency-critical loop where an allocation that may synchronise the device is
 * not acceptable). Same result as lsyn_eval, on buffers the caller already
 * holds on the current device:
 *   atom_words  device, [n_props][n_traces] words of word_bits bits, row-major
 *               by proposition (bit t of word (p, i): p holds at position t of
 *               trace i); bits at positions >= the trace's length are ignored.
 *   lengths     device, int32[n_traces]; each is clamped to 0..word_bits (one
 *               word per trace: longer traces need lsyn_eval).
 *   dst         device, n_traces words of word_bits bits: the formula's CM.
 *   stream      cudaStream_t (NULL = legacy default stream); the call only
 *               enqueues work, synchronise the stream before reading dst.
 * Per-node scratch lives in a fixed 8 MiB device array inside the library,
 * one per GPU, held until the process exits: (nodes x n_traces x word_bits/8)
 * must not exceed 8 MiB and a formula may have at most 960 nodes, otherwise
 * LSYN_E_INVAL with a message in lsyn_last_error(NULL). The CUDA runtime loads
 * the library's device code lazily, so the array is reserved on a device when
 * the first call there loads this entry point's code (that first call also
 * looks the array's device address up, with cudaGetSymbolAddress): it may
 * allocate and synchronise inside the driver. Make that first call on each
 * device as a warm-up (a one-node formula will do) before a memory manager
 * claims the GPU's memory, and before capturing the stream into a graph.
 * Every call shares the array and it keeps the last call's contents (nothing
 * in it needs clearing); calls that overlap on the GPU race on it. The call
 * itself invokes no cudaMalloc, cudaFree or other allocating routine.
 */
lsyn_status lsyn_eval_noalloc(int32_t n_props, int32_t n_traces, int32_t word_bits, const void* atom_words,
                              const int32_t* lengths, const char* formula, void* dst, void* stream);

/*
 * Host-only helper (no GPU needed): the number of candidates level k builds
 * when every level i < k holds level_sizes[i - 1] entries (k >= 2; and/or
 * counted once per unordered pair, U per ordered pair, unary once per entry).
 */
int64_t lsyn_level_candidates(const int64_t* level_sizes, int32_t k, uint32_t op_mask);

/* Library version string. */
const char* lsyn_version(void);

#ifdef __cplusplus
}
#endif

#endif /* LSYN_H_ */
