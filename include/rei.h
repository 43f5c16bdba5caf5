/*
 * rei.h -- C ABI of the GB300 (sm_103a) regular-expression-inference library.
 *
 * The library solves the problem stated in Valizadeh & Berger, "Search-Based
 * Regular Expression Inference on a GPU" (PLDI 2023): given an alphabet,
 * positive examples P and negative examples N (Def. "specification", Sec. 3),
 * a cost homomorphism (c_sym, c_?, c_*, c_., c_+) with every constant >= 1
 * (Def. "cost function", Sec. 3) and a maximum cost (Alg. 1 inputs), return a
 * regular expression that accepts all of P, rejects all of N and has minimal
 * cost, or report that none exists up to the maximum cost.
 *
 * Method (Sec. 3): every candidate language is a bitvector (characteristic
 * sequence, CS) over the infix closure ic(P u N) in shortlex order; languages
 * are built bottom-up by cost (Alg. 1), union by OR, r? by OR with the eps
 * bit, concatenation and star through a guide table of splits (Alg. 2 and the
 * "Staging: guide table" paragraph), deduplicated against every language seen
 * so far ("Uniqueness checking") and tested for precision.
 *
 * Conventions of every entry point:
 *   - Return values are rei_status codes; no exception crosses the ABI.
 *   - Inputs are read (or copied) during the call: the caller may free them
 *     when it returns.  Outputs go to caller-owned buffers; a buffer that is
 *     too small yields REI_EBUFSZ with the needed size written back.
 *   - Device memory comes from the context's allocator (rei_alloc callbacks,
 *     e.g. a framework's caching allocator) or, without one, cudaMallocAsync
 *     on the context stream.  Work is issued on the context stream.
 *   - A context is used by one host thread at a time, except the server
 *     calls that say otherwise.
 *
 * Fixed readings of the paper (the CPU oracle in the tests follows the same):
 *   - ic words are ordered shortlex: by length, then by the caller's alphabet
 *     order (Sec. 2 shortlex; Example 1 and its figure put eps at index 0).
 *   - The search leaves are the alphabet symbols at cost c_sym (Alg. 1 seeds
 *     only them); eps and the empty set are returned only by the trivial
 *     cases (P empty -> the empty set, P = {eps} -> eps, both at cost c_sym).
 *   - Level c (c > c_sym) enumerates, in this order: r? for r in level
 *     c - c_?; r* for r in level c - c_*; l.r over splits cl + cr = c - c_.
 *     with cl ascending from c_sym, l outer and r inner; l + r likewise with
 *     c_+, restricted to cl <= cr and, when cl == cr, to l before r.  The
 *     first candidate with a language is the one kept; the first precise
 *     candidate is the answer.  Leaves are checked for precision too.
 *   - Memory: a language costs 4*W + 28 bytes, W the 32-bit words of a padded
 *     CS (1 for |ic| <= 32, 2 for |ic| <= 64, else 4*ceil(|ic|/128)); the
 *     cache holds at most cap = min(floor(mem_budget / (4*W + 28)),
 *     0x7FFF0000) languages.  A level whose new languages would exceed cap
 *     without yielding an answer ends the search with REI_OOM, or, with
 *     REI_F_ONTHEFLY, continues uncached while every operand level it needs
 *     is complete ("OnTheFly mode", Sec. 3).
 */
#ifndef REI_H
#define REI_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define REI_ABI_VERSION 2

#define REI_MAX_IC 4096      /* largest |ic(P u N)| */
#define REI_MAX_STRLEN 4095  /* longest example string */
#define REI_MAX_COST 255     /* largest max_cost */

typedef enum rei_status {
    REI_OK = 0,          /* a minimal precise expression was found */
    REI_NOT_FOUND = 1,   /* none with cost <= max_cost (Alg. 1 "not_found") */
    REI_OOM = 2,         /* the language cache reached its cap first */
    REI_EINVAL = 3,      /* invalid argument (see each call) */
    REI_EBUFSZ = 4,      /* an output buffer is too small; sizes written back */
    REI_ECUDA = 5,       /* a CUDA call failed */
    REI_ETIMEOUT = 6,    /* a bounded device wait or a server wait ran out */
    REI_EBUSY = 7,       /* server full / ticket not finished */
    REI_ESCRATCH = 8     /* the problem, or the cache its memory budget asks
                            for, is larger than rei_solve_noalloc's scratch */
} rei_status;

/* Cost homomorphism (c_sym, c_?, c_*, c_., c_+), Def. "cost function" (Sec. 3).
 * All constants must be >= 1. */
typedef struct rei_costs {
    uint32_t c_sym, c_opt, c_star, c_cat, c_alt;
} rei_costs;

/* One example string: `len` bytes at `ptr`, each byte a symbol. */
typedef struct rei_str {
    const uint8_t *ptr;
    uint32_t len;
} rei_str;

typedef struct rei_stats {
    uint64_t candidates;   /* candidates enumerated: all of the completed
                              levels, plus those up to and including the answer
                              in its level */
    uint64_t unique;       /* languages cached by the completed levels */
    uint32_t levels;       /* last cost level entered */
    uint32_t n_ic;         /* |ic(P u N)| */
    uint32_t words;        /* W, 32-bit words per stored CS */
    uint32_t max_len;      /* longest ic word */
    uint64_t guide_pairs;  /* sum over ic words w of |w| + 1 */
    double ms_stage;       /* staging (ic, guide table, masks, leaves) */
    double ms_total;       /* whole call, host clock */
    uint64_t launches;     /* kernels this call launched */
    uint64_t bytes_h2d;    /* host-to-device bytes this call copied */
    uint64_t bytes_d2h;    /* device-to-host bytes this call copied */
    uint64_t cand_op[5];   /* `candidates` split by outermost operator:
                              symbol, ?, *, concatenation, union */
    uint64_t star_pairs;   /* sum over ic words w != eps of |w| (the splits
                              a star evaluates per candidate) */
    double ms_search_kernel; /* device time of the search launches (CUDA events) */
    double ms_stage_kernel;  /* device time of the staging launch (CUDA events) */
    uint32_t search_launches; /* search-kernel launches (more than 1 when the
                                 cache grew) */
    uint32_t grid;           /* CTAs of the search launch */
} rei_stats;

/* Result of one solve; caller-owned.  `regex` receives the pretty string
 * (UTF-8; "ε" for eps, "∅" for the empty set; * and ? bind tighter than
 * concatenation, which binds tighter than +; only needed parentheses), NUL
 * terminated if it fits.  `tree` receives the expression in postfix order,
 * two bytes per node: ('a', symbol index) for a symbol, ('e', 0) eps,
 * ('0', 0) empty set, ('?', 0), ('*', 0), ('.', 0) concatenation, ('+', 0)
 * union.  Either buffer may be NULL with cap 0 to query the lengths. */
typedef struct rei_result {
    int32_t status;
    uint32_t cost;
    char *regex;
    size_t regex_cap;
    size_t regex_len;
    uint8_t *tree;
    size_t tree_cap;
    size_t tree_len;
    rei_stats stats;
} rei_result;

/* Optional device allocator.  alloc returns NULL on failure.  Both get the
 * context stream; the library frees everything it allocated before
 * rei_ctx_destroy returns. */
typedef struct rei_alloc {
    void *(*alloc)(void *user, size_t bytes, void *stream);
    void (*free)(void *user, void *ptr, size_t bytes, void *stream);
    void *user;
} rei_alloc;

#define REI_F_DEVICE_INPUT 1u  /* `bytes` and `offsets` are device pointers */
#define REI_F_ONTHEFLY 2u      /* OnTheFly mode after the cache fills */

/* One problem in packed form.  Strings are P first then N: string k is
 * bytes[offsets[k] .. offsets[k+1]) for k < n_pos + n_neg.  `alphabet` is
 * always host memory.  max_errors: allowed number of misclassified examples
 * ("REI with error", Sec. 6; 0 = precise). */
typedef struct rei_problem {
    const uint8_t *alphabet;
    uint32_t n_sym;
    const uint8_t *bytes;
    const uint32_t *offsets;
    uint32_t n_pos, n_neg;
    uint64_t total_bytes;  /* = offsets[n_pos + n_neg]; required with REI_F_DEVICE_INPUT */
    rei_costs costs;
    uint32_t max_cost;
    uint64_t mem_budget;
    uint32_t max_errors;
    uint32_t flags;
    /* Per-symbol costs (Sec. 3: a cost homomorphism may give different alphabet
     * symbols different costs): NULL = every symbol costs costs.c_sym; else
     * n_sym costs >= 1 in host memory, one per alphabet symbol in alphabet
     * order.  A level c starts with the symbols of cost c (alphabet order);
     * eps and the empty set keep costs.c_sym. */
    const uint32_t *sym_costs;
} rei_problem;

typedef struct rei_ctx rei_ctx;

/* Create a context on CUDA device `device`.  `alloc` may be NULL (then
 * cudaMallocAsync / cudaFreeAsync); `stream` is a cudaStream_t or NULL for a
 * stream the context creates.  Errors: REI_EINVAL (bad device), REI_ECUDA. */
rei_status rei_ctx_create(rei_ctx **out, int device, const rei_alloc *alloc, void *stream);

/* Release every device and host resource of the context. */
void rei_ctx_destroy(rei_ctx *ctx);

/* Tuning options (defaults chosen by the library):
 *   REI_OPT_CHUNK      candidates per dedup chunk (0 = automatic: up to
 *                      2^25, or 2^28 for |ic| <= 30 with exact keys;
 *                      larger values are taken as 2^26, or 2^28 for those);
 *                      the value only changes how a level is split into
 *                      chunks
 *   REI_OPT_GRID       CTAs of the search kernel (0 = all that fit)
 *   REI_OPT_KEEP_CACHE 1 = keep the cache after a solve for rei_cache_dump
 *   REI_OPT_CACHE_INIT initial cache capacity in languages (0 = automatic)
 *   REI_OPT_SOLO_TILES chunks of at most this many 32-candidate tiles run on
 *                      one CTA without grid-wide synchronisation (-1 =
 *                      automatic, 0 = never)
 *   REI_OPT_SMALL_ROWS languages the search keeps in one CTA's shared memory
 *                      at its start, with their uniqueness table (-1 =
 *                      automatic, 0 = never, else a power of two 256..16384;
 *                      shrunk until the launch keeps two CTAs per SM).
 *   REI_OPT_EXACT_KEYS 1 = for |ic| <= 62 the uniqueness table keys are the
 *                      languages themselves (no row comparisons; the
 *                      default), 0 = fingerprint and row keys always
 *   REI_OPT_HANDOVER   a level with more candidates than this leaves the
 *                      first (latency-shaped) launch for a relaunch shaped
 *                      for throughput (default 4 Mi; 0 = never)
 *   REI_OPT_YIELD_US   a batched or served problem still searching on its one
 *                      CTA after this many microseconds stops there and
 *                      continues from the levels it has cached, in its
 *                      slot on a group of CTAs beside the other such
 *                      problems (on the whole GPU once it outgrows its
 *                      slot) (default 500; 0 = never; rei_tune.yield_us,
 *                      when given, takes its place for a batch)
 *   REI_OPT_FUSED_STAGE 1 = stage a problem inside its search launch when the
 *                      launch can hold it (|ic| <= 2048, strings <= 8 KiB;
 *                      the default), 0 = always a separate staging launch.
 *                      Results never depend on any option. */
#define REI_OPT_CHUNK 1
#define REI_OPT_GRID 2
#define REI_OPT_KEEP_CACHE 3
#define REI_OPT_CACHE_INIT 4
#define REI_OPT_SOLO_TILES 5
#define REI_OPT_SMALL_ROWS 6
#define REI_OPT_FUSED_STAGE 7
#define REI_OPT_EXACT_KEYS 8
#define REI_OPT_HANDOVER 9
#define REI_OPT_YIELD_US 10
rei_status rei_ctx_set_option(rei_ctx *ctx, int option, int64_t value);

/* Number of kernels this context launched since it was created. */
uint64_t rei_ctx_launches(const rei_ctx *ctx);

/* Solve one problem given as string arrays in host memory (Alg. 1 over the
 * whole cost range).  Errors: REI_EINVAL when a cost is 0, n_sym is 0 or
 * > 256, the alphabet repeats a symbol, an example uses a byte outside the
 * alphabet, P and N share a string, max_cost > REI_MAX_COST, |ic| >
 * REI_MAX_IC or a string is longer than REI_MAX_STRLEN; REI_EBUFSZ when
 * out->regex or out->tree is too small (needed sizes written back);
 * REI_ECUDA.  The search outcome (REI_OK, REI_NOT_FOUND, REI_OOM) is both
 * returned and stored in out->status. */
rei_status rei_solve(rei_ctx *ctx, const uint8_t *alphabet, uint32_t n_sym, const rei_str *P,
                     uint32_t nP, const rei_str *N, uint32_t nN, rei_costs costs,
                     uint32_t max_cost, uint64_t mem_budget, rei_result *out);

/* Solve one packed problem; with REI_F_DEVICE_INPUT the example bytes and
 * offsets are read straight from device memory.  Errors as rei_solve. */
rei_status rei_solve_problem(rei_ctx *ctx, const rei_problem *prob, rei_result *out);

/* Staged form of a problem (Sec. 3 "Staging: guide table"), for inspection.
 * ic words in shortlex order as (word_start, word_len): word w is
 * bytes[word_start[w] .. + word_len[w]) of the packed example bytes (word 0
 * is eps, length 0).  gt_off[n_ic + 1] and gt_pair[G]: the splits of word w
 * are gt_pair[gt_off[w] .. gt_off[w+1]), each (u | v << 16) with u the
 * prefix and v the suffix, in order of the split position 0..|w|.
 * pos_mask / neg_mask: W words each; leaf: n_sym * W words, the CS of each
 * symbol.  Caller sets the capacities; on REI_EBUFSZ the needed n_ic,
 * guide_pairs and words are written back. */
typedef struct rei_staged {
    uint32_t n_ic, words, max_len;
    uint64_t guide_pairs;
    uint32_t *word_start, *word_len;  /* cap_words entries each */
    uint32_t *gt_off;                 /* cap_words + 1 */
    uint32_t *gt_pair;                /* cap_pairs */
    uint32_t *pos_mask, *neg_mask;    /* cap_w each */
    uint32_t *leaf;                   /* n_sym * cap_w */
    uint32_t cap_words, cap_pairs, cap_w;
} rei_staged;
rei_status rei_stage(rei_ctx *ctx, const rei_problem *prob, rei_staged *out);

/* Copy the language cache of the last solve (needs REI_OPT_KEEP_CACHE = 1):
 * for cached languages k < *count: cs[k*W .. k*W + W) (the CS words),
 * op[k] (0 symbol, 1 ?, 2 *, 3 ., 4 +), left[k], right[k] (operand cache
 * indices; left = symbol index for a symbol; right = 0xFFFFFFFF when unused),
 * and per cost c <= max_cost: level_start[c], level_count[c].  *count is the
 * capacity on entry and the number of cached languages on return. */
rei_status rei_cache_dump(rei_ctx *ctx, uint32_t *cs, uint8_t *op, uint32_t *left,
                          uint32_t *right, uint64_t *count, uint64_t *level_start,
                          uint64_t *level_count, uint32_t n_levels);

/* ---- batched form: many independent problems, one persistent launch ---- */

/* Shape and scheduling of the batched launch, in which each CTA solves one
 * problem at a time in its own memory slot.  A field left 0 is chosen by the
 * library: warps_per_cta and chunk by an autotuner that times the first parts
 * of a batch (samples of one problem per SM each) under a few settings and
 * keeps, for the context, the one with the most candidates per millisecond of
 * the whole call; yield_us from the context's REI_OPT_YIELD_US.  Results never
 * depend on any field.  NULL = every field 0.  A field out of range gives
 * REI_EINVAL. */
typedef struct rei_tune {
    uint32_t warps_per_cta; /* warps of each CTA: 1, 2, 4 or 8 */
    uint32_t chunk;         /* candidates per dedup chunk in a slot: 256 .. 65536 */
    uint32_t yield_us;      /* a problem still searching on its CTA after this
                               many microseconds continues from where it
                               stopped, in its slot on a group of CTAs beside
                               the other such problems, or on the whole GPU
                               once it outgrows its slot (0xFFFFFFFF = never) */
} rei_tune;

/* Solve n problems.  outs[i] receives problem i's result exactly as
 * rei_solve_problem would produce it.  Returns REI_OK when every problem was
 * processed (per-problem outcomes in outs[i].status) or the first error. */
rei_status rei_solve_batch(rei_ctx *ctx, const rei_problem *probs, uint32_t n, rei_result *outs,
                           const rei_tune *tune);

/* ---- served form: continuous batching of arriving problems ----
 *
 * Independent problems that arrive over time, each searched as in Alg. 1
 * (the paper solves one problem per run; serving many is this library's).
 * One persistent launch, one CTA per memory slot, takes problems from a ring
 * in mapped host memory as its CTAs free up; each CTA stages its problem
 * itself (Sec. 3 staging: infix closure, guide table, leaves) and searches
 * it alone.  A worker thread of the server admits queued problems into the
 * ring, reads answers back and relaunches the search when it returned after
 * going idle.  Problems with more than 255 strings or 8192 bytes, or whose
 * search outgrows a slot (2^17 languages, |ic| <= 2048), are solved alone by
 * rei_solve_problem while the launch is stopped; searches past their time
 * allowance (REI_OPT_YIELD_US) continue meanwhile in their slots, side by
 * side on groups of CTAs.  Every result equals
 * rei_solve_problem's for the problem alone.  The server owns its context's
 * device while it lives: make no other call
 * on that context until rei_server_destroy. */

typedef struct rei_server rei_server;

/* budget_bytes: device memory the live problems may hold together (each
 * problem is charged min(its mem_budget, one slot's cache) at admission; one
 * problem is always admitted when none is live); max_live: problems on the
 * device at once.  The server allocates its slots (about 38 MiB per slot, one
 * slot per resident CTA) from the context's allocator.  REI_OOM when that
 * fails, REI_ECUDA on a CUDA error. */
rei_status rei_server_create(rei_ctx *ctx, uint64_t budget_bytes, uint32_t max_live,
                             rei_server **out);

/* Queue a problem (inputs are copied; thread-safe).  *ticket identifies it. */
rei_status rei_server_submit(rei_server *srv, const rei_problem *prob, uint64_t *ticket);

/* Wait up to block_ms (0 = poll, < 0 = forever) for a ticket's result.
 * out->stats.ms_total is the time from submission to the answer.
 * REI_EBUSY when not finished in time; REI_EINVAL for a ticket that was not
 * issued or was already released; REI_EBUFSZ (ticket kept) when out's regex
 * or tree buffer is too small.  The ticket is released on success.  Once the
 * server's launch has failed (a CUDA error), every unanswered ticket and
 * every later submission get REI_ECUDA. */
rei_status rei_server_poll(rei_server *srv, uint64_t ticket, rei_result *out, int block_ms);

/* Stop the server's worker (finishing queued and live problems) and free it. */
void rei_server_destroy(rei_server *srv);

/* ---- solving without allocating ---- */

/* Size of the device array rei_solve_noalloc works in.  The array is a
 * file-scope device variable of the library: every GPU that loads the
 * library holds these bytes until the process exits. */
#define REI_NOALLOC_SCRATCH_BYTES (64u << 20)

/* Solve one problem exactly as rei_solve_problem would (same statuses, cost,
 * expression, candidate and unique counts), without allocating any memory.
 * The paper has no counterpart: this entry point exists for callers that
 * cannot allocate device memory while they solve -- code working inside
 * another framework's fixed memory arena, or a host thread that must not
 * enter the CUDA allocator (it can block on device-wide synchronisation) --
 * and it calls no cudaMalloc, cudaFree, pinned-host or other allocating
 * routine.  It needs no context: it runs on the current device and on
 * `stream` (a cudaStream_t; NULL for the default stream), and returns after
 * the stream has finished its work.
 *
 * Every piece of device scratch comes from one shared array of
 * REI_NOALLOC_SCRATCH_BYTES.  The first call on each device looks up the
 * array's device address (once per device).  Every call waits for its stream
 * partway through (it reads the staged sizes back) and copies through
 * pageable host memory, so no call may be made while its stream is being
 * captured into a CUDA graph.  The array keeps the previous call's contents;
 * each call clears on its stream what must start cleared.  Calls that overlap
 * on the GPU (other streams or host threads) race on the array: issue one at
 * a time.
 *
 * The whole language cache of the budget is resident: with W the 32-bit
 * words of a CS (see the memory rule above), cap = floor(mem_budget /
 * (4*W + 28)) languages must fit, with their uniqueness table and a chunk
 * workspace, in what the staged problem leaves of the array (about 61 MiB;
 * e.g. cap up to about 1.3 million languages at W = 2).  Example bytes are
 * limited to 1 MiB, examples to 65535 and guide-table pairs to 262144.  A
 * problem beyond these limits returns REI_ESCRATCH (nothing is truncated);
 * other errors as rei_solve_problem (the argument rules are the same; a
 * failed CUDA call gives REI_ECUDA in both the return value and
 * out->status).  A regex buffer too small for the answer receives its first
 * regex_cap - 1 bytes and a terminating NUL, with REI_EBUFSZ returned and
 * out->regex_len set to the full length. */
rei_status rei_solve_noalloc(const rei_problem *prob, void *stream, rei_result *out);

#ifdef __cplusplus
}
#endif

#endif /* REI_H */
