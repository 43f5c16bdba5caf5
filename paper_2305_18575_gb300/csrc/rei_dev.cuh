// rei_dev.cuh -- device-side data structures of the REI library (internal).
//
// Layout in HBM for one problem:
//   staging   : word_start/word_len[n], len_start[max_len+2], gt_off[n+1],
//               gt_pair[G] (u | v << 16), pos/neg masks [W], leaf[n_sym][W]
//   cache     : cs[cache_alloc][W] (row per language, write-once, cost order),
//               bp_op[]/bp_l[]/bp_r[] back-pointers
//   dedup     : table[2^k] of u64 slots = (fingerprint << 32) | index, where
//               index < 2^31 is a cache row and PENDING|j marks chunk-local
//               candidate j whose CS sits in tmp[j][W] until compaction
//   chunk     : tmp[chunk][W], pending[chunk] (new slots), slotpos[chunk],
//               bitmap[chunk/32] (survivors), blk[grid] (per-CTA counts)
//   state     : SolveState (level, chunk position, counts, barrier, answer)
#pragma once
#include <cstdint>

#include "../../include/rei.h"

namespace rei {

constexpr uint32_t kMaxIC = REI_MAX_IC;
constexpr uint32_t kMaxWords = (REI_MAX_IC + 31) / 32;
constexpr uint32_t kMaxCost = REI_MAX_COST;
constexpr uint64_t kEmpty = ~0ull;
constexpr uint32_t kPending = 0x80000000u;
constexpr uint32_t kMaxTeam = 2047;  // CTAs of a plain search launch at most (the ordered append's prefix table)
constexpr uint32_t kNoRight = 0xFFFFFFFFu;
constexpr uint32_t kNoOperand = 0xFFFFFFFFu;  // no cache row (rows are < 2^31)
constexpr unsigned long long kNone = ~0ull;
constexpr uint32_t kSeenBits = 30;   // largest |ic| with a bitmap of cached languages (2^30 bits = 128 MiB)
constexpr uint32_t kDirectBits = 26; // largest |ic| whose table has a slot per language (2^26 x 12 bytes)

// operators of a cache entry / candidate
enum Op : uint32_t { OP_LEAF = 0, OP_OPT = 1, OP_STAR = 2, OP_CAT = 3, OP_ALT = 4 };

// device status codes (internal; mapped to rei_status by the host)
enum DevStatus : uint32_t {
    ST_RUNNING = 0,
    ST_FOUND = 1,
    ST_NOT_FOUND = 2,
    ST_OOM = 3,
    ST_NEED_MEM = 4,
    ST_TIMEOUT = 5,
    ST_BAD = 6,
    ST_RESTAGE = 7,  // staged in the search launch, but the launch cannot hold the problem
};

// staging error codes
enum StageErr : uint32_t {
    SE_OK = 0,
    SE_SYMBOL = 1,     // a byte outside the alphabet
    SE_OVERLAP = 2,    // P and N share a string
    SE_IC_LARGE = 3,   // |ic| > REI_MAX_IC
    SE_STRLEN = 4,     // a string longer than REI_MAX_STRLEN
    SE_PAIRS = 5,      // guide table larger than the pair buffer (retry bigger)
    SE_OFFSETS = 6,    // offsets do not start at 0, decrease, or end elsewhere than total_bytes
    SE_INTERNAL = 7,   // an infix lookup failed (never expected)
};

// words of a padded CS (32-bit units): 1, 2, or a multiple of 4
__host__ __device__ inline uint32_t padded_words(uint32_t n) {
    return n <= 32 ? 1u : n <= 64 ? 2u : 4u * ((n + 127u) / 128u);
}

struct StageInfo {
    uint32_t status;      // StageErr
    uint32_t n;           // |ic|
    uint32_t W;           // padded words
    uint32_t max_len;
    uint32_t G;           // guide pairs
    uint32_t n_pos_set;   // distinct positive examples
    uint32_t n_neg_set;
    uint32_t pos_eps;     // eps in P
    uint32_t neg_eps;     // eps in N
    uint32_t pad[7];
};

struct StageJob {
    // inputs (device)
    const uint8_t *bytes;
    const uint32_t *offs;
    uint32_t n_pos, n_neg;
    uint8_t alphabet[256];
    uint32_t n_sym;
    uint32_t total_bytes;             // = offs[n_pos + n_neg], checked on the device
    // outputs (device)
    StageInfo *info;
    uint32_t *word_start, *word_len;  // kMaxIC
    uint32_t *len_start;              // REI_MAX_STRLEN + 2
    uint32_t *gt_off;                 // kMaxIC + 1
    uint32_t *gt_pair;                // pair_cap
    uint32_t pair_cap;
    uint32_t *pos_mask, *neg_mask;    // kMaxWords
    uint32_t *leaf;                   // n_sym * kMaxWords (row stride kMaxWords)
};

// one segment of a level's enumeration (level-local index space)
struct Seg {
    uint64_t start;     // first level-local index
    uint64_t size;      // indices covered (binary ops: lcnt * rcnt)
    uint32_t op;
    uint32_t tri;       // union with cl == cr: only l < r is a candidate
    uint32_t lbase, lcnt, rbase, rcnt;
    uint32_t swap;      // concatenation tiled over 32 left operands (few right ones)
    uint32_t pad;
};

// words of a published chunk plan: nseg, tiles, then the segments, their
// tiles in the chunk and the first tile of each (nseg + 1)
__host__ __device__ inline size_t plan_words(uint32_t seg_cap) {
    return 2 + (size_t)seg_cap * ((sizeof(Seg) + sizeof(uint64_t) * 5) / 8 + 1) + 1;
}

struct SolveState {
    uint32_t status;          // DevStatus
    uint32_t level;           // current cost level
    uint64_t chunk_pos;       // next level-local index to process
    uint32_t size;            // cached languages
    uint32_t full;            // cache cap reached in this level
    uint32_t otf;             // OnTheFly mode
    uint32_t partial_level;   // first level not completely cached
    unsigned long long found; // level-local index of the answer, or kNone
    uint32_t pending_count;
    uint32_t ans_op, ans_l, ans_r, ans_cost;
    uint32_t tree_len;        // postfix tokens written
    uint64_t candidates;      // completed levels
    uint64_t unique_done;     // languages of completed levels
    uint64_t level_total;     // index-space size of the current level
    uint32_t err;             // barrier / bounds error detail
    uint32_t need_rows;       // NEED_MEM: cache rows wanted
    uint64_t cand_op[5];      // candidates by operator (completed levels + answer prefix)
    unsigned long long bar_arrive;  // grid-barrier arrivals of this launch
    uint32_t dbg_cta, dbg_epoch, dbg_site, dbg_seen;  // where a barrier wait ran out
    uint32_t nseg;
    // command from CTA 0 to the other CTAs, and the chunk it describes
    uint32_t cmd, cmd_seq;
    uint32_t c_level, c_size, c_dedup;
    uint64_t c_cs0, c_ce0;
    // CTA 0's wall time (ns) in: planning, chunks alone, chunks with the grid,
    // level ends; and how many solo chunks, team chunks, levels
    uint64_t t_phase[4];
    uint64_t n_phase[3];
    uint64_t t_sub[48];  // steps of CTA 0's chunks and launch (timing builds only)
    uint32_t tile_next;  // the next tile of a team chunk handed out dynamically
    uint32_t pad;
    // the fused launch that owns this state: CTA 0 resets the state, stages,
    // then writes its launch id here; the other CTAs start once it names theirs
    unsigned long long launch;
};

struct SolveJob {
    // staged problem
    uint32_t n, W, G, n_sym, max_len;
    const uint32_t *gt_off, *gt_pair, *len_start;
    const uint32_t *pos_mask, *neg_mask, *leaf;  // leaf row stride = leaf_stride
    uint32_t leaf_stride;
    uint32_t n_pos_set, pos_eps, neg_eps;
    uint32_t c[5];
    uint32_t max_cost, max_errors, flags;
    uint64_t cap;  // budget cap in languages
    // cache
    uint32_t *cs;
    uint8_t *bp_op;
    uint32_t *bp_l, *bp_r;
    uint32_t *used;  // table slot of every cached row (to clear the table after the search)
    uint64_t cache_alloc;
    unsigned long long *table;
    uint64_t table_mask;
    // chunk workspace
    uint32_t *tmp, *pending, *slotpos, *bitmap, *blk;
    uint64_t chunk_max;
    // bookkeeping
    int64_t *lvl_start, *lvl_count;  // max_cost + 1 entries
    uint64_t *plan;                  // a team chunk's plan as CTA 0 publishes it (plan_words(seg_cap)); null: every CTA plans
    uint32_t seg_cap;
    SolveState *st;
    uint8_t *tree;                   // 2 * (max_cost + 1) bytes
    uint32_t *tstack;                // 4 * (max_cost + 2) words: answer-walk stack
    uint32_t *trace;                 // per CTA: (barriers passed << 8) | last barrier site
    uint32_t gt_in_smem;             // guide table copied to shared memory
    uint32_t solo_tiles;             // chunks of at most this many tiles run on CTA 0 alone
    uint32_t small_rows;             // languages CTA 0 keeps in shared memory at the start (0 = none)
    // exact keys (|ic| <= 62, W <= 2): a table slot holds the language itself
    // (bit 63: added in the current chunk), minidx[slot] the first candidate
    // of the chunk with that language; 0 = fingerprint | row slots
    uint32_t exact;
    uint32_t *minidx;
    // 1-word languages (|ic| <= kSeenBits, exact keys): bit L of seen[] is set
    // once language L is cached, so that a candidate whose language is already
    // cached is told by one bit instead of a table probe; nullptr = none.  All
    // zero between searches (a search clears the words of the rows it cached).
    uint32_t *seen;
    // exact keys with a table of at least 2^|ic| slots: the slot of a
    // language is the language itself (no hash, never a second probe)
    uint32_t direct, direct_pad;
    // leaves: the alphabet symbols ordered by (cost, alphabet order) and
    // their costs (every symbol costs c[0] unless costs are given per
    // symbol; a cost above REI_MAX_COST is stored as REI_MAX_COST + 1);
    // cmin is the cheapest, below which no expression costs
    uint32_t cmin, leaf_pad;
    uint64_t handover;  // levels above this many candidates end the launch (0 = never)
    // a search on one CTA of the batched or served form gives up (and is
    // solved again on the whole GPU) after yield_ns from t_start (0 = never)
    uint64_t yield_ns, t_start;
    // the CTAs that search this problem: team_size of them from team_base on
    // (0, 0: every CTA of the launch); the first of them leads
    uint32_t team_base, team_size;
    uint16_t leaf_cost[256];
    uint8_t leaf_sym[256];
};

static_assert(sizeof(SolveJob) % 8 == 0, "the job is copied in 8-byte words");

// the search launch that stages its problem first (CTA 0), then searches it
struct FuseArgs {
    StageJob sj;              // inputs, and where the staged problem goes
    SolveJob tmpl;            // the job without the staged sizes and what depends on them
    SolveJob *job;            // global: the completed job, for every CTA
    uint64_t mem_budget;
    uint64_t rows_alloc;      // rows of the back-pointer arrays
    uint64_t cs_words, tmp_words, pend_cap, table_slots;
    uint64_t chunk_opt;       // chunk size asked for (0 = automatic)
    uint32_t small_opt;       // languages in shared memory at the start: 0xFFFFFFFF automatic, 0 none
    uint64_t handover;        // levels above this many candidates go to the relaunch (0 = never)
    uint32_t smem_cap;        // dynamic shared memory of the launch
    uint32_t seen_bits;       // the seen bitmap covers languages of up to this many bits (0 = none)
    uint32_t *seen;           // 2^seen_bits bits, all zero
    unsigned long long launch_id;  // larger than any id the state buffer can hold
    // where CTA 0 writes the final state, the answer's tokens and the staging
    // report (out_words 8-byte words, the state buffer's layout) for the host,
    // in mapped pinned memory; null: the host copies them itself
    unsigned long long *host_out;
    uint64_t out_words;
};


// ---- batched search

// memory of the batch launch's slots (one per CTA), each `rows` cache rows
struct SlotMem {
    uint32_t *cs;            // slots * cs_words
    uint8_t *bp_op;          // slots * rows
    uint32_t *bp_l, *bp_r;   // slots * rows
    uint32_t *used;          // slots * rows
    unsigned long long *table;  // slots * table_slots
    uint32_t *tmp;           // slots * tmp_words
    uint32_t *pending, *slotpos;  // slots * chunk
    uint32_t *bitmap;        // slots * ceil(chunk / 32)
    uint32_t *blk;           // slots
    int64_t *lvl;            // slots * 2 * (kMaxCost + 2)
    SolveState *state;       // slots
    uint32_t *tstack;        // slots * 4 * (kMaxCost + 2)
    uint64_t rows, cs_words, table_slots, tmp_words, chunk;
};

// what one batched solve reports (device side)
struct BatchOut {
    uint32_t status, cost, tree_len, levels;
    uint64_t candidates, unique;
    uint64_t cand_op[5];
    uint64_t ns;
    // ST_NEED_MEM from the search: the memory slot that still holds its
    // cache, uniqueness table, level table and state (the CTA took no more
    // work), so that the search continues from there; kNoSlot = not searched
    // here.  need_rows: the cache rows the search asked for (0: it stopped at
    // its time allowance, and fits its slot)
    uint32_t slot, need_rows;
};
constexpr uint32_t kNoSlot = 0xFFFFFFFFu;

// one problem of a batch: its job (staged data, costs; memory fields are
// filled in by the CTA that takes it), where its tree and report go
struct BatchJob {
    SolveJob job;
    uint8_t *tree;
    BatchOut *out;
};

// searches a batch left in their slots at their time allowance, continued
// side by side in one launch: group g (group_ctas CTAs from g * group_ctas on)
// continues problem prob[g] in slot slot[g], in the slot's memory
struct GroupArgs {
    SlotMem slot;
    const uint32_t *prob, *slot_of;  // per group
    uint32_t groups, group_ctas;
    uint32_t *blk;                   // groups * group_ctas
    uint64_t *plan;                  // groups * plan_stride words
    uint64_t plan_stride;
    // chunk workspace of each group (larger chunks than a slot's): `chunk`
    // candidates, tmp_words words of candidate rows; the bitmaps start zeroed
    uint32_t *tmp, *pending, *slotpos, *bitmap;
    uint64_t chunk, tmp_words;
};

struct BatchArgs {
    SlotMem slot;
    uint32_t n;        // problems
    uint32_t *queue;   // next problem to take
    uint64_t yield_ns; // a problem still searching after this long goes back to the host (0 = never)
};

// ---- served search

constexpr uint32_t kServeMaxStrings = 255;   // examples per served request
constexpr uint32_t kServeMaxBytes = 8192;    // example bytes per served request
constexpr uint32_t kServeMaxIC = 2048;       // |ic| of a request a server CTA stages and solves
constexpr uint32_t kServePairCap = 1u << 16; // guide pairs a served request may stage

// a request in the ring (mapped host memory), written before it is published
struct ServeReq {
    unsigned long long seq;        // job + 1, written by the host after every other field
    uint32_t n_pos, n_neg, n_sym, total_bytes;
    uint8_t alphabet[256];
    rei_costs costs;
    uint32_t max_cost, max_errors, flags;
    uint64_t mem_budget;
    uint32_t cmin;                 // leaves, as in SolveJob
    uint16_t leaf_cost[256];
    uint8_t leaf_sym[256];
    uint32_t offs[kServeMaxStrings + 1];
    uint8_t bytes[kServeMaxBytes];
};

// a result in the ring (mapped host memory); `done` = job + 1 once written
struct ServeOut {
    unsigned long long done;
    BatchOut out;
    StageInfo info;
    uint8_t tree[2 * (REI_MAX_COST + 1)];
};

struct ServeArgs {
    SlotMem slot;
    // per slot: the request's offsets, staged problem
    uint32_t *in_offs;
    uint32_t *word_start, *word_len, *len_start, *gt_off, *gt_pair, *pos, *neg, *leaf;
    uint32_t pair_cap;
    StageInfo *sinfo;
    // the ring and its control words
    const ServeReq *ring;
    ServeOut *outs;
    uint32_t ring_size;
    const volatile unsigned long long *avail;  // jobs published (mapped)
    const volatile unsigned long long *stop;   // nonzero: return (mapped)
    uint64_t yield_ns;  // as BatchArgs::yield_ns
    unsigned long long *head;                  // next job to claim (device); head[1]: entries
                                               // found incomplete when first read, head[2]: given up
    unsigned long long idle_ns;
    size_t smem_cap;
    // per slot: the job of a request whose search parked there (its time
    // allowance ran out or it outgrew the slot), for its continuation
    BatchJob *parked;
};

}  // namespace rei
