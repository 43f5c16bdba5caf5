// solve.cu -- the cost-ordered search of one REI problem (Alg. 1, Alg. 2).
//
// One persistent launch per problem (cooperative: every CTA is resident, so
// the grid barrier below cannot deadlock; each of its waits is bounded and
// ends the launch with ST_TIMEOUT instead of hanging).  The device plans every
// cost level from the level sizes it has itself produced, so a whole search
// needs no host round trip unless the cache must grow (ST_NEED_MEM, resumable
// at the same chunk).
//
// A level c is the concatenation of segments (Alg. 1 order): r? over level
// c - c_?, r* over level c - c_*, l.r over splits cl + cr = c - c_. (cl
// ascending, l outer, r inner), l + r over splits of c - c_+ with cl <= cr
// (l < r when cl == cr).  It is processed in chunks of consecutive candidates:
//   A  build every candidate's CS (warp tiles of 32 candidates), test
//      precision (Def. "specification"; atomicMin keeps the first precise
//      index), and insert it into the uniqueness table ("Uniqueness
//      checking"): a slot holds the lowest chunk index of its language, so the
//      first candidate in order survives;
//   B  mark each new language's survivor in a bitmap;
//   C  count survivors per CTA;
//   D  append survivors in order to the cache with back-pointers (the
//      temporary storage -> language cache copy of Sec. 3, "GPU language
//      cache implementation"), and make their table slots point at the cache.
#include <cstdint>
#include <cstddef>
#include <map>
#include <mutex>
#include <tuple>

#include "rei_dev.cuh"
#include "stage_dev.cuh"

namespace rei {

constexpr long long kSpinLimit = 100000000;             // polls of a grid barrier, at most
constexpr unsigned long long kBarrierWaitNs = 2000000000ull;  // a grid barrier gives up after 2 s
#ifndef REI_BAR_NAP
#define REI_BAR_NAP 32  // ns between polls of a grid barrier
#endif
#ifndef REI_CMD_NAP
#define REI_CMD_NAP 256  // longest back-off (ns) of an idle CTA between polls for work
#endif

// ---------------------------------------------------------------------------
// memory helpers: data written during the launch by other CTAs is read through
// L2 (ld.cg / acquire), never from a possibly stale L1 line.

__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long *p) {
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ uint32_t ldcg(const uint32_t *p) { return __ldcg(p); }

// strong (coherent) loads of control words written by other CTAs
__device__ __forceinline__ uint32_t ld_relaxed_u32(const uint32_t *p) {
    uint32_t v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ unsigned long long ld_relaxed_u64(const void *p) {
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ uint64_t umin64(uint64_t a, uint64_t b) { return a < b ? a : b; }

__device__ __forceinline__ unsigned long long globaltimer_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}

// ---------------------------------------------------------------------------
// bounded grid barrier: a monotonic 64-bit arrival counter (never reset during
// a launch); barrier number e of a launch completes when the counter reaches
// e times the team's CTAs.  A wait that runs out records where it gave up,
// marks the search ST_TIMEOUT and returns false so every CTA of the team
// leaves the kernel.

// the CTAs that search a problem (SolveJob::team_base/team_size; 0 = the
// whole launch) and this CTA's rank among them; rank 0 leads
__device__ __forceinline__ uint32_t team_size_of(const SolveJob &J) { return J.team_size ? J.team_size : gridDim.x; }
__device__ __forceinline__ uint32_t team_rank_of(const SolveJob &J) { return blockIdx.x - J.team_base; }

__device__ bool grid_barrier(SolveState *st, uint32_t &epoch, uint32_t site, uint32_t *trace, uint32_t team_n,
                             uint32_t team_r) {
    __shared__ int s_ok;
    // the CTA's threads have finished their global writes and reductions
    // (atomicMin of the answer, atomicOr of survivors, table and cache stores)
    // when they pass __syncthreads; thread 0's fence then orders all of them
    // (the barrier makes them visible to it) before its arrival, and its fence
    // after the wait orders what the other CTAs wrote before every thread's
    // later reads (the same pattern as a cooperative-groups grid sync)
    __syncthreads();
    epoch++;
    if (threadIdx.x == 0) {
        int ok = 1;
        const unsigned long long target = (unsigned long long)epoch * team_n;
        __threadfence();
        atomicAdd(&st->bar_arrive, 1ull);
        unsigned long long seen;
        long long spins = 0;
        const unsigned long long t0 = globaltimer_ns();
        while ((seen = ld_acquire_u64(&st->bar_arrive)) < target) {
            if (REI_BAR_NAP) __nanosleep(REI_BAR_NAP);
            if (++spins > kSpinLimit || globaltimer_ns() - t0 > kBarrierWaitNs) {
                ok = 0;
                break;
            }
        }
        __threadfence();
        if (trace) trace[team_r] = (epoch << 8) | site;
        if (!ok) {
            if (atomicCAS(&st->err, 0u, 1u) == 0u) {
                st->dbg_cta = team_r;
                st->dbg_epoch = epoch;
                st->dbg_site = site;
                st->dbg_seen = (uint32_t)seen;
            }
            atomicExch(&st->status, (uint32_t)ST_TIMEOUT);
        }
        if (ld_relaxed_u32(&st->err)) ok = 0;
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// ---------------------------------------------------------------------------
// 32 x 32 bit transpose across a warp: lane j holds row j (bit t = M[j][t]);
// returns column `lane` (bit j = M[j][lane]).  Five butterfly stages.

__device__ __forceinline__ uint32_t transpose32(uint32_t x, uint32_t lane) {
#pragma unroll
    for (int s = 16; s >= 1; s >>= 1) {
        const uint32_t m = s == 16 ? 0x0000FFFFu : s == 8 ? 0x00FF00FFu : s == 4 ? 0x0F0F0F0Fu
                         : s == 2  ? 0x33333333u : 0x55555555u;
        const uint32_t o = __shfl_xor_sync(0xFFFFFFFFu, x, s);
        x = (lane & s) ? ((x & ~m) | ((o & ~m) >> s)) : ((x & m) | ((o & m) << s));
    }
    return x;
}

// ---------------------------------------------------------------------------
// hashing of a CS (W words)

__device__ __forceinline__ uint64_t cs_hash(const uint32_t *c, uint32_t W, uint32_t stride) {
    uint64_t h = 0x243F6A8885A308D3ull;
    for (uint32_t b = 0; b < W; b++) {
        h ^= c[b * stride];
        h *= 0x9E3779B97F4A7C15ull;
        h ^= h >> 32;
    }
    h ^= h >> 29;
    h *= 0xBF58476D1CE4E5B9ull;
    h ^= h >> 32;
    return h;
}

// ---------------------------------------------------------------------------
// per-CTA shared-memory view

// tiling of one segment inside the current chunk (segment-local indices)
struct SegTile {
    uint64_t lo, hi;  // chunk intersected with the segment
    uint64_t r0;      // first row (binary ops)
    uint32_t nb;      // column blocks per row, or row blocks per column (swapped)
    uint32_t nb_mul;  // x / nb = (umulhi(nb_mul, x) + x) >> nb_shift for x < 2^31
    uint32_t nb_shift, pad;
};

// Division by a divisor fixed for many dividends (Granlund and Montgomery,
// "Division by invariant integers using multiplication", 1994, the round-up
// method with a 33-bit multiplier 2^32 + m): for 1 <= d < 2^31 and x < 2^31,
// x / d = (umulhi(m, x) + x) >> l with l = ceil(log2 d) and
// m = floor(2^32 (2^l - d) / d) + 1.
__host__ __device__ inline void div_magic(uint32_t d, uint32_t &m, uint32_t &l) {
    l = 0;
    while ((1ull << l) < d) l++;
    m = (uint32_t)((((1ull << l) - d) << 32) / d + 1);
}

__device__ __forceinline__ uint32_t div_by(uint32_t x, uint32_t m, uint32_t l) {
    return (__umulhi(m, x) + x) >> l;
}

// per-warp shared memory (32-bit words): the shared operand's words, two
// 32-candidate tiles (candidate-major and bit-sliced); for 1-word languages
// also the nibble tables of the concatenation's shared operand and its id
constexpr uint32_t kW1Tab = 128;   // 8 nibble tables of 16 words
constexpr uint32_t kW1TabAt = 68;  // their offset (4 + 2 * 32 words; 16-byte aligned)
// candidates per tile of a concatenation or union segment: 32 (one per lane),
// or for 1-word languages 32 * kW1Per (kW1Per per lane, built side by side)
constexpr uint32_t kW1Per = 4;
__host__ __device__ inline uint32_t bin_block(uint32_t W) { return W == 1 ? 32u * kW1Per : 32u; }

__host__ __device__ inline uint32_t warp_words(uint32_t W) {
    const uint32_t Ws = (W & 1u) ? W : W + 1;
    const uint32_t base = ((W + 3) & ~3u) + 2 * 32 * Ws;
    return W == 1 ? kW1TabAt + kW1Tab + 4 : base;
}

struct Shared {
    Seg *seg;                // level plan
    uint64_t *tile_first;    // first tile of each segment in the current chunk (nseg + 1)
    SegTile *tiles;          // per segment
    uint32_t *pos, *neg;     // precision masks (W words)
    const uint32_t *gt_off, *gt_pair, *len_start;
    unsigned long long *sortbuf;  // kSortMax words: a small chunk's slot entries, or the append's per-CTA prefix and survivor list
    uint32_t *solo_bits;     // kSortMax / 32 words: candidates of a small chunk that hold a slot
    uint32_t *solo_pref;     // kSortMax / 32 + 4 words: survivors before each bitmap word, total
    // the search's start, while every language fits in CTA 0's shared memory
    uint32_t *sm_rows;       // small_rows rows of W words: the cached languages
    uint32_t *sm_table;      // 2 * small_rows slots: fp (15 bits) | pending | row or candidate
    uint32_t *sm_tmp;        // kSortMax rows: the candidates of the current chunk
    uint32_t *lvs, *lvc;     // level table (start, count per cost), mirrored in shared memory
    uint32_t *warp_mem;      // per warp: lw[W], A[32*Ws], B[32*Ws]
    uint32_t warp_words;
};

// the search state CTA 0 keeps in shared memory while it leads; written back
// to the global SolveState when the launch ends
struct Lead {
    uint32_t status, level, size, full, otf, partial_level;
    uint32_t smode;  // languages and their uniqueness table live in shared memory
    // the answer was found and the other CTAs were told to empty the table
    // (rows and pending slots given) while the leader writes out the answer
    uint32_t cleaned, clean_rows, clean_pend;
    uint64_t chunk_pos, candidates, unique_done;
    uint64_t cand_op[5];
};

struct Plan {
    uint32_t nseg;
    uint64_t total;          // index-space size of the level
};

// inclusive warp scan of 64-bit values
__device__ __forceinline__ uint64_t warp_incl_scan(uint64_t v, uint32_t lane) {
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const uint64_t y = __shfl_up_sync(0xFFFFFFFFu, v, d);
        if (lane >= (uint32_t)d) v += y;
    }
    return v;
}

// Alg. 1 order for level c; only segments with candidates are kept.  Run by
// one whole warp: lane k describes candidate segment k of each round of 32,
// the non-empty ones are compacted with a ballot and their starts are a warp
// scan of the sizes.
__device__ void plan_level(const SolveJob &J, uint32_t c, const uint32_t *lvs, const uint32_t *lvc, Seg *seg,
                           Plan &P) {
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t c1 = J.cmin;  // no expression is cheaper
    uint32_t ns = 0;
    uint64_t start = 0;
    // the symbols of cost c: entries [lo, hi) of the cost-ordered leaf table
    uint32_t lo = 0, hi = 0;
    for (uint32_t a = lane; a < J.n_sym; a += 32) {
        lo += J.leaf_cost[a] < c;
        hi += J.leaf_cost[a] <= c;
    }
    for (int d = 16; d > 0; d >>= 1) {
        lo += __shfl_xor_sync(0xFFFFFFFFu, lo, d);
        hi += __shfl_xor_sync(0xFFFFFFFFu, hi, d);
    }
    // candidate segments: [0] symbols, [1] ?, [2] *, then concatenation
    // splits, then union splits
    const int rem_c = (int)c - (int)J.c[3], rem_u = (int)c - (int)J.c[4];
    const int ncat = rem_c >= 2 * (int)c1 ? rem_c - 2 * (int)c1 + 1 : 0;
    const int nalt = rem_u >= 2 * (int)c1 ? rem_u / 2 - (int)c1 + 1 : 0;
    const int total = 3 + ncat + nalt;

    for (int r0 = 0; r0 < total; r0 += 32) {
        const int k = r0 + (int)lane;
        Seg s{};
        uint64_t size = 0;
        if (k < total) {
            if (k == 0) {
                s.op = OP_LEAF;
                s.lbase = lo;
                s.lcnt = hi - lo;
                size = hi - lo;
            } else if (k < 3) {
                const uint32_t d = J.c[k];
                if (c >= c1 + d) {
                    s.op = k == 1 ? OP_OPT : OP_STAR;
                    s.lbase = lvs[c - d];
                    s.lcnt = lvc[c - d];
                    size = s.lcnt;
                }
            } else if (k < 3 + ncat) {
                const uint32_t cl = c1 + (uint32_t)(k - 3), cr = (uint32_t)rem_c - cl;
                s.op = OP_CAT;
                s.lbase = lvs[cl];
                s.lcnt = lvc[cl];
                s.rbase = lvs[cr];
                s.rcnt = lvc[cr];
                size = (uint64_t)s.lcnt * s.rcnt;
                // tiles of 32 right operands per left one, or (swapped) of 32
                // left operands per right one: whichever needs fewer tiles
                // (fewer partly empty tiles)
                const uint32_t bw = bin_block(J.W);
                uint64_t t_rows = (uint64_t)s.lcnt * ((s.rcnt + bw - 1) / bw);
                uint64_t t_cols = (uint64_t)s.rcnt * ((s.lcnt + bw - 1) / bw);
                if (J.W == 1) {
                    // (and the lookup tables of each shared operand, about
                    // one and a half tiles' work each)
                    t_rows += s.lcnt + s.lcnt / 2;
                    t_cols += s.rcnt + s.rcnt / 2;
                }
                s.swap = t_cols < t_rows ? 1u : 0u;
            } else {
                const uint32_t cl = c1 + (uint32_t)(k - 3 - ncat), cr = (uint32_t)rem_u - cl;
                s.op = OP_ALT;
                s.tri = cl == cr;
                s.lbase = lvs[cl];
                s.lcnt = lvc[cl];
                s.rbase = lvs[cr];
                s.rcnt = lvc[cr];
                size = (s.tri && s.lcnt < 2) ? 0 : (uint64_t)s.lcnt * s.rcnt;
            }
        }
        const bool keep = size > 0;
        const uint32_t mask = __ballot_sync(0xFFFFFFFFu, keep);
        const uint64_t incl = warp_incl_scan(size, lane);
        if (keep) {
            s.size = size;
            s.start = start + incl - size;
            seg[ns + __popc(mask & ((1u << lane) - 1))] = s;
        }
        ns += __popc(mask);
        start += __shfl_sync(0xFFFFFFFFu, incl, 31);
    }
    if (lane == 0) {
        P.nseg = ns;
        P.total = start;
    }
    __syncwarp();
}

// candidates that are real (the triangle of a cl == cr union) among local
// indices 0..x of a segment
__device__ __forceinline__ uint64_t valid_upto(const Seg &s, uint64_t x) {
    if (s.op != OP_ALT || !s.tri) return x + 1;
    const uint64_t m = s.rcnt, row = x / m, col = x % m;
    return row * (m - 1) - row * (row - 1) / 2 + (col > row ? col - row : 0);
}

__device__ __forceinline__ uint64_t valid_count(const Seg &s) {
    if (s.op == OP_ALT && s.tri) return (uint64_t)s.lcnt * (s.lcnt - 1) / 2;
    return s.size;
}

// the highest operand level a level refers to (OnTheFly feasibility)
__device__ int max_operand_level(const SolveJob &J, int c) {
    const int c1 = (int)J.cmin;
    int m = -1;
    if (c - (int)J.c[1] >= c1) m = max(m, c - (int)J.c[1]);
    if (c - (int)J.c[2] >= c1) m = max(m, c - (int)J.c[2]);
    if (c - (int)J.c[3] >= 2 * c1) m = max(m, c - (int)J.c[3] - c1);
    if (c - (int)J.c[4] >= 2 * c1) m = max(m, c - (int)J.c[4] - c1);
    return m;
}

// ---------------------------------------------------------------------------
// phase A: one warp tile of up to 32 candidates

// step timing of CTA 0's chunks alone, compiled in with -DREI_TIMING only
#ifdef REI_TIMING
#define REI_TMARK(cond, k)                                          \
    do {                                                            \
        if ((cond) && threadIdx.x == 0) {                           \
            const unsigned long long t_now = globaltimer_ns();      \
            st->t_sub[k] += t_now - t_mark;                         \
            t_mark = t_now;                                         \
        }                                                           \
    } while (0)
#define REI_TSTART() const unsigned long long t_mark0 = globaltimer_ns(); unsigned long long t_mark = t_mark0
// a span of CTA 0's thread 0, added to t_sub[k]
#define REI_TSPAN_BEGIN(v) const unsigned long long v = globaltimer_ns()
#define REI_TSPAN_END(st_, v, k)                                                                   \
    do {                                                                                           \
        if (blockIdx.x == 0 && threadIdx.x == 0) (st_)->t_sub[k] += globaltimer_ns() - (v); \
    } while (0)
#else
#define REI_TSPAN_BEGIN(v) \
    do {                   \
    } while (0)
#define REI_TSPAN_END(st_, v, k) \
    do {                         \
    } while (0)
#define REI_TMARK(cond, k) \
    do {                   \
    } while (0)
#define REI_TSTART() \
    do {             \
    } while (0)
#endif

struct TileCtx {
    const SolveJob *J;
    SolveState *st;
    const Shared *S;
    uint64_t chunk_start;
    uint32_t W, Ws, n;
    bool dedup;
    bool grid;  // every CTA works on the chunk (else CTA 0 alone)
    unsigned long long *found;  // minimum precise candidate: shared (small chunk alone) or global
    unsigned long long *ent;    // small chunk alone: per candidate, fingerprint << 32 | slot; else null
    uint32_t *bits;             // small chunk alone: candidates that took or won a slot
    const uint32_t *ops;        // the cached languages operands are read from (shared or global)
    bool smem;                  // uniqueness in CTA 0's shared table
};

// an operand word: generic relaxed load (the rows are in shared memory at
// the search's start, in global memory, written by other CTAs, later)
__device__ __forceinline__ uint32_t ldop(const uint32_t *p) {
    uint32_t v;
    asm volatile("ld.relaxed.gpu.u32 %0, [%1];" : "=r"(v) : "l"(p));
    return v;
}

constexpr uint32_t kSmEmpty = 0xFFFFFFFFu;
constexpr uint32_t kSmPending = 0x10000u;

// uniqueness insert of candidate xl while the languages live in shared
// memory: the same protocol as dedup_insert_solo on a 32-bit table whose
// entries are fp (15 bits) << 17 | pending << 16 | row or candidate
template <uint32_t WT>
__device__ void dedup_insert_smem(const TileCtx &T, const uint32_t *c, uint32_t xl) {
    const Shared &S = *T.S;
    const uint32_t W = WT ? WT : T.W;
    const uint64_t h = cs_hash(c, W, 1);
    const uint32_t fp = (uint32_t)(h >> 49);  // 15 bits
    const uint32_t mine = (fp << 17) | kSmPending | xl;
    const uint32_t mask = 2 * T.J->small_rows - 1;
    uint32_t p = (uint32_t)h & mask;
    uint32_t *dst = S.sm_tmp + xl * W;
    for (uint32_t b = 0; b < W; b++) dst[b] = c[b];
    __threadfence_block();
    for (uint32_t probe = 0; probe <= mask; probe++) {
        const uint32_t v = atomicCAS(&S.sm_table[p], kSmEmpty, mine);
        if (v == kSmEmpty) {
            T.ent[xl] = p;
            atomicOr(&T.bits[xl >> 5], 1u << (xl & 31));
            return;
        }
        if ((v >> 17) == fp) {
            __threadfence_block();
            const uint32_t idx = v & 0xFFFFu;
            const volatile uint32_t *src = (v & kSmPending) ? S.sm_tmp + idx * W : S.sm_rows + idx * W;
            bool eq = true;
            for (uint32_t b = 0; b < W && eq; b++) eq = src[b] == c[b];
            if (eq) {
                if ((v & kSmPending) && idx > xl && atomicMin(&S.sm_table[p], mine) > mine) {
                    T.ent[xl] = p;
                    atomicOr(&T.bits[xl >> 5], 1u << (xl & 31));
                }
                return;
            }
        }
        p = (p + 1) & mask;
    }
    atomicExch(&T.st->err, 2u);  // table full: cannot happen with load <= 1/2
}

// A fingerprint entry names a cached row (below the cache's rows) or, marked
// pending, a candidate of the current chunk (below the chunk size).  Any other
// value was not written by this search (memory not emptied before the search
// began): the search is stopped with an error and nothing is read through it.
__device__ __forceinline__ bool entry_ok(const TileCtx &T, uint32_t idx) {
    const SolveJob &J = *T.J;
    const bool ok = (idx & kPending) ? (idx & ~kPending) < J.chunk_max : idx < J.cache_alloc;
    if (!ok) {
        atomicCAS(&T.st->err, 0u, 6u);
        atomicExch(&T.st->status, (uint32_t)ST_TIMEOUT);
    }
    return ok;
}

// uniqueness insert of candidate xl of a small chunk that CTA 0 runs alone
// (no other CTA touches the table meanwhile).  The candidate's row goes to
// tmp first, then the slot is claimed with one CAS whose result doubles as
// the probe; a candidate that takes an empty slot, or replaces a later
// pending holder of the same language, is marked in T.bits with its slot in
// T.ent; the append keeps the marks whose slot still names them.
template <uint32_t WT>
__device__ void dedup_insert_solo(const TileCtx &T, const uint32_t *c, uint32_t xl) {
    const SolveJob &J = *T.J;
    const uint32_t W = WT ? WT : T.W;
    const uint64_t h = cs_hash(c, W, 1);
    const uint32_t fp = (uint32_t)(h >> 32);
    const unsigned long long mine = ((uint64_t)fp << 32) | kPending | xl;
    uint64_t p = h & J.table_mask;
    uint32_t *dst = J.tmp + (uint64_t)xl * W;
    for (uint32_t b = 0; b < W; b++) dst[b] = c[b];
    __threadfence_block();
    for (uint64_t probe = 0; probe <= J.table_mask; probe++) {
        const unsigned long long v = atomicCAS(&J.table[p], kEmpty, mine);
        if (v == kEmpty) {
            T.ent[xl] = ((unsigned long long)fp << 32) | (uint32_t)p;
            atomicOr(&T.bits[xl >> 5], 1u << (xl & 31));
            return;
        }
        if ((uint32_t)(v >> 32) == fp && entry_ok(T, (uint32_t)v)) {
            __threadfence_block();
            const uint32_t idx = (uint32_t)v;
            const uint32_t *src = (idx & kPending) ? J.tmp + (uint64_t)(idx & ~kPending) * W
                                                   : J.cs + (uint64_t)idx * W;
            bool eq = true;
            for (uint32_t b = 0; b < W && eq; b++) eq = ldcg(src + b) == c[b];
            if (eq) {
                if ((idx & kPending) && (idx & ~kPending) > xl && atomicMin(&J.table[p], mine) > mine) {
                    T.ent[xl] = ((unsigned long long)fp << 32) | (uint32_t)p;
                    atomicOr(&T.bits[xl >> 5], 1u << (xl & 31));
                }
                return;
            }
        }
        p = (p + 1) & J.table_mask;
    }
    atomicExch(&T.st->err, 2u);  // table full: cannot happen with load <= 1/2
}

constexpr unsigned long long kXPend = 1ull << 63;  // exact keys: the language was added in this chunk

// the exact key of a W <= 2 language (padding bits and bit 63 are zero)
__device__ __forceinline__ unsigned long long exact_key(const uint32_t *c, uint32_t W) {
    return W == 1 ? (unsigned long long)c[0] : ((unsigned long long)c[1] << 32) | c[0];
}

// uniqueness insert with exact keys: the slot's key is the language, so a
// duplicate costs one probe and no row read; a language new in this chunk is
// claimed with a CAS and every candidate with it lowers minidx[slot] (a
// reduction, no round trip); `mark` (a small chunk on one CTA) records the
// claimants in T.bits / T.ent, else the claimed slot joins the pending list
template <uint32_t WT>
__device__ void dedup_insert_exact(const TileCtx &T, const uint32_t *c, uint32_t xl) {
    const SolveJob &J = *T.J;
    const uint32_t W = WT ? WT : T.W;
    // a language cached by an earlier chunk: one bit of the seen bitmap (set
    // by the append of that chunk, visible after its grid barriers; read
    // through L2).  Languages new in this chunk take the table protocol below.
    if (J.seen && ((ldcg(J.seen + (c[0] >> 5)) >> (c[0] & 31u)) & 1u)) return;
    const unsigned long long key = exact_key(c, W), pk = key | kXPend;
    uint64_t p = J.direct ? key : cs_hash(c, W, 1) & J.table_mask;
    for (uint64_t probe = 0; probe <= J.table_mask; probe++) {
        unsigned long long v = ld_relaxed_u64(&J.table[p]);
        if (v == kEmpty) {
            v = atomicCAS(&J.table[p], kEmpty, pk);
            if (v == kEmpty) {
                atomicMin(&J.minidx[p], xl);
                if (T.bits) {
                    T.ent[xl] = p;
                    atomicOr(&T.bits[xl >> 5], 1u << (xl & 31));
                } else {
                    const uint32_t am = __activemask(), lane = threadIdx.x & 31, lead = __ffs(am) - 1;
                    uint32_t k0 = 0;
                    if (lane == lead) k0 = atomicAdd(&T.st->pending_count, (uint32_t)__popc(am));
                    k0 = __shfl_sync(am, k0, lead);
                    J.pending[k0 + __popc(am & ((1u << lane) - 1u))] = (uint32_t)p;
                }
                return;
            }
        }
        if ((v & ~kXPend) == key) {
            if (v & kXPend) {
                atomicMin(&J.minidx[p], xl);
                if (T.bits) {
                    T.ent[xl] = p;
                    atomicOr(&T.bits[xl >> 5], 1u << (xl & 31));
                }
            }
            return;
        }
        p = (p + 1) & J.table_mask;
    }
    atomicExch(&T.st->err, 2u);  // table full: cannot happen with load <= 1/2
}

// uniqueness insert of candidate xl (chunk-local) whose CS is c[b * 1] (smem)
template <uint32_t WT>
__device__ void dedup_insert(const TileCtx &T, const uint32_t *c, uint32_t xl) {
    const SolveJob &J = *T.J;
    const uint32_t W = WT ? WT : T.W;
    const uint64_t h = cs_hash(c, W, 1);
    const uint32_t fp = (uint32_t)(h >> 32);
    const uint64_t mine = ((uint64_t)fp << 32) | kPending | xl;
    uint64_t p = h & J.table_mask;
    bool wrote = false;
    auto write_tmp = [&]() {
        if (wrote) return;
        uint32_t *dst = J.tmp + (uint64_t)xl * W;
        for (uint32_t b = 0; b < W; b++) dst[b] = c[b];
        // the row must be visible before the slot that points at it: to every
        // CTA when the grid works on the chunk, to this CTA when it works alone
        if (T.grid) __threadfence();
        else __threadfence_block();
        wrote = true;
    };
    for (uint64_t probe = 0; probe <= J.table_mask; probe++) {
        unsigned long long v = ld_acquire_u64(&J.table[p]);
        if (v == kEmpty) {
            write_tmp();
            const unsigned long long old = atomicCAS(&J.table[p], kEmpty, mine);
            if (old == kEmpty) {
                // one counter update per group of lanes that inserted together
                const uint32_t am = __activemask(), lane = threadIdx.x & 31, lead = __ffs(am) - 1;
                uint32_t k0 = 0;
                if (lane == lead) k0 = atomicAdd(&T.st->pending_count, (uint32_t)__popc(am));
                k0 = __shfl_sync(am, k0, lead);
                J.pending[k0 + __popc(am & ((1u << lane) - 1u))] = (uint32_t)p;
                return;
            }
            v = old;
            __threadfence();
        }
        if ((uint32_t)(v >> 32) == fp && entry_ok(T, (uint32_t)v)) {
            const uint32_t idx = (uint32_t)v;
            const uint32_t *src = (idx & kPending) ? J.tmp + (uint64_t)(idx & ~kPending) * W
                                                   : J.cs + (uint64_t)idx * W;
            bool eq = true;
            for (uint32_t b = 0; b < W && eq; b++) eq = ldcg(src + b) == c[b];
            if (eq) {
                if (idx & kPending) {
                    write_tmp();
                    atomicMin(&J.table[p], mine);
                }
                return;
            }
        }
        p = (p + 1) & J.table_mask;
    }
    atomicExch(&T.st->err, 2u);  // table full: cannot happen with load <= 1/2
}

// build the CSs of one tile into A (candidate-major, row stride Ws), then test
// precision and insert; lanes with !valid only help with the warp collectives.
// WT > 0 fixes the language width at compile time (W = WT), 0 reads it from T.
template <uint32_t WT>
__device__ void run_tile(const TileCtx &T, const Seg &sg, const SegTile &tl, uint64_t tile, uint32_t *wm) {
    const SolveJob &J = *T.J;
    const Shared &S = *T.S;
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t W = WT ? WT : T.W, Ws = WT ? ((WT & 1u) ? WT : WT + 1) : T.Ws, n = T.n;
    uint32_t *lw = wm;
    uint32_t *A = wm + ((W + 3) & ~3u);
    uint32_t *B = A + 32 * Ws;
    const uint32_t *cs = T.ops;
    const uint64_t lo = tl.lo, hi = tl.hi;
    // word i of the tile's candidate-major rows is word b of row j (shift for a power-of-two W)
    const uint32_t wlog = (W & (W - 1)) == 0 ? (uint32_t)(__ffs(W) - 1) : 32u;
#define TILE_JB(i, j, b)                                     \
    const uint32_t j = wlog < 32 ? (i) >> wlog : (i) / W; \
    const uint32_t b = (i) - j * W

    // which candidate this lane holds; `first` is the first of the tile's 32
    // consecutive operands (the right ones, the left ones when swapped, or
    // the only ones)
    uint64_t x;  // segment-local index
    uint32_t row = 0, col = 0, first = 0, nrow;
    bool valid;
    const bool binary = sg.op == OP_CAT || sg.op == OP_ALT;
    const bool swapped = sg.op == OP_CAT && sg.swap;
    if (!binary) {
        first = (uint32_t)(lo + tile * 32);
        x = (uint64_t)first + lane;
        valid = x < hi;
        nrow = (uint32_t)umin64(32, hi - first);
    } else if (swapped) {
        // (a segment's tiles in a chunk and its blocks per row fit 31 bits)
        const uint32_t t32 = (uint32_t)tile, nb = tl.nb, qt = div_by(t32, tl.nb_mul, tl.nb_shift);
        col = qt;
        first = (uint32_t)tl.r0 + (t32 - qt * nb) * 32;
        row = first + lane;
        x = (uint64_t)row * sg.rcnt + col;
        valid = row < sg.lcnt && x >= lo && x < hi;
        nrow = min(32u, sg.lcnt - first);
    } else {
        const uint32_t t32 = (uint32_t)tile, nb = tl.nb, qt = div_by(t32, tl.nb_mul, tl.nb_shift);
        row = (uint32_t)tl.r0 + qt;
        first = (t32 - qt * nb) * 32;
        col = first + lane;
        x = (uint64_t)row * sg.rcnt + col;
        valid = col < sg.rcnt && x >= lo && x < hi && (!sg.tri || col > row);
        nrow = min(32u, sg.rcnt - first);
    }
    const uint32_t vmask = __ballot_sync(0xFFFFFFFFu, valid);
    if (vmask == 0) return;
#ifdef REI_TIMING
    SolveState *st = T.st;
    REI_TSTART();
    const bool tmk = !T.grid && threadIdx.x == 0;
#endif

    // ---- build
    if (sg.op == OP_LEAF) {
        for (uint32_t i = lane; i < 32 * W; i += 32) {
            TILE_JB(i, j, b);
            A[j * Ws + b] = j < nrow ? __ldg(J.leaf + (uint64_t)J.leaf_sym[sg.lbase + first + j] * J.leaf_stride + b)
                                     : 0u;
        }
        __syncwarp();
    } else if (sg.op == OP_OPT) {
        const uint32_t *src = cs + (uint64_t)(sg.lbase + first) * W;
        for (uint32_t i = lane; i < 32 * W; i += 32) {
            TILE_JB(i, j, b);
            A[j * Ws + b] = j < nrow ? ldop(src + i) : 0u;
        }
        __syncwarp();
        A[lane * Ws] |= 1u;  // eps is ic word 0
        __syncwarp();
    } else if (sg.op == OP_ALT) {
        const uint32_t *l = cs + (uint64_t)(sg.lbase + row) * W;
        const uint32_t *src = cs + (uint64_t)(sg.rbase + first) * W;
        for (uint32_t b = lane; b < W; b += 32) lw[b] = ldop(l + b);
        __syncwarp();
        for (uint32_t i = lane; i < 32 * W; i += 32) {
            TILE_JB(i, j, b);
            A[j * Ws + b] = j < nrow ? (lw[b] | ldop(src + i)) : 0u;
        }
        __syncwarp();
    } else {
        // CAT / STAR: bit-sliced over 32 operands (the right ones of a
        // concatenation, its left ones when swapped, or a star's only ones)
        const uint32_t base = sg.op == OP_STAR ? sg.lbase : swapped ? sg.lbase : sg.rbase;
        const uint32_t *src = cs + (uint64_t)(base + first) * W;
        for (uint32_t i = lane; i < 32 * W; i += 32) {
            TILE_JB(i, j, b);
            A[j * Ws + b] = j < nrow ? ldop(src + i) : 0u;
        }
        if (sg.op == OP_CAT) {
            // the one operand shared by the tile
            const uint32_t *o = cs + (uint64_t)(swapped ? sg.rbase + col : sg.lbase + row) * W;
            for (uint32_t b = lane; b < W; b += 32) lw[b] = ldop(o + b);
        }
        __syncwarp();
        REI_TMARK(tmk, 6);
        // slices: B[v] bit j = operand j contains word v
        for (uint32_t b = 0; b < W; b++) B[32 * b + lane] = transpose32(A[lane * Ws + b], lane);
        __syncwarp();
        const uint32_t *go = S.gt_off, *gp = S.gt_pair;
        if (sg.op == OP_CAT) {
            // out[w] = OR over splits w = u v of l[u] and r[v]  (Alg. 2)
            for (uint32_t b = 0; b < W; b++) {
                const uint32_t w = 32 * b + lane;
                uint32_t acc = 0;
                if (WT == 1 || WT == 2) {
                    // the shared operand's words in registers
                    if (w < n) {
                        const uint32_t l0 = lw[0], l1 = WT == 2 ? lw[1] : 0u;
                        const uint32_t p1 = go[w + 1];
                        const uint32_t sh = swapped ? 16u : 0u;  // which half of a pair indexes the shared operand
#pragma unroll 4
                        for (uint32_t p = go[w]; p < p1; p++) {
                            const uint32_t pr = gp[p];
                            const uint32_t k = (pr >> sh) & 0xFFFFu, o = (pr >> (16u - sh)) & 0xFFFFu;
                            const uint32_t lv = (WT == 2 && (k & 32u)) ? l1 : l0;
                            acc |= B[o] & (0u - ((lv >> (k & 31u)) & 1u));
                        }
                    }
                } else if (w < n) {
                    const uint32_t p1 = go[w + 1];
                    if (!swapped) {
#pragma unroll 4
                        for (uint32_t p = go[w]; p < p1; p++) {
                            const uint32_t pr = gp[p];
                            const uint32_t u = pr & 0xFFFFu, v = pr >> 16;
                            acc |= B[v] & (0u - ((lw[u >> 5] >> (u & 31)) & 1u));
                        }
                    } else {
#pragma unroll 4
                        for (uint32_t p = go[w]; p < p1; p++) {
                            const uint32_t pr = gp[p];
                            const uint32_t u = pr & 0xFFFFu, v = pr >> 16;
                            acc |= B[u] & (0u - ((lw[v >> 5] >> (v & 31)) & 1u));
                        }
                    }
                }
                A[lane * Ws + b] = transpose32(acc, lane);
            }
            __syncwarp();
        } else {
            // r* as the least S with S = 1 + r.S, by increasing word length:
            // S[w] = OR over splits w = u v with u != eps of r[u] and S[v]
            uint32_t *Sl = A;
            for (uint32_t w = lane; w < 32 * W; w += 32) Sl[w] = 0u;
            __syncwarp();
            if (lane == 0) Sl[0] = 0xFFFFFFFFu;
            __syncwarp();
            const uint32_t *ls = S.len_start;
            for (uint32_t L = 1; L <= J.max_len; L++) {
                const uint32_t w1 = ls[L + 1];
                for (uint32_t w = ls[L] + lane; w < w1; w += 32) {
                    uint32_t acc = 0;
                    const uint32_t p1 = go[w + 1];
#pragma unroll 4
                    for (uint32_t p = go[w] + 1; p < p1; p++) {
                        const uint32_t pr = gp[p];
                        acc |= B[pr & 0xFFFFu] & Sl[pr >> 16];
                    }
                    Sl[w] = acc;
                }
                __syncwarp();
            }
            for (uint32_t b = 0; b < W; b++) B[lane * Ws + b] = transpose32(Sl[32 * b + lane], lane);
            __syncwarp();
            for (uint32_t i = lane; i < 32 * Ws; i += 32) A[i] = B[i];
            __syncwarp();
        }
    }

    REI_TMARK(tmk, 7);
    // ---- precision and uniqueness, one candidate per lane
    if (!valid) return;
    const uint32_t *c = A + lane * Ws;
    uint32_t errs = 0;
    for (uint32_t b = 0; b < W; b++) errs += __popc(S.pos[b] & ~c[b]) + __popc(S.neg[b] & c[b]);
    const uint64_t xlev = sg.start + x;
    if (errs <= J.max_errors) atomicMin(T.found, (unsigned long long)xlev);
    REI_TMARK(tmk, 8);
    if (T.dedup) {
        const uint32_t xl = (uint32_t)(xlev - T.chunk_start);
        if (T.smem) dedup_insert_smem<WT>(T, c, xl);
        else if (J.exact) dedup_insert_exact<WT>(T, c, xl);
        else if (T.bits) dedup_insert_solo<WT>(T, c, xl);
        else dedup_insert<WT>(T, c, xl);
    }
    REI_TMARK(tmk, 9);
}

#undef TILE_JB

// ---------------------------------------------------------------------------
// phase A for 1-word languages (|ic| <= 32): one candidate per lane, its
// language built in a register.  A concatenation l.r with one operand shared
// by the whole tile (l, or r when swapped) is a map of the other operand's
// words: out = OR over the set bits b of the other operand of M[b], with M[b]
// the words w = u v of ic with u in l and v = b (swapped: u = b and v in r),
// read off the guide table (Alg. 2).  The map is kept as 8 nibble tables,
// T[t][x] = OR over the set bits i of x of M[4t + i], so a candidate costs one
// shared-memory read per 4 bits of ic; the tables are rebuilt only when the
// tile's shared operand differs from the previous tile's.

__device__ __forceinline__ void w1_tables(const Shared &S, uint32_t n, uint32_t shared_cs, bool swapped,
                                          uint32_t *tab, uint32_t lane) {
    // lane w: column w of M (bit b set when M[b] holds w)
    uint32_t col = 0;
    if (lane < n) {
        const uint32_t p1 = S.gt_off[lane + 1];
        for (uint32_t p = S.gt_off[lane]; p < p1; p++) {
            const uint32_t pr = S.gt_pair[p];
            const uint32_t u = pr & 0xFFFFu, v = pr >> 16;
            const uint32_t have = swapped ? v : u, other = swapped ? u : v;
            col |= ((shared_cs >> have) & 1u) << other;
        }
    }
    const uint32_t m = transpose32(col, lane);  // lane b: M[b]
    // lane 4t + q fills entries 4q .. 4q + 3 of table t
    const uint32_t t = lane >> 2, q = lane & 3u;
    const uint32_t m0 = __shfl_sync(0xFFFFFFFFu, m, 4 * t), m1 = __shfl_sync(0xFFFFFFFFu, m, 4 * t + 1);
    const uint32_t m2 = __shfl_sync(0xFFFFFFFFu, m, 4 * t + 2), m3 = __shfl_sync(0xFFFFFFFFu, m, 4 * t + 3);
    const uint32_t base = ((q & 1u) ? m2 : 0u) | ((q & 2u) ? m3 : 0u);
    *reinterpret_cast<uint4 *>(tab + 16 * t + 4 * q) = make_uint4(base, base | m0, base | m1, base | m0 | m1);
}

__device__ __forceinline__ uint32_t w1_lookup(const uint32_t *tab, uint32_t x, uint32_t nt) {
    uint32_t out = 0;
#pragma unroll
    for (uint32_t t = 0; t < 8; t++)
        if (t < nt) out |= tab[16 * t + ((x >> (4 * t)) & 15u)];
    return out;
}

// precision and uniqueness of a lane's kW1Per 1-word candidates c[k]
// (level-segment indices x0 + k * dx, valid where bit k of vb is set): every
// seen-bitmap word is read before any is tested, so the reads overlap
template <uint32_t K>
__device__ __forceinline__ void w1_finish(const TileCtx &T, const Seg &sg, uint32_t (&c)[K], uint64_t x0, uint64_t dx,
                                          uint32_t vb) {
    const SolveJob &J = *T.J;
    const Shared &S = *T.S;
    const uint32_t pos = S.pos[0], neg = S.neg[0];
    const uint64_t xlev0 = sg.start + x0;
    if (T.dedup && !T.smem && J.exact && J.seen) {
        // Languages cached by earlier chunks end here, at one bit each, and
        // need no precision test: a cached language was tested when its
        // first candidate was, and a precise one would have ended the search.
        uint32_t w[K];
#pragma unroll
        for (uint32_t k = 0; k < K; k++) w[k] = ((vb >> k) & 1u) ? ldcg(J.seen + (c[k] >> 5)) : 0xFFFFFFFFu;
#pragma unroll
        for (uint32_t k = 0; k < K; k++) {
            if ((w[k] >> (c[k] & 31u)) & 1u) continue;
            const uint64_t xlev = xlev0 + k * dx;
            if (__popc(pos & ~c[k]) + __popc(neg & c[k]) <= J.max_errors) atomicMin(T.found, (unsigned long long)xlev);
            dedup_insert_exact<1>(T, &c[k], (uint32_t)(xlev - T.chunk_start));
        }
        return;
    }
#pragma unroll
    for (uint32_t k = 0; k < K; k++) {
        if (!((vb >> k) & 1u)) continue;
        const uint64_t xlev = xlev0 + k * dx;
        if (__popc(pos & ~c[k]) + __popc(neg & c[k]) <= J.max_errors) atomicMin(T.found, (unsigned long long)xlev);
        if (!T.dedup) continue;
        const uint32_t xl = (uint32_t)(xlev - T.chunk_start);
        if (T.smem) dedup_insert_smem<1>(T, &c[k], xl);
        else if (J.exact) dedup_insert_exact<1>(T, &c[k], xl);
        else if (T.bits) dedup_insert_solo<1>(T, &c[k], xl);
        else dedup_insert<1>(T, &c[k], xl);
    }
}

// one tile of 1-word candidates: 32 of a unary segment (one per lane), or
// 32 * kW1Per of a binary one (kW1Per per lane, 32 apart)
__device__ void run_tile_w1(const TileCtx &T, const Seg &sg, const SegTile &tl, uint64_t tile, uint32_t *wm) {
    if (sg.op == OP_STAR) {  // (few candidates: the bit-sliced fixed point)
        run_tile<1>(T, sg, tl, tile, wm);
        return;
    }
    const SolveJob &J = *T.J;
    const Shared &S = *T.S;
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t *cs = T.ops;
    const uint64_t lo = tl.lo, hi = tl.hi;
    if (sg.op == OP_LEAF || sg.op == OP_OPT) {
        const uint64_t x = lo + tile * 32 + lane;
        const bool valid = x < hi;
        if (__ballot_sync(0xFFFFFFFFu, valid) == 0) return;
        uint32_t c[1] = {0u};
        if (sg.op == OP_LEAF) {
            if (valid) c[0] = __ldg(J.leaf + (uint64_t)J.leaf_sym[sg.lbase + (uint32_t)x] * J.leaf_stride);
        } else {
            c[0] = (valid ? ldop(cs + sg.lbase + (uint32_t)x) : 0u) | 1u;  // eps is ic word 0
        }
        w1_finish<1>(T, sg, c, x, 0, valid ? 1u : 0u);
        return;
    }
    // binary: candidate k of the lane is (row, col0 + 32 k), or, swapped,
    // (row0 + 32 k, col)
    constexpr uint32_t K = kW1Per;
    const bool swapped = sg.op == OP_CAT && sg.swap;
    const uint32_t t32 = (uint32_t)tile, qt = div_by(t32, tl.nb_mul, tl.nb_shift);
    const uint32_t off = (t32 - qt * tl.nb) * (32 * K) + lane;
    uint32_t row, col;  // of candidate 0
    uint64_t x0, dx;
    uint32_t vb = 0;
    if (swapped) {
        col = qt;
        row = (uint32_t)tl.r0 + off;
        x0 = (uint64_t)row * sg.rcnt + col;
        dx = 32ull * sg.rcnt;
#pragma unroll
        for (uint32_t k = 0; k < K; k++) {
            const uint64_t x = x0 + k * dx;
            if (row + 32 * k < sg.lcnt && x >= lo && x < hi) vb |= 1u << k;
        }
    } else {
        row = (uint32_t)tl.r0 + qt;
        col = off;
        x0 = (uint64_t)row * sg.rcnt + col;
        dx = 32;
#pragma unroll
        for (uint32_t k = 0; k < K; k++) {
            const uint64_t x = x0 + 32 * k;
            const uint32_t ck = col + 32 * k;
            if (ck < sg.rcnt && x >= lo && x < hi && (!sg.tri || ck > row)) vb |= 1u << k;
        }
    }
    if (__ballot_sync(0xFFFFFFFFu, vb != 0) == 0) return;
    uint32_t c[K];
    if (sg.op == OP_ALT) {
        const uint32_t l = ldop(cs + sg.lbase + row);
        uint32_t r[K];
#pragma unroll
        for (uint32_t k = 0; k < K; k++) r[k] = ((vb >> k) & 1u) ? ldop(cs + sg.rbase + col + 32 * k) : 0u;
#pragma unroll
        for (uint32_t k = 0; k < K; k++) c[k] = l | r[k];
    } else {
        // the tables of the shared operand (its id in the word after them)
        uint32_t *tab = wm + kW1TabAt;
        const uint32_t sid = swapped ? (0x80000000u | (sg.rbase + col)) : (sg.lbase + row);
        if (tab[kW1Tab] != sid) {
            const uint32_t sh = ldop(cs + (sid & 0x7FFFFFFFu));
            __syncwarp();  // (every lane has read the old id)
            w1_tables(S, T.n, sh, swapped, tab, lane);
            if (lane == 0) tab[kW1Tab] = sid;
            __syncwarp();
        }
        const uint32_t *ob = swapped ? cs + sg.lbase + row : cs + sg.rbase + col;
        uint32_t o[K];
#pragma unroll
        for (uint32_t k = 0; k < K; k++) o[k] = ((vb >> k) & 1u) ? ldop(ob + 32 * k) : 0u;
        const uint32_t nt = (T.n + 3) >> 2;
#pragma unroll
        for (uint32_t k = 0; k < K; k++) c[k] = w1_lookup(tab, o[k], nt);
    }
    w1_finish<K>(T, sg, c, x0, dx, vb);
}

// ---------------------------------------------------------------------------
// decode a level-local index into (segment, op, left, right)

__device__ void decode(const Seg *seg, uint32_t nseg, const uint8_t *leaf_sym, uint64_t xlev, uint32_t &op,
                       uint32_t &l, uint32_t &r) {
    uint32_t s = 0;
    while (s + 1 < nseg && seg[s + 1].start <= xlev) s++;
    const Seg &g = seg[s];
    const uint64_t x = xlev - g.start;
    op = g.op;
    if (g.op == OP_LEAF) {
        l = leaf_sym[g.lbase + x];  // the symbol's alphabet index
        r = kNoRight;
    } else if (g.op == OP_OPT || g.op == OP_STAR) {
        l = g.lbase + (uint32_t)x;
        r = kNoRight;
    } else {
        l = g.lbase + (uint32_t)(x / g.rcnt);
        r = g.rbase + (uint32_t)(x % g.rcnt);
    }
}

// postfix tokens of the answer (op, l, r), walking back-pointers; the walk's
// stack (4 words per frame, at most max_cost + 1 frames deep since every node
// costs at least 1) lives in global scratch
__device__ uint32_t emit_tree(const SolveJob &J, uint32_t op, uint32_t l, uint32_t r) {
    uint32_t *stack = J.tstack;
    const int depth_cap = (int)J.max_cost + 2;
    int sp = 0;
    uint32_t nt = 0;
    const uint32_t cap = J.max_cost + 1;
    auto push = [&](uint32_t o, uint32_t a, uint32_t b) {
        if (sp < depth_cap) {
            stack[4 * sp] = o;
            stack[4 * sp + 1] = a;
            stack[4 * sp + 2] = b;
            stack[4 * sp + 3] = 0;
            sp++;
        }
    };
    auto push_entry = [&](uint32_t e) {
        push(*(volatile const uint8_t *)(J.bp_op + e), ldcg(J.bp_l + e), ldcg(J.bp_r + e));
    };
    push(op, l, r);
    while (sp > 0) {
        uint32_t *f = stack + 4 * (sp - 1);
        const uint32_t fop = f[0];
        const bool bin = fop == OP_CAT || fop == OP_ALT;
        const bool un = fop == OP_OPT || fop == OP_STAR;
        if (f[3] == 0 && (bin || un)) {
            f[3] = 1;
            push_entry(f[1]);
            continue;
        }
        if (f[3] == 1 && bin) {
            f[3] = 2;
            push_entry(f[2]);
            continue;
        }
        uint8_t k = '+', a = 0;
        switch (fop) {
        case OP_LEAF: k = 'a'; a = (uint8_t)f[1]; break;
        case OP_OPT: k = '?'; break;
        case OP_STAR: k = '*'; break;
        case OP_CAT: k = '.'; break;
        default: break;
        }
        if (nt < cap) {
            J.tree[2 * nt] = k;
            J.tree[2 * nt + 1] = a;
        }
        nt++;
        sp--;
    }
    return nt;
}

// The same postfix tokens, by one whole warp, in a few rounds of loads
// instead of one per node: the tree is gathered breadth first (every node of
// a depth fetches its children's back-pointers at once), subtree sizes are
// summed bottom-up and postfix positions handed down top-down, depth by depth,
// in shared scratch (`scr`, kTreeScratchWords words).  Returns the token count
// (in every lane), or falls back to emit_tree when the tree does not fit.
constexpr uint32_t kTreeNodes = 480;  // nodes the scratch holds (7 arrays + depth starts)
constexpr uint32_t kTreeScratchWords = 7 * kTreeNodes + kTreeNodes + 1;
__device__ uint32_t emit_tree_warp(const SolveJob &J, uint32_t op, uint32_t l, uint32_t r, uint32_t *scr) {
    const uint32_t lane = threadIdx.x & 31;
    uint32_t *nop = scr, *na = nop + kTreeNodes, *nb = na + kTreeNodes, *c0 = nb + kTreeNodes;
    uint32_t *c1 = c0 + kTreeNodes, *sz = c1 + kTreeNodes, *pos = sz + kTreeNodes, *dep = pos + kTreeNodes;
    if (lane == 0) {
        nop[0] = op;
        na[0] = l;
        nb[0] = r;
        dep[0] = 0;
        dep[1] = 1;
    }
    __syncwarp();
    // ---- gather, one depth per round: node v's children are appended in
    // order (left, right) at the positions a warp scan of the child counts gives
    uint32_t nd = 1, f0 = 0, f1 = 1;  // depths, current frontier [f0, f1)
    bool fits = true;
    while (f0 < f1) {
        uint32_t next = f1;
        for (uint32_t b0 = f0; b0 < f1; b0 += 32) {
            const uint32_t v = b0 + lane;
            uint32_t k = 0, o = 0;
            if (v < f1) {
                o = nop[v];
                k = (o == OP_CAT || o == OP_ALT) ? 2u : (o == OP_OPT || o == OP_STAR) ? 1u : 0u;
            }
            uint32_t incl = k;
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, incl, d);
                if (lane >= (uint32_t)d) incl += y;
            }
            const uint32_t at = next + incl - k, tot = __shfl_sync(0xFFFFFFFFu, incl, 31);
            if (next + tot > kTreeNodes) {
                fits = false;
                break;
            }
            if (k) {
                const uint32_t e0 = na[v];
                uint32_t op0 = *(volatile const uint8_t *)(J.bp_op + e0), l0 = ldcg(J.bp_l + e0), r0 = ldcg(J.bp_r + e0);
                uint32_t op1 = 0, l1 = 0, r1 = 0;
                if (k == 2) {
                    const uint32_t e1 = nb[v];
                    op1 = *(volatile const uint8_t *)(J.bp_op + e1);
                    l1 = ldcg(J.bp_l + e1);
                    r1 = ldcg(J.bp_r + e1);
                }
                nop[at] = op0;
                na[at] = l0;
                nb[at] = r0;
                c0[v] = at;
                if (k == 2) {
                    nop[at + 1] = op1;
                    na[at + 1] = l1;
                    nb[at + 1] = r1;
                    c1[v] = at + 1;
                }
            }
            next += tot;
        }
        fits = __all_sync(0xFFFFFFFFu, fits);
        if (!fits) break;
        __syncwarp();
        f0 = f1;
        f1 = next;
        if (f0 < f1) {
            if (nd + 1 > kTreeNodes) {
                fits = false;
                break;
            }
            nd++;
            if (lane == 0) dep[nd] = f1;
        }
        __syncwarp();
    }
    if (!fits) {
        uint32_t nt = 0;
        if (lane == 0) nt = emit_tree(J, op, l, r);
        return __shfl_sync(0xFFFFFFFFu, nt, 0);
    }
    const uint32_t nodes = f1;
    // ---- subtree sizes, deepest depth first
    for (int d = (int)nd - 1; d >= 0; d--) {
        for (uint32_t v = dep[d] + lane; v < dep[d + 1]; v += 32) {
            const uint32_t o = nop[v];
            uint32_t t = 1;
            if (o == OP_CAT || o == OP_ALT) t += sz[c0[v]] + sz[c1[v]];
            else if (o == OP_OPT || o == OP_STAR) t += sz[c0[v]];
            sz[v] = t;
        }
        __syncwarp();
    }
    // ---- postfix positions, from the root down: a node is last in its
    // subtree, its left subtree first, then its right one
    if (lane == 0) pos[0] = sz[0] - 1;
    __syncwarp();
    for (uint32_t d = 0; d < nd; d++) {
        for (uint32_t v = dep[d] + lane; v < dep[d + 1]; v += 32) {
            const uint32_t o = nop[v], p = pos[v];
            if (o == OP_CAT || o == OP_ALT) {
                const uint32_t start = p + 1 - sz[v];
                pos[c0[v]] = start + sz[c0[v]] - 1;
                pos[c1[v]] = p - 1;
            } else if (o == OP_OPT || o == OP_STAR) {
                pos[c0[v]] = p - 1;
            }
        }
        __syncwarp();
    }
    // ---- tokens
    const uint32_t cap = J.max_cost + 1;
    for (uint32_t v = lane; v < nodes; v += 32) {
        const uint32_t o = nop[v], p = pos[v];
        uint8_t k = '+', a = 0;
        switch (o) {
        case OP_LEAF: k = 'a'; a = (uint8_t)na[v]; break;
        case OP_OPT: k = '?'; break;
        case OP_STAR: k = '*'; break;
        case OP_CAT: k = '.'; break;
        default: break;
        }
        if (p < cap) {
            J.tree[2 * p] = k;
            J.tree[2 * p + 1] = a;
        }
    }
    __syncwarp();
    return nodes;
}

// ---------------------------------------------------------------------------
// the persistent search kernel
//
// The team's first CTA (CTA 0 of a plain launch) leads: it plans levels, moves
// from level to level and decides, chunk by chunk, whether to process the
// chunk alone (small chunks: its own warps, __syncthreads between phases, no
// grid-wide wait) or with the whole team.  The other CTAs wait for a command
// (a sequence number and parameters in the state, published with release /
// read with acquire), join the chunk's phases with grid barriers, and go back
// to waiting.  A team is every CTA of the launch, or (continued batch
// searches) a group of them per problem.

// CTAs of the plain path, 16 warps each: the fused launch (staging, then the
// levels of a small or medium search, latency-bound) runs one per SM, at up
// to 128 registers and with the SM's shared memory, so that CTA 0 alone has
// 16 warps for the small chunks; the relaunch that takes over large levels
// runs two per SM at 64 registers for more loads in flight
constexpr uint32_t kFusedThreads = 512;
constexpr uint32_t kSolveThreads = 512;
constexpr uint32_t kSortMax = 2048;  // candidates of a chunk CTA 0 runs with shared-memory bookkeeping
static_assert(kMaxTeam < kSortMax, "the append's prefix table of per-CTA counts lives in sortbuf");
static_assert(kTreeScratchWords <= 2 * kSortMax, "the answer's tree is gathered in sortbuf");

__host__ __device__ size_t solve_smem_bytes(uint32_t W, uint32_t n, uint32_t G, uint32_t max_len,
                                            uint32_t seg_cap, bool gt_in_smem, uint32_t warps, uint32_t small_rows) {
    const uint32_t Ws = (W & 1u) ? W : W + 1;
    size_t b = sizeof(Seg) * seg_cap + sizeof(uint64_t) * (seg_cap + 1) + sizeof(SegTile) * seg_cap;
    b += sizeof(unsigned long long) * kSortMax;
    b += sizeof(uint32_t) * (2 * (kSortMax / 32) + 4);
    if (small_rows) b += sizeof(uint32_t) * ((size_t)small_rows * W + 2 * small_rows + (size_t)kSortMax * W);
    b += 2 * sizeof(uint32_t) * seg_cap;
    b += 2 * sizeof(uint32_t) * W;
    if (gt_in_smem) b += sizeof(uint32_t) * (((n + 1 + G + max_len + 2) + 3) & ~3u);
    b += 16;  // (the per-warp areas start on a 16-byte boundary)
    b += sizeof(uint32_t) * (size_t)warps * warp_words(W);
    (void)Ws;
    return b;
}

enum Cmd : uint32_t { CMD_NONE = 0, CMD_CHUNK = 1, CMD_EXIT = 2, CMD_CLEAN = 3 };

struct ChunkArgs {
    uint32_t level, size, dedup, nseg;
    uint64_t cs0, ce0;
};

// tiles of the chunk [cs0, ce0) in every segment; run by one whole warp
__device__ void tile_setup(Shared &S, uint32_t nseg, uint64_t cs0, uint64_t ce0, uint64_t *s_tiles, uint32_t bw) {
    const uint32_t lane = threadIdx.x & 31;
    uint64_t t = 0;
    for (uint32_t r0 = 0; r0 < nseg; r0 += 32) {
        const uint32_t s = r0 + lane;
        uint64_t tiles = 0;
        if (s < nseg) {
            const Seg &g = S.seg[s];
            // chunk [cs0, ce0) intersected with the segment, in segment-local
            // indices (empty when the segment lies wholly before or after it)
            const uint64_t g_end = g.start + g.size;
            const uint64_t a = cs0 <= g.start ? 0 : (cs0 >= g_end ? g.size : cs0 - g.start);
            const uint64_t e = ce0 <= g.start ? 0 : (ce0 >= g_end ? g.size : ce0 - g.start);
            SegTile &tl = S.tiles[s];
            tl.lo = a;
            tl.hi = e;
            tl.r0 = 0;
            tl.nb = 1;
            if (a < e) {
                if (g.op == OP_CAT || g.op == OP_ALT) {
                    // (32-bit division when the chunk's indices fit)
                    const bool narrow = e <= 0xFFFFFFFFull;
                    const uint64_t r0w = narrow ? (uint64_t)((uint32_t)a / g.rcnt) : a / g.rcnt;
                    const uint64_t r1 = narrow ? (uint64_t)((uint32_t)(e - 1) / g.rcnt) : (e - 1) / g.rcnt;
                    tl.r0 = r0w;
                    if (g.op == OP_CAT && g.swap) {
                        tl.nb = (uint32_t)((r1 - r0w + bw) / bw);
                        tiles = (uint64_t)g.rcnt * tl.nb;
                    } else {
                        tl.nb = (g.rcnt + bw - 1) / bw;
                        tiles = (r1 - r0w + 1) * tl.nb;
                    }
                } else {
                    tiles = (e - a + 31) / 32;
                }
            }
            if (tl.nb > 1) div_magic(tl.nb, tl.nb_mul, tl.nb_shift);
            else tl.nb_mul = 1, tl.nb_shift = 0;  // (x / 1 = (umulhi(1, x) + x) >> 0)
        }
        const uint64_t incl = warp_incl_scan(tiles, lane);
        if (s < nseg) S.tile_first[s] = t + incl - tiles;
        t += __shfl_sync(0xFFFFFFFFu, incl, 31);
    }
    if (lane == 0) {
        S.tile_first[nseg] = t;
        *s_tiles = t;
    }
    __syncwarp();
}

// the team's barrier: the grid barrier when every CTA works on the chunk,
// __syncthreads when CTA 0 works alone (global writes of a CTA are visible
// to its own threads after __syncthreads)
__device__ __forceinline__ bool team_barrier(bool full, SolveState *st, uint32_t &epoch, uint32_t site,
                                             uint32_t *trace, uint32_t team_n, uint32_t team_r) {
    if (full) return grid_barrier(st, epoch, site, trace, team_n, team_r);
    __syncthreads();
    return true;
}

// survivors of a chunk while the languages live in shared memory: as
// solo_append, with the holders read from the shared table; each survivor's
// row goes to the shared rows and to the global cache, its back-pointer to
// the global table of back-pointers
__device__ void smem_append(const SolveJob &J, Shared &S, const ChunkArgs &a, uint32_t W, Lead *L) {
    const uint32_t tid = threadIdx.x, nt = blockDim.x, lane = tid & 31;
    const uint32_t C = (uint32_t)(a.ce0 - a.cs0), nw = (C + 31) / 32;
    uint32_t *bits = S.solo_bits, *pref = S.solo_pref;
    const unsigned long long *ent = S.sortbuf;
    for (uint32_t xl = tid; xl < C; xl += nt) {
        if (!((bits[xl >> 5] >> (xl & 31)) & 1u)) continue;
        const uint32_t v = S.sm_table[(uint32_t)ent[xl]];
        if ((v & 0x1FFFFu) != (kSmPending | xl)) atomicAnd(&bits[xl >> 5], ~(1u << (xl & 31)));
    }
    __syncthreads();
    if (tid < 32) {
        const uint32_t c0 = 2 * lane < nw ? __popc(bits[2 * lane]) : 0u;
        const uint32_t c1 = 2 * lane + 1 < nw ? __popc(bits[2 * lane + 1]) : 0u;
        uint32_t x = c0 + c1;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, d);
            if (lane >= (uint32_t)d) x += y;
        }
        const uint32_t before = x - c0 - c1;
        if (2 * lane < nw) pref[2 * lane] = before;
        if (2 * lane + 1 < nw) pref[2 * lane + 1] = before + c0;
        if (lane == 31) pref[kSortMax / 32] = x;
    }
    __syncthreads();
    const uint32_t total = pref[kSortMax / 32];
    const uint64_t limit = J.cache_alloc < J.cap ? J.cache_alloc : J.cap;
    const uint64_t room = limit > a.size ? limit - a.size : 0;
    for (uint32_t xl = tid; xl < C; xl += nt) {
        const uint32_t wb = bits[xl >> 5];
        if (!((wb >> (xl & 31)) & 1u)) continue;
        const uint32_t rank = pref[xl >> 5] + __popc(wb & ((1u << (xl & 31)) - 1u));
        const uint32_t q = (uint32_t)ent[xl];
        if (rank >= room) {
            S.sm_table[q] = kSmEmpty;
            continue;
        }
        const uint32_t k = a.size + rank;
        const uint32_t *src = S.sm_tmp + xl * W;
        uint32_t *ds = S.sm_rows + k * W, *dg = J.cs + (uint64_t)k * W;
        for (uint32_t b = 0; b < W; b++) {
            const uint32_t x = src[b];
            ds[b] = x;
            dg[b] = x;
        }
        uint32_t op, l, r;
        decode(S.seg, a.nseg, J.leaf_sym, a.cs0 + xl, op, l, r);
        J.bp_op[k] = (uint8_t)op;
        J.bp_l[k] = l;
        J.bp_r[k] = r;
        S.sm_table[q] = (S.sm_table[q] & 0xFFFE0000u) | k;
    }
    __syncthreads();
    for (uint32_t w = tid; w < nw; w += nt) bits[w] = 0;
    if (tid == 0) {
        const uint64_t added = total < room ? total : room;
        if (total > room) L->full = 1;
        L->size = a.size + (uint32_t)added;
        S.lvc[a.level] = L->size - S.lvs[a.level];
        J.lvl_count[a.level] = S.lvc[a.level];
    }
    __syncthreads();
}

// leave the shared-memory start: every cached language goes into the global
// uniqueness table (all are distinct), so that other CTAs, later launches
// and the table cleanup see them
__device__ void switch_to_global(const SolveJob &J, Shared &S, Lead *L) {
    const uint32_t W = J.W, rows = L->size;
    REI_TSPAN_BEGIN(t_sw);
    for (uint32_t k = threadIdx.x; k < rows; k += blockDim.x) {
        const uint32_t *row = S.sm_rows + (uint64_t)k * W;
        const uint64_t h = cs_hash(row, W, 1);
        const unsigned long long v = J.exact ? exact_key(row, W) : ((uint64_t)(uint32_t)(h >> 32) << 32) | k;
        uint64_t p = J.direct ? v : h & J.table_mask;
        for (uint64_t probe = 0; probe <= J.table_mask; probe++) {
            if (atomicCAS(&J.table[p], kEmpty, v) == kEmpty) {
                J.used[k] = (uint32_t)p;
                break;
            }
            p = (p + 1) & J.table_mask;
        }
        if (J.seen) atomicOr(J.seen + (row[0] >> 5), 1u << (row[0] & 31u));
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) L->smode = 0;
    __syncthreads();
    REI_TSPAN_END(J.st, t_sw, 16);
}

// survivors of a small chunk CTA 0 ran alone, appended in candidate order: a
// marked candidate survives when its slot still names it (no later-marked
// candidate of the same language took the slot from it)
__device__ void solo_append(const SolveJob &J, SolveState *st, Shared &S, const ChunkArgs &a, uint32_t W,
                            Lead *L) {
    const uint32_t tid = threadIdx.x, nt = blockDim.x, lane = tid & 31;
    const uint32_t C = (uint32_t)(a.ce0 - a.cs0), nw = (C + 31) / 32;
    uint32_t *bits = S.solo_bits, *pref = S.solo_pref;
    const unsigned long long *ent = S.sortbuf;
    REI_TSTART();
    // 1. drop the marks that lost their slot (loads issued before any use)
    for (uint32_t base = 0; base < C; base += 8 * nt) {
        unsigned long long v[8];
        bool mk[8];
#pragma unroll
        for (int u = 0; u < 8; u++) {
            const uint32_t xl = base + u * nt + tid;
            mk[u] = xl < C && ((bits[xl >> 5] >> (xl & 31)) & 1u);
            v[u] = !mk[u] ? 0ull
                   : J.exact ? ld_relaxed_u32(J.minidx + (uint32_t)ent[xl])
                             : ld_relaxed_u64(J.table + (uint32_t)ent[xl]);
        }
#pragma unroll
        for (int u = 0; u < 8; u++) {
            const uint32_t xl = base + u * nt + tid;
            const uint32_t want = J.exact ? xl : (kPending | xl);
            if (mk[u] && (uint32_t)v[u] != want) atomicAnd(&bits[xl >> 5], ~(1u << (xl & 31)));
        }
    }
    __syncthreads();
    REI_TMARK(true, 3);
    // 2. survivors before each bitmap word (nw <= 64: two words per lane of warp 0)
    if (tid < 32) {
        const uint32_t c0 = 2 * lane < nw ? __popc(bits[2 * lane]) : 0u;
        const uint32_t c1 = 2 * lane + 1 < nw ? __popc(bits[2 * lane + 1]) : 0u;
        uint32_t x = c0 + c1;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, d);
            if (lane >= (uint32_t)d) x += y;
        }
        const uint32_t before = x - c0 - c1;
        if (2 * lane < nw) pref[2 * lane] = before;
        if (2 * lane + 1 < nw) pref[2 * lane + 1] = before + c0;
        if (lane == 31) pref[kSortMax / 32] = x;
    }
    __syncthreads();
    REI_TMARK(true, 4);
    // 3. rows, back-pointers and slots of the survivors; beyond the cache's
    // room they are not cached and their slots are emptied
    const uint32_t total = pref[kSortMax / 32];
    const uint64_t limit = J.cache_alloc < J.cap ? J.cache_alloc : J.cap;
    const uint64_t room = limit > a.size ? limit - a.size : 0;
    for (uint32_t xl = tid; xl < C; xl += nt) {
        const uint32_t wb = bits[xl >> 5];
        if (!((wb >> (xl & 31)) & 1u)) continue;
        const uint32_t rank = pref[xl >> 5] + __popc(wb & ((1u << (xl & 31)) - 1u));
        const unsigned long long e = ent[xl];
        const uint32_t q = (uint32_t)e;
        if (rank >= room) {
            J.table[q] = kEmpty;
            if (J.exact) J.minidx[q] = 0xFFFFFFFFu;
            continue;
        }
        const uint64_t k = (uint64_t)a.size + rank;
        uint32_t *dst = J.cs + k * W;
        if (J.exact) {
            // the language is the slot's key
            const unsigned long long key = ld_relaxed_u64(J.table + q) & ~kXPend;
            dst[0] = (uint32_t)key;
            if (W == 2) dst[1] = (uint32_t)(key >> 32);
            J.table[q] = key;
            J.minidx[q] = 0xFFFFFFFFu;
            if (J.seen) atomicOr(J.seen + ((uint32_t)key >> 5), 1u << (key & 31u));
        } else {
            const uint32_t *srcp = J.tmp + (uint64_t)xl * W;
            for (uint32_t b = 0; b < W; b++) dst[b] = ldcg(srcp + b);
            J.table[q] = (e & 0xFFFFFFFF00000000ull) | (uint32_t)k;
        }
        uint32_t op, l, r;
        decode(S.seg, a.nseg, J.leaf_sym, a.cs0 + xl, op, l, r);
        J.bp_op[k] = (uint8_t)op;
        J.bp_l[k] = l;
        J.bp_r[k] = r;
        J.used[k] = q;
    }
    __syncthreads();
    for (uint32_t w = tid; w < nw; w += nt) bits[w] = 0;
    if (tid == 0) {
        const uint64_t added = total < room ? total : room;
        if (total > room) L->full = 1;
        L->size = a.size + (uint32_t)added;
        S.lvc[a.level] = L->size - S.lvs[a.level];
        J.lvl_count[a.level] = S.lvc[a.level];
    }
    __syncthreads();
    REI_TMARK(true, 5);
}

// a chunk with at least this many tiles per warp hands its tiles out
// dynamically, kGrab at a time
constexpr uint32_t kDynTilesPerWarp = 32;
constexpr uint32_t kGrab = 4;

// one chunk of candidates; returns 1 when a precise candidate was found in it,
// 0 when done, -1 when a grid barrier gave up
__device__ int process_chunk(const SolveJob &J, SolveState *st, Shared &S, const ChunkArgs &a, bool full,
                             bool tiles_ready, uint32_t &bar_epoch, uint64_t *s_tiles, uint32_t *s_red,
                             unsigned long long *s_found, uint32_t *s_npend, uint32_t *wm, Lead *L) {
    const uint32_t W = J.W, n = J.n;
    const uint32_t Ws = (W & 1u) ? W : W + 1;
    const uint32_t tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const uint32_t nwarps = blockDim.x >> 5;
    const uint32_t team_n = full ? team_size_of(J) : 1, team_r = full ? team_rank_of(J) : 0;
    const bool dedup = a.dedup != 0;
    REI_TSTART();

    if (!tiles_ready) {
        if (wid == 0) tile_setup(S, a.nseg, a.cs0, a.ce0, s_tiles, bin_block(W));
        __syncthreads();
    }

    // a small chunk CTA 0 runs alone keeps its bookkeeping in shared memory;
    // at the search's start the languages and their table live there too
    const bool small = !full && a.ce0 - a.cs0 <= kSortMax;
    const bool sm = small && L && L->smode;
    if (small && !tiles_ready) {
        if (tid == 0) *s_found = kNone;
        __syncthreads();
    }

    // ---- phase A: build, precision, uniqueness insert
    {
        TileCtx TC{&J, st, &S, a.cs0, W, Ws, n, dedup, full, small ? s_found : &st->found,
                   small ? S.sortbuf : nullptr, small ? S.solo_bits : nullptr, sm ? S.sm_rows : J.cs, sm};
        // (a chunk's tiles, at most 2^26 / 32 plus one per segment, fit 32 bits)
        const uint32_t ntiles = (uint32_t)*s_tiles;
        const uint32_t gw = team_r * nwarps + wid, nw = team_n * nwarps;
        uint32_t s = 0;
        // many tiles per warp: hand them out kGrab at a time from a counter,
        // so that every warp ends within a few tiles of the others (the
        // order of tiles does not change any result); the next grab is in
        // flight while the warp works on the current one.  Else tile t goes
        // to warp t mod (warps of the team).
        const bool dyn = full && ntiles >= kDynTilesPerWarp * nw;
        // (1-word languages: longer runs of tiles that share an operand, whose
        // lookup tables are then built once per run)
        const uint32_t grab = W == 1 ? 4 * kGrab : kGrab;
        uint32_t t = gw, end = ntiles, step = nw;
        uint32_t nxt = 0;
#ifdef REI_TIMING
        __shared__ unsigned long long s_wmax;
        if (tid == 0) s_wmax = 0;
        __syncthreads();
        const unsigned long long t_loop0 = globaltimer_ns();
        if (!full && tid == 0) st->t_sub[25] += t_loop0 - t_mark0;
        if (!full && tid == 0) st->t_sub[24] += ntiles;
        if (full && tid == 0) atomicMax((unsigned long long *)&st->t_sub[45], t_loop0 - ld_relaxed_u64(&st->t_sub[47]));
#endif
        if (dyn) {
            uint32_t cur = 0;
            if (lane == 0) cur = atomicAdd(&st->tile_next, grab);
            t = __shfl_sync(0xFFFFFFFFu, cur, 0);
            end = min(t + grab, ntiles);
            step = 1;
            if (lane == 0 && t < ntiles) nxt = atomicAdd(&st->tile_next, grab);
        }
        while (t < ntiles) {
            while (s + 1 < a.nseg && S.tile_first[s + 1] <= t) s++;
            const SegTile &tl = S.tiles[s];
            if (tl.lo < tl.hi) {
#ifdef REI_TIMING
                const unsigned long long t_tile0 = globaltimer_ns();
#endif
                if (W == 1) run_tile_w1(TC, S.seg[s], tl, t - S.tile_first[s], wm);
                else if (W == 2) run_tile<2>(TC, S.seg[s], tl, t - S.tile_first[s], wm);
                else run_tile<0>(TC, S.seg[s], tl, t - S.tile_first[s], wm);
                __syncwarp();
#ifdef REI_TIMING
                if (!full && lane == 0) {
                    atomicAdd((unsigned long long *)&st->t_sub[26 + S.seg[s].op], globaltimer_ns() - t_tile0);
                    atomicAdd((unsigned long long *)&st->t_sub[32 + S.seg[s].op], 1ull);
                }
#endif
            }
            t += step;
            if (dyn && t >= end) {
                t = __shfl_sync(0xFFFFFFFFu, nxt, 0);
                end = min(t + grab, ntiles);
                if (lane == 0 && t < ntiles) nxt = atomicAdd(&st->tile_next, grab);
            }
        }
#ifdef REI_TIMING
        if (lane == 0) atomicMax(&s_wmax, globaltimer_ns() - t_loop0);
        __syncthreads();
        if (!full && tid == 0) st->t_sub[23] += s_wmax;
        if (full && tid == 0) {
            atomicMax((unsigned long long *)&st->t_sub[46], s_wmax);
            atomicMax((unsigned long long *)&st->t_sub[44], globaltimer_ns() - ld_relaxed_u64(&st->t_sub[47]));
            if (blockIdx.x == 0) st->t_sub[37] += s_wmax;
        }
#endif
    }
    if (!team_barrier(full, st, bar_epoch, 5, J.trace, team_n, team_r)) return -1;
#ifdef REI_TIMING
    if (full && blockIdx.x == 0 && tid == 0) {
        st->t_sub[39] += globaltimer_ns() - ld_relaxed_u64(&st->t_sub[47]);
        st->t_sub[41] += ld_relaxed_u64(&st->t_sub[45]);
        st->t_sub[42] += ld_relaxed_u64(&st->t_sub[46]);
        st->t_sub[43] += ld_relaxed_u64(&st->t_sub[44]);
        st->t_sub[44] = st->t_sub[45] = st->t_sub[46] = 0;
    }
#endif
    REI_TMARK(!full, 0);
    REI_TMARK(full && blockIdx.x == 0, 12);
    if (small) {
        const unsigned long long f = *s_found;
        if (f != kNone) {
            // the answer is in this chunk: its survivors are not cached, so
            // the slots they took are emptied now
            const uint32_t C = (uint32_t)(a.ce0 - a.cs0);
            if (!sm)
                for (uint32_t xl = tid; xl < C; xl += blockDim.x)
                    if ((S.solo_bits[xl >> 5] >> (xl & 31)) & 1u) {
                        const uint32_t q = (uint32_t)S.sortbuf[xl];
                        J.table[q] = kEmpty;
                        if (J.exact) J.minidx[q] = 0xFFFFFFFFu;
                    }
            __syncthreads();
            for (uint32_t w = tid; w < kSortMax / 32; w += blockDim.x) S.solo_bits[w] = 0;
            if (tid == 0) st->found = f;
            __syncthreads();
            return 1;
        }
        if (dedup) {
            if (sm) smem_append(J, S, a, W, L);
            else solo_append(J, st, S, a, W, L);
        }
        REI_TMARK(!full, 2);
        return 0;
    }
    if (tid == 0) {
        *s_found = ld_relaxed_u64(&st->found);
        *s_npend = ld_relaxed_u32(&st->pending_count);
    }
    __syncthreads();
    REI_TMARK(!full, 1);
    if (*s_found != kNone) return 1;
    if (!dedup) return 0;
    const uint32_t npend = *s_npend;
    __syncthreads();

    // no new language: nothing to append
    if (npend == 0) return 0;

    // ---- phase B: survivors are the slot holders of new languages
    const uint64_t C = a.ce0 - a.cs0;
    {
        const uint64_t gt = (uint64_t)team_r * blockDim.x + tid, nt = (uint64_t)team_n * blockDim.x;
        for (uint64_t i = gt; i < npend; i += nt) {
            const uint32_t q = ldcg(J.pending + i);
            const uint32_t j = J.exact ? ld_relaxed_u32(J.minidx + q) : (uint32_t)ld_relaxed_u64(J.table + q) & ~kPending;
            atomicOr(&J.bitmap[j >> 5], 1u << (j & 31));
            J.slotpos[j] = q;
        }
    }
    if (!team_barrier(full, st, bar_epoch, 7, J.trace, team_n, team_r)) return -1;
    REI_TMARK(full && blockIdx.x == 0, 13);

    // ---- phase C: survivors per CTA (contiguous word ranges of the bitmap),
    // counted, then listed in order into pending[] over the CTA's own range
    // of candidates (phase B has read the pending list; the k-th survivor of
    // a range starting at candidate w0 * 32 is a candidate >= w0 * 32 + k, so
    // the lists stay inside their ranges); the bitmap is cleared on the way.
    // Each warp takes a contiguous part of the CTA's range and reads it 32
    // consecutive words at a time: counted first, then listed with a warp scan.
    const uint64_t nwords = (C + 31) / 32;
    const uint64_t per_cta = (nwords + team_n - 1) / team_n;
    const uint64_t w0 = umin64(nwords, team_r * per_cta);
    const uint64_t w1 = umin64(nwords, w0 + per_cta);
    {
        const uint64_t per_warp = (w1 - w0 + nwarps - 1) / nwarps;
        const uint64_t a0 = umin64(w1, w0 + wid * per_warp), a1 = umin64(w1, a0 + per_warp);
        uint32_t wcnt = 0;
        for (uint64_t w = a0 + lane; w < a1; w += 32) wcnt += __popc(ldcg(J.bitmap + w));
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) wcnt += __shfl_xor_sync(0xFFFFFFFFu, wcnt, d);
        if (lane == 0) s_red[wid] = wcnt;
        __syncthreads();
        uint32_t wbefore = 0, cta_cnt = 0;
        for (uint32_t k = 0; k < nwarps; k++) {
            if (k < wid) wbefore += s_red[k];
            cta_cnt += s_red[k];
        }
        uint32_t *out = J.pending + w0 * 32;
        uint32_t pos = wbefore;
        for (uint64_t base = a0; base < a1 && wcnt; base += 32) {
            const uint64_t w = base + lane;
            uint32_t bits = w < a1 ? ldcg(J.bitmap + w) : 0u;
            const uint32_t cnt = __popc(bits);
            uint32_t incl = cnt;
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, incl, d);
                if (lane >= (uint32_t)d) incl += y;
            }
            if (bits) {
                J.bitmap[w] = 0;
                uint32_t p = pos + incl - cnt;
                while (bits) {
                    out[p++] = (uint32_t)(w * 32 + (__ffs(bits) - 1));
                    bits &= bits - 1;
                }
            }
            pos += __shfl_sync(0xFFFFFFFFu, incl, 31);
        }
        if (tid == 0) J.blk[team_r] = cta_cnt;
        __syncthreads();
    }
    if (team_r == 0 && tid == 0) st->pending_count = 0;
    if (!team_barrier(full, st, bar_epoch, 8, J.trace, team_n, team_r)) return -1;
    REI_TMARK(full && blockIdx.x == 0, 14);

    // ---- phase D: append survivors in candidate order.  Survivor g (of all
    // the chunk's, in order) is the (g - pref[b])-th of CTA range b's list;
    // every CTA appends an equal share of the ranks, however unevenly the
    // new languages fall over the ranges.
    {
        uint32_t *pref = reinterpret_cast<uint32_t *>(S.sortbuf);  // team_n + 1 entries (team_n < kSortMax)
        uint32_t *list = pref + kSortMax;                          // kSortMax candidates per round
        for (uint32_t b = tid; b < team_n; b += blockDim.x) pref[b + 1] = ldcg(J.blk + b);
        if (tid == 0) pref[0] = 0;
        __syncthreads();
        if (wid == 0) {
            uint32_t carry = 0;
            for (uint32_t b0 = 1; b0 <= team_n; b0 += 32) {
                const uint32_t b = b0 + lane;
                const uint32_t v = b <= team_n ? pref[b] : 0u;
                uint32_t x = v;
                for (int d = 1; d < 32; d <<= 1) {
                    const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, d);
                    if (lane >= (uint32_t)d) x += y;
                }
                if (b <= team_n) pref[b] = carry + x;
                carry += __shfl_sync(0xFFFFFFFFu, x, 31);
            }
        }
        __syncthreads();
        const uint64_t total = pref[team_n];
        const uint64_t g0 = total * team_r / team_n, g1 = total * (team_r + 1) / team_n;
        const uint64_t limit = J.cache_alloc < J.cap ? J.cache_alloc : J.cap;
        const uint32_t nt = blockDim.x;
        for (uint64_t lo = g0; lo < g1; lo += kSortMax) {
            const uint32_t cnt = (uint32_t)umin64(kSortMax, g1 - lo);
            // the round's candidates: rank g -> its range b (the last b with pref[b] <= g)
            for (uint32_t i = tid; i < cnt; i += nt) {
                const uint32_t g = (uint32_t)(lo + i);
                uint32_t b = 0, hi_b = team_n;  // pref[b] <= g < pref[hi_b]
                while (hi_b - b > 1) {
                    const uint32_t m = (b + hi_b) >> 1;
                    if (pref[m] <= g) b = m;
                    else hi_b = m;
                }
                const uint64_t bw0 = umin64(nwords, b * per_cta);
                list[i] = ldcg(J.pending + bw0 * 32 + (g - pref[b]));
            }
            __syncthreads();
            const uint64_t b0 = (uint64_t)a.size + lo;  // cache row of the round's first survivor
            const uint32_t nfit = b0 >= limit ? 0u : (uint32_t)umin64(cnt, limit - b0);
            const uint32_t nf = J.exact ? 0u : nfit * W;  // (exact keys: rows from the keys)
            for (uint32_t f0 = tid; f0 < nf; f0 += 4 * nt) {
                uint32_t v[4];
#pragma unroll
                for (int u = 0; u < 4; u++) {
                    const uint32_t f = f0 + u * nt;
                    if (f < nf) {
                        const uint32_t i = f / W, b = f - i * W;
                        v[u] = ldcg(J.tmp + (uint64_t)list[i] * W + b);
                    }
                }
#pragma unroll
                for (int u = 0; u < 4; u++) {
                    const uint32_t f = f0 + u * nt;
                    if (f < nf) {
                        const uint32_t i = f / W, b = f - i * W;
                        J.cs[(b0 + i) * W + b] = v[u];
                    }
                }
            }
            for (uint32_t i0 = tid; i0 < cnt; i0 += 4 * nt) {
                uint32_t q[4];
                unsigned long long old[4];
#pragma unroll
                for (int u = 0; u < 4; u++) {
                    const uint32_t i = i0 + u * nt;
                    if (i < cnt) q[u] = ldcg(J.slotpos + list[i]);
                }
#pragma unroll
                for (int u = 0; u < 4; u++) {
                    const uint32_t i = i0 + u * nt;
                    if (i < nfit) old[u] = ld_relaxed_u64(J.table + q[u]);
                }
#pragma unroll
                for (int u = 0; u < 4; u++) {
                    const uint32_t i = i0 + u * nt;
                    if (i >= cnt) continue;
                    if (i >= nfit) {
                        J.table[q[u]] = kEmpty;  // not cached: free the slot
                        if (J.exact) J.minidx[q[u]] = 0xFFFFFFFFu;
                        continue;
                    }
                    const uint64_t k = b0 + i;
                    uint32_t op, l, r;
                    decode(S.seg, a.nseg, J.leaf_sym, a.cs0 + list[i], op, l, r);
                    J.bp_op[k] = (uint8_t)op;
                    J.bp_l[k] = l;
                    J.bp_r[k] = r;
                    if (J.exact) {
                        const unsigned long long key = old[u] & ~kXPend;
                        J.cs[k * W] = (uint32_t)key;
                        if (W == 2) J.cs[k * W + 1] = (uint32_t)(key >> 32);
                        J.table[q[u]] = key;
                        J.minidx[q[u]] = 0xFFFFFFFFu;
                        if (J.seen) atomicOr(J.seen + ((uint32_t)key >> 5), 1u << (key & 31u));
                    } else {
                        J.table[q[u]] = (old[u] & 0xFFFFFFFF00000000ull) | (uint32_t)k;
                    }
                    J.used[k] = q[u];
                }
            }
            __syncthreads();  // (the list is refilled next round)
        }
        if (team_r == 0 && tid == 0) {
            const uint64_t room = limit > a.size ? limit - a.size : 0;
            const uint64_t added = total < room ? total : room;
            if (total > room) L->full = 1;  // every drop shows as total > room
            L->size = a.size + (uint32_t)added;
            S.lvc[a.level] = L->size - S.lvs[a.level];
            J.lvl_count[a.level] = S.lvc[a.level];
        }
    }
    if (!team_barrier(full, st, bar_epoch, 9, J.trace, team_n, team_r)) return -1;
    REI_TMARK(full && blockIdx.x == 0, 15);
    return 0;
}

// a team chunk's plan (segments, their tiles in the chunk, first tiles), as
// CTA 0 made it, for the other CTAs: written before the command that names
// the chunk, read with it
static_assert(sizeof(Seg) % 8 == 0 && sizeof(SegTile) == 40, "plan words");
__device__ void write_plan(const SolveJob &J, const Shared &S, uint32_t nseg, uint64_t ntiles) {
    const uint32_t sw = sizeof(Seg) / 8, tw = sizeof(SegTile) / 8;
    uint64_t *P = J.plan;
    if (threadIdx.x == 0) {
        P[0] = nseg;
        P[1] = ntiles;
    }
    const uint64_t *seg = reinterpret_cast<const uint64_t *>(S.seg);
    const uint64_t *til = reinterpret_cast<const uint64_t *>(S.tiles);
    for (uint32_t i = threadIdx.x; i < nseg * sw; i += blockDim.x) P[2 + i] = seg[i];
    for (uint32_t i = threadIdx.x; i < nseg * tw; i += blockDim.x) P[2 + J.seg_cap * sw + i] = til[i];
    for (uint32_t i = threadIdx.x; i <= nseg; i += blockDim.x) P[2 + J.seg_cap * (sw + tw) + i] = S.tile_first[i];
}

__device__ void read_plan(const SolveJob &J, Shared &S, uint64_t *s_tiles, uint32_t *s_nseg) {
    const uint32_t sw = sizeof(Seg) / 8, tw = sizeof(SegTile) / 8, cap = J.seg_cap;
    const uint64_t *P = J.plan;
    uint64_t *seg = reinterpret_cast<uint64_t *>(S.seg);
    uint64_t *til = reinterpret_cast<uint64_t *>(S.tiles);
    if (threadIdx.x == 0) {
        *s_nseg = (uint32_t)ld_relaxed_u64(P);
        *s_tiles = ld_relaxed_u64(P + 1);
    }
    for (uint32_t i = threadIdx.x; i < cap * sw; i += blockDim.x) seg[i] = ld_relaxed_u64(P + 2 + i);
    for (uint32_t i = threadIdx.x; i < cap * tw; i += blockDim.x) til[i] = ld_relaxed_u64(P + 2 + cap * sw + i);
    for (uint32_t i = threadIdx.x; i <= cap; i += blockDim.x) S.tile_first[i] = ld_relaxed_u64(P + 2 + cap * (sw + tw) + i);
}

// CTA 0 publishes a command (release); the workers pick it up (acquire)
__device__ void publish(SolveState *st, uint32_t cmd) {
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();  // (after the barrier: covers every thread's writes)
        st->cmd = cmd;
        __threadfence();
        atomicAdd(&st->cmd_seq, 1u);
    }
    __syncthreads();
}

constexpr unsigned long long kWorkerWaitNs = 20000000000ull;  // a worker waits at most 20 s for work


// the shared memory of a search CTA, carved for one staged problem
__device__ void carve_shared(const SolveJob &J, Shared &S, uint8_t *smem_raw, uint32_t **wm_out) {
    const uint32_t W = J.W, n = J.n;
    const uint32_t Ws = (W & 1u) ? W : W + 1;
    const uint32_t tid = threadIdx.x, wid = tid >> 5;
    uint8_t *p = smem_raw;
    S.seg = reinterpret_cast<Seg *>(p);
    p += sizeof(Seg) * J.seg_cap;
    S.tile_first = reinterpret_cast<uint64_t *>(p);
    p += sizeof(uint64_t) * (J.seg_cap + 1);
    S.tiles = reinterpret_cast<SegTile *>(p);
    p += sizeof(SegTile) * J.seg_cap;
    S.sortbuf = reinterpret_cast<unsigned long long *>(p);
    p += sizeof(unsigned long long) * kSortMax;
    S.solo_bits = reinterpret_cast<uint32_t *>(p);
    p += sizeof(uint32_t) * (kSortMax / 32);
    S.solo_pref = reinterpret_cast<uint32_t *>(p);
    p += sizeof(uint32_t) * (kSortMax / 32 + 4);
    S.sm_rows = S.sm_table = S.sm_tmp = nullptr;
    if (J.small_rows) {
        S.sm_rows = reinterpret_cast<uint32_t *>(p);
        p += sizeof(uint32_t) * J.small_rows * W;
        S.sm_table = reinterpret_cast<uint32_t *>(p);
        p += sizeof(uint32_t) * 2 * J.small_rows;
        S.sm_tmp = reinterpret_cast<uint32_t *>(p);
        p += sizeof(uint32_t) * kSortMax * W;
    }
    for (uint32_t i = tid; i < kSortMax / 32; i += blockDim.x) S.solo_bits[i] = 0;
    S.lvs = reinterpret_cast<uint32_t *>(p);
    p += sizeof(uint32_t) * J.seg_cap;
    S.lvc = reinterpret_cast<uint32_t *>(p);
    p += sizeof(uint32_t) * J.seg_cap;
    S.pos = reinterpret_cast<uint32_t *>(p);
    p += sizeof(uint32_t) * W;
    S.neg = reinterpret_cast<uint32_t *>(p);
    p += sizeof(uint32_t) * W;
    if (J.gt_in_smem) {
        uint32_t *g = reinterpret_cast<uint32_t *>(p);
        for (uint32_t i = tid; i <= n; i += blockDim.x) g[i] = J.gt_off[i];
        for (uint32_t i = tid; i < J.G; i += blockDim.x) g[n + 1 + i] = J.gt_pair[i];
        for (uint32_t i = tid; i < J.max_len + 2; i += blockDim.x) g[n + 1 + J.G + i] = J.len_start[i];
        S.gt_off = g;
        S.gt_pair = g + n + 1;
        S.len_start = g + n + 1 + J.G;
        p += sizeof(uint32_t) * (((n + 1 + J.G + J.max_len + 2) + 3) & ~3u);
    } else {
        S.gt_off = J.gt_off;
        S.gt_pair = J.gt_pair;
        S.len_start = J.len_start;
    }
    p = smem_raw + ((size_t)(p - smem_raw + 15) & ~size_t(15));
    S.warp_words = warp_words(W);
    S.warp_mem = reinterpret_cast<uint32_t *>(p);
    (void)Ws;
    // no concatenation tables built yet (1-word languages)
    if (W == 1)
        for (uint32_t w = tid; w < blockDim.x / 32; w += blockDim.x) S.warp_mem[w * S.warp_words + kW1TabAt + kW1Tab] = kNoOperand;
    for (uint32_t b = tid; b < W; b += blockDim.x) {
        S.pos[b] = J.pos_mask[b];
        S.neg[b] = J.neg_mask[b];
    }
    // the level table as left by earlier launches of this search (parallel loads)
    for (uint32_t c = tid; c <= J.max_cost + 1 && c < J.seg_cap; c += blockDim.x) {
        S.lvs[c] = (uint32_t)ld_relaxed_u64(&J.lvl_start[c]);
        S.lvc[c] = (uint32_t)ld_relaxed_u64(&J.lvl_count[c]);
    }
    *wm_out = S.warp_mem + wid * S.warp_words;
    __syncthreads();
}

// per-CTA static scratch the search functions share
struct Cta {
    Plan *plan;
    uint32_t *red;
    uint64_t *tiles;
    unsigned long long *found;
    uint32_t *npend;
    Lead *L;
    uint32_t *wm;
};

// Empty every table slot this search filled, so that the table can be reused
// without clearing it: the slot of every cached row, and the pending slots of
// a chunk that ended with the answer before its survivors were appended.
__device__ void clean_table(const SolveJob &J, uint32_t rows, uint32_t npending, uint32_t team_n,
                            uint32_t team_r) {
    const uint64_t t = (uint64_t)team_r * blockDim.x + threadIdx.x, nt = (uint64_t)team_n * blockDim.x;
    for (uint64_t k = t; k < rows; k += nt) J.table[ldcg(J.used + k)] = kEmpty;
    // the seen bitmap holds bits of cached languages only: zero every word
    // that holds one
    if (J.seen)
        for (uint64_t k = t; k < rows; k += nt) J.seen[ldcg(J.cs + k) >> 5] = 0u;
    for (uint64_t i = t; i < npending; i += nt) {
        const uint32_t q = ldcg(J.pending + i);
        J.table[q] = kEmpty;
        if (J.exact) J.minidx[q] = 0xFFFFFFFFu;
    }
}

// The leader's search loop (Alg. 1): level after level, chunk after chunk,
// until the answer, not_found, out-of-memory, or a request for more memory.
// With allow_team, large chunks are handed to every CTA of the launch.
// Returns -1 when a grid barrier gave up, else 0; the final state is written
// back to `st`.
__device__ int lead_search(const SolveJob &J, SolveState *st, Shared &S, const Cta &K, bool allow_team,
                           uint32_t &bar_epoch) {
    const uint32_t tid = threadIdx.x, wid = tid >> 5;
    Lead &L = *K.L;
    Plan &s_plan = *K.plan;
    REI_TSPAN_BEGIN(t_init);
    if (tid == 0) {
        L.cleaned = 0;
        L.status = st->status;
        L.level = st->level;
        L.size = st->size;
        L.full = st->full;
        L.otf = st->otf;
        L.partial_level = st->partial_level;
        L.chunk_pos = st->chunk_pos;
        L.candidates = st->candidates;
        L.unique_done = st->unique_done;
        for (int k = 0; k < 5; k++) L.cand_op[k] = st->cand_op[k];
        // a fresh search starts with its languages in shared memory
        L.smode = J.small_rows && L.status == ST_RUNNING && L.level == J.cmin && L.chunk_pos == 0 && L.size == 0;
        // trivial specifications (Alg. 1): the empty set, then eps
        if (L.status == ST_RUNNING && L.level == J.cmin && L.chunk_pos == 0 && L.size == 0) {
            const uint32_t e_empty = J.n_pos_set;
            const uint32_t e_eps = J.n_pos_set - J.pos_eps + J.neg_eps;
            if (e_empty <= J.max_errors || e_eps <= J.max_errors) {
                J.tree[0] = e_empty <= J.max_errors ? '0' : 'e';
                J.tree[1] = 0;
                st->tree_len = 1;
                st->ans_cost = J.c[0];
                L.candidates = 0;
                L.status = ST_FOUND;
                st->found = kNone;
            }
        }
    }
    __syncthreads();
    if (L.smode)
        for (uint32_t i = tid; i < 2 * J.small_rows; i += blockDim.x) S.sm_table[i] = kSmEmpty;
    __syncthreads();
    REI_TSPAN_END(st, t_init, 17);

    bool found = false;
    uint32_t planned = 0xFFFFFFFFu;  // the level whose plan is in S.seg / s_plan
    // end of a level (thread 0): count it, check the cache cap, enter the next one
    auto end_level = [&](uint32_t level, uint32_t nseg) {
        uint64_t vc = 0;
        for (uint32_t s = 0; s < nseg; s++) {
            const uint64_t v = valid_count(S.seg[s]);
            vc += v;
            L.cand_op[S.seg[s].op] += v;
        }
        L.candidates += vc;
        uint32_t next_status = ST_RUNNING;
        if (!L.otf) {
            if (L.full) {
                if (J.flags & REI_F_ONTHEFLY) {
                    L.otf = 1;
                    L.partial_level = level;
                } else {
                    next_status = ST_OOM;
                }
            } else {
                L.unique_done = L.size;
            }
        }
        const uint32_t nl = level + 1;
        if (next_status == ST_RUNNING) {
            if (nl > J.max_cost) {
                next_status = ST_NOT_FOUND;
            } else {
                S.lvs[nl] = L.size;
                S.lvc[nl] = 0;
                J.lvl_start[nl] = L.size;
                J.lvl_count[nl] = 0;
                if (L.otf && max_operand_level(J, (int)nl) >= (int)L.partial_level) next_status = ST_OOM;
            }
        }
        L.level = next_status == ST_RUNNING ? nl : level;
        L.chunk_pos = 0;
        L.full = 0;
        L.status = next_status;
    };
    // per-phase wall time of the leader (ns): plan, solo chunk, team chunk, level end
    unsigned long long tm[4] = {0, 0, 0, 0}, tcnt[3] = {0, 0, 0};
    for (;;) {
        const unsigned long long t_it = globaltimer_ns();
        const uint32_t status = L.status, level = L.level, size = L.size, full = L.full, otf = L.otf;
        const uint64_t pos = L.chunk_pos;
        __syncthreads();
        if (status != ST_RUNNING) break;
        if (level > J.max_cost) {
            // no level left (also when c_sym > max_cost): Alg. 1 "not_found"
            if (tid == 0) L.status = ST_NOT_FOUND;
            __syncthreads();
            continue;
        }
        // a level's plan depends on lower levels only: once per level
        if (level != planned) {
            REI_TSPAN_BEGIN(t_pl);
            if (wid == 0) plan_level(J, level, S.lvs, S.lvc, S.seg, s_plan);
            __syncthreads();
            planned = level;
            REI_TSPAN_END(st, t_pl, 18);
        }
        const uint32_t nseg = s_plan.nseg;
        const uint64_t T = s_plan.total;

        if (pos >= T) {
            if (tid == 0) {
                end_level(level, nseg);
                tm[3] += globaltimer_ns() - t_it;
                tcnt[2]++;
            }
            __syncthreads();
            continue;
        }

        // a level larger than `handover` candidates goes to the relaunch
        // (a launch shaped for throughput), which continues from here
        if (J.handover && pos == 0 && T > J.handover && size > 0) {
            if (L.smode) switch_to_global(J, S, &L);
            if (tid == 0) {
                st->need_rows = size;
                L.status = ST_NEED_MEM;
            }
            __syncthreads();
            continue;
        }
        // a search on one CTA past its time allowance goes back to the host
        if (J.yield_ns) {
            if (tid == 0 && globaltimer_ns() - J.t_start > J.yield_ns) L.status = ST_NEED_MEM;
            __syncthreads();
            if (L.status == ST_NEED_MEM) continue;
        }
        // chunk [pos, pos + C) of the level
        const bool dedup = !full && !otf;
        uint64_t C = T - pos;
        if (C > J.chunk_max) C = J.chunk_max;
        // (no more than 2^|ic| distinct languages exist: a cache that holds
        // that many, or the budget's cap, never runs out of room in a chunk)
        const uint64_t ceil_rows = J.n < 63 ? umin64(J.cap, 1ull << J.n) : J.cap;
        if (dedup && J.cache_alloc < ceil_rows) {
            const uint64_t room = J.cache_alloc - size;
            if (room < C) {
                if (room * 4 >= J.chunk_max || room >= T - pos) {
                    C = room;
                } else {
                    // the next launch continues from the global tables
                    if (L.smode) switch_to_global(J, S, &L);
                    if (tid == 0) {
                        st->need_rows = (uint32_t)umin64(ceil_rows, (uint64_t)size + C);
                        L.status = ST_NEED_MEM;
                    }
                    __syncthreads();
                    continue;
                }
            }
        }
        if (C == 0) C = 1;  // unreachable with room >= 1; guards the loop
        ChunkArgs a{level, size, dedup ? 1u : 0u, nseg, pos, pos + C};
        // alone when the chunk is a few tiles per warp of this CTA
        REI_TSPAN_BEGIN(t_ts);
        if (wid == 0) tile_setup(S, nseg, a.cs0, a.ce0, K.tiles, bin_block(J.W));
        if (tid == 0) *K.found = kNone;  // a small chunk's answer slot
        __syncthreads();
        REI_TSPAN_END(st, t_ts, 19);
        const bool team = allow_team && *K.tiles > (uint64_t)J.solo_tiles;
        // the shared-memory start ends before a chunk it cannot hold
        if (L.smode && (team || !dedup || C > kSortMax || (uint64_t)size + C > J.small_rows))
            switch_to_global(J, S, &L);
        const unsigned long long t_chunk = globaltimer_ns();
        if (tid == 0) tm[0] += t_chunk - t_it;
        if (team) {
            if (tid == 0) {
                st->tile_next = 0;  // (every CTA left the previous chunk's tiles at its barriers)
                st->c_level = a.level;
                st->c_size = a.size;
                st->c_dedup = a.dedup;
                st->c_cs0 = a.cs0;
                st->c_ce0 = a.ce0;
            }
#ifdef REI_TIMING
            if (tid == 0) st->t_sub[47] = globaltimer_ns();
#endif
            if (J.plan) write_plan(J, S, nseg, *K.tiles);
            publish(st, CMD_CHUNK);
#ifdef REI_TIMING
            if (tid == 0) st->t_sub[40] += globaltimer_ns() - st->t_sub[47];
#endif
        }
        const int r = process_chunk(J, st, S, a, team, true, bar_epoch, K.tiles, K.red, K.found, K.npend, K.wm, &L);
        if (r < 0) return -1;
        if (tid == 0) {
            tm[team ? 2 : 1] += globaltimer_ns() - t_chunk;
            tcnt[team ? 1 : 0]++;
        }
        if (r == 1) {
            found = true;
            break;
        }
        if (tid == 0) {
            L.chunk_pos = a.ce0;
            if (a.ce0 >= T) end_level(level, nseg);  // the level's last chunk
        }
        __syncthreads();
    }

    // ---- answer: back-pointers of the first precise candidate, then its tree.
    // With a team, its other CTAs empty the table meanwhile (the walk reads
    // back-pointers only)
    if (found && allow_team) {
        if (tid == 0) {
            L.cleaned = 1;
            L.clean_rows = L.smode ? 0u : L.size;
            L.clean_pend = ld_relaxed_u32(&st->pending_count);
            st->c_level = L.clean_rows;
            st->c_size = L.clean_pend;
        }
        publish(st, CMD_CLEAN);
    }
    REI_TSPAN_BEGIN(t_ans);
    // (warp 0: thread 0 decodes, the warp gathers the tree)
    if (found && wid == 0) {
        const uint32_t lane = tid & 31;
        uint32_t op = 0, l = 0, r = 0, ok = 0;
        if (lane == 0) {
            const unsigned long long f = ld_relaxed_u64(&st->found);
            if (L.status == ST_RUNNING && f != kNone) {
                ok = 1;
                decode(S.seg, s_plan.nseg, J.leaf_sym, f, op, l, r);
                st->ans_op = op;
                st->ans_l = l;
                st->ans_r = r;
                st->ans_cost = L.level;
                uint64_t cnt = 0;
                for (uint32_t s = 0; s < s_plan.nseg; s++) {
                    const Seg &g = S.seg[s];
                    uint64_t v = 0;
                    if (g.start + g.size <= f) v = valid_count(g);
                    else if (g.start <= f) v = valid_upto(g, f - g.start);
                    cnt += v;
                    L.cand_op[g.op] += v;
                }
                L.candidates += cnt;
            }
        }
        ok = __shfl_sync(0xFFFFFFFFu, ok, 0);
        if (ok) {
            op = __shfl_sync(0xFFFFFFFFu, op, 0);
            l = __shfl_sync(0xFFFFFFFFu, l, 0);
            r = __shfl_sync(0xFFFFFFFFu, r, 0);
            // (the chunk's shared scratch is free once its answer is known)
            const uint32_t nt = emit_tree_warp(J, op, l, r, reinterpret_cast<uint32_t *>(S.sortbuf));
            if (lane == 0) {
                st->tree_len = nt;
                L.status = ST_FOUND;
            }
        }
    }
    // the state the host reads, and a later launch of this search resumes from
    if (tid == 0) {
        if (ld_relaxed_u32(&st->status) != ST_TIMEOUT) st->status = L.status;
        st->level = L.level;
        st->size = L.size;
        st->full = L.full;
        st->otf = L.otf;
        st->partial_level = L.partial_level;
        st->chunk_pos = L.chunk_pos;
        st->candidates = L.candidates;
        st->unique_done = L.unique_done;
        for (int k = 0; k < 5; k++) st->cand_op[k] = L.cand_op[k];
        for (int k = 0; k < 4; k++) st->t_phase[k] += tm[k];
        for (int k = 0; k < 3; k++) st->n_phase[k] += tcnt[k];
    }
    __syncthreads();
    REI_TSPAN_END(st, t_ans, 20);
    return 0;
}

// the search of one problem by its team of CTAs (the first one leads)
__device__ __forceinline__ void solve_body(const SolveJob &J, uint32_t &bar_epoch) {
    SolveState *st = J.st;
    extern __shared__ __align__(16) uint8_t smem_raw[];
    __shared__ Plan s_plan;
    __shared__ uint32_t s_red[32];
    __shared__ uint64_t s_tiles;
    __shared__ uint32_t s_ctl[8];
    __shared__ uint64_t s_pos[2];
    __shared__ unsigned long long s_found;
    __shared__ uint32_t s_npend;
    __shared__ Lead L;

    const uint32_t tid = threadIdx.x;
    Shared S;
    uint32_t *wm;
    carve_shared(J, S, smem_raw, &wm);
    const Cta K{&s_plan, s_red, &s_tiles, &s_found, &s_npend, &L, wm};

    if (team_rank_of(J) != 0) {
        // ---- worker: run the chunks the leader hands out, until told to stop
        uint32_t seen = 0;
        for (;;) {
            if (tid == 0) {
                // back off up to REI_CMD_NAP ns between polls: hundreds of
                // idle CTAs must not crowd the L2 while CTA 0 works alone
                const unsigned long long t0 = globaltimer_ns();
                uint32_t seq, nap = 64;
                while ((seq = ld_relaxed_u32(&st->cmd_seq)) == seen) {
                    __nanosleep(nap);
                    if (nap < REI_CMD_NAP) nap <<= 1;
                    if (globaltimer_ns() - t0 > kWorkerWaitNs) break;
                }
                __threadfence();
                s_ctl[4] = seq != seen;
                if (seq == seen) {
                    atomicCAS(&st->err, 0u, 3u);
                    atomicExch(&st->status, (uint32_t)ST_TIMEOUT);
                }
            }
            __syncthreads();
            if (!s_ctl[4]) return;
            // the command, and the plan of a chunk CTA 0 published with it,
            // read at once (the plan of the largest level fits; entries past
            // the chunk's segments are not used)
            if (tid == 0) {
                s_ctl[0] = ld_relaxed_u32(&st->cmd);
                s_ctl[1] = ld_relaxed_u32(&st->c_level);
                s_ctl[2] = ld_relaxed_u32(&st->c_size);
                s_ctl[3] = ld_relaxed_u32(&st->c_dedup);
                s_pos[0] = ld_relaxed_u64(&st->c_cs0);
                s_pos[1] = ld_relaxed_u64(&st->c_ce0);
            }
            if (J.plan) read_plan(J, S, &s_tiles, &s_ctl[5]);
            __syncthreads();
            seen++;
            if (s_ctl[0] == CMD_CLEAN) {
                clean_table(J, s_ctl[1], s_ctl[2], team_size_of(J), team_rank_of(J));
                return;
            }
            if (s_ctl[0] != CMD_CHUNK) return;
            ChunkArgs a{s_ctl[1], s_ctl[2], s_ctl[3], 0, s_pos[0], s_pos[1]};
            if (J.plan) {
                a.nseg = s_ctl[5];
            } else {
                // the level table up to this level, as CTA 0 published it
                for (uint32_t c = tid; c <= a.level; c += blockDim.x) {
                    S.lvs[c] = (uint32_t)ld_relaxed_u64(&J.lvl_start[c]);
                    S.lvc[c] = (uint32_t)ld_relaxed_u64(&J.lvl_count[c]);
                }
                __syncthreads();
                if ((tid >> 5) == 0) plan_level(J, a.level, S.lvs, S.lvc, S.seg, s_plan);
                __syncthreads();
                a.nseg = s_plan.nseg;
            }
            if (process_chunk(J, st, S, a, true, J.plan != nullptr, bar_epoch, &s_tiles, s_red, &s_found, &s_npend,
                              wm, nullptr) < 0)
                return;
        }
    }

    // ---- CTA 0 leads
    if (lead_search(J, st, S, K, true, bar_epoch) < 0) return;
    REI_TSPAN_BEGIN(t_cl);
    const uint32_t status = ld_relaxed_u32(&st->status);
    if (L.cleaned) {
        // (the other CTAs were told while the answer was written out)
        clean_table(J, L.clean_rows, L.clean_pend, team_size_of(J), 0);
        __syncthreads();
        if (tid == 0) st->pending_count = 0;
    } else if (status == ST_FOUND || status == ST_NOT_FOUND || status == ST_OOM) {
        // every CTA empties its share of the slots this search filled
        // (languages that never left shared memory are in no global slot)
        const uint32_t rows = L.smode ? 0u : L.size, npending = ld_relaxed_u32(&st->pending_count);
        if (tid == 0) {
            st->c_level = rows;
            st->c_size = npending;
        }
        publish(st, CMD_CLEAN);
        clean_table(J, rows, npending, team_size_of(J), 0);
        __syncthreads();
        if (tid == 0) st->pending_count = 0;
    } else {
        publish(st, CMD_EXIT);
    }
    REI_TSPAN_END(st, t_cl, 21);
}

__global__ void __launch_bounds__(kSolveThreads, 2) k_solve(const __grid_constant__ SolveJob J) {
    uint32_t bar_epoch = 0;
    solve_body(J, bar_epoch);
}

// chunk size for W-word languages (the host's rule for the plain launch)
__device__ __forceinline__ uint64_t auto_chunk(uint32_t W) {
    uint64_t c = (1ull << 28) / (4ull * W);
    if (c < (1ull << 16)) c = 1ull << 16;
    if (c > (1ull << 22)) c = 1ull << 22;
    return c;
}

// Stage (CTA 0, the strings and the staging scratch in its shared memory),
// size the search from the staged problem, then search, all in one launch.
// A problem whose staging or search the launch cannot hold (|ic| > 2048, a
// guide table beyond the pair buffer, shared memory) ends with ST_RESTAGE.
static_assert(sizeof(StageInfo) % 8 == 0 && offsetof(SolveState, launch) % 8 == 0, "state reset by 8-byte words");

// CTA 0's last step: the final state, tokens and staging report to the host
__device__ void state_out(const FuseArgs &F) {
    if (!F.host_out) return;
    __syncthreads();
    const unsigned long long *src = reinterpret_cast<const unsigned long long *>(F.tmpl.st);
    for (uint64_t i = threadIdx.x; i < F.out_words; i += blockDim.x) F.host_out[i] = ld_relaxed_u64(src + i);
    __threadfence_system();
}

__global__ void __launch_bounds__(kFusedThreads, 1) k_solve_fused(const __grid_constant__ FuseArgs F) {
    extern __shared__ __align__(16) uint8_t smem_raw[];
    __shared__ SolveJob J;
    __shared__ uint32_t s_go;
    SolveState *st = F.tmpl.st;
    uint32_t bar_epoch = 0;
#ifdef REI_TIMING
    const unsigned long long t_begin = globaltimer_ns();
    const long long c_begin = clock64();
#endif
    if (blockIdx.x == 0) {
        // this launch's state starts from zero (the state buffer holds the
        // previous launch's; the other CTAs read none of it before the release
        // below), and so does the level table
        {
            unsigned long long *w = reinterpret_cast<unsigned long long *>(st);
            for (uint32_t i = threadIdx.x; i < offsetof(SolveState, launch) / 8; i += blockDim.x) w[i] = 0;
            unsigned long long *si = reinterpret_cast<unsigned long long *>(F.sj.info);
            for (uint32_t i = threadIdx.x; i < sizeof(StageInfo) / 8; i += blockDim.x) si[i] = 0;
        }
        for (uint32_t c = threadIdx.x; c < F.tmpl.max_cost + 2; c += blockDim.x) {
            F.tmpl.lvl_start[c] = 0;
            F.tmpl.lvl_count[c] = 0;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            st->level = F.tmpl.cmin;
            st->found = kNone;
            st->partial_level = F.tmpl.max_cost + 1;
        }
        {
#ifdef REI_TIMING
            REI_TSPAN_BEGIN(t_sr);
#endif
            StageSmem M;
            stage_layout(kServeMaxIC, kServeMaxBytes, smem_raw, &M);
            stage_run(F.sj, M);
            __syncthreads();
            REI_TSPAN_END(st, t_sr, 22);
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            const StageInfo I = *F.sj.info;
            SolveJob j = F.tmpl;
            bool ok = I.status == SE_OK;
            if (ok) {
                j.n = I.n;
                j.W = I.W;
                j.G = I.G;
                j.max_len = I.max_len;
                j.n_pos_set = I.n_pos_set;
                j.pos_eps = I.pos_eps;
                j.neg_eps = I.neg_eps;
                const uint32_t W = I.W;
                j.cap = umin64(F.mem_budget / (4ull * W + 28), 0x7FFF0000ull);
                j.exact = F.tmpl.exact && W <= 2 && I.n <= 62 ? 1u : 0u;
                j.seen = j.exact && W == 1 && I.n <= F.seen_bits ? F.seen : nullptr;
                j.direct = j.exact && W == 1 && (1ull << I.n) <= F.table_slots ? 1u : 0u;
                j.handover = F.handover;
                const uint64_t tmax = F.table_slots / 2;
                j.cache_alloc = umin64(umin64(j.cap, F.rows_alloc), umin64(F.cs_words / W, tmax / 2));
                uint64_t ch = F.chunk_opt ? F.chunk_opt : auto_chunk(W);
                ch = umin64(umin64(ch, 1ull << 24), umin64(F.tmp_words / W, F.pend_cap));
                j.chunk_max = umin64(ch, tmax - j.cache_alloc);
                // shared memory: guide table there if it fits, then the
                // largest shared-memory start that fits
                const uint32_t warps = blockDim.x / 32;
                j.gt_in_smem = solve_smem_bytes(W, I.n, I.G, I.max_len, j.seg_cap, true, warps, 0) <= F.smem_cap;
                j.small_rows = 0;
                if (F.small_opt && W <= 8) {
                    uint32_t r = F.small_opt != 0xFFFFFFFFu ? F.small_opt : W <= 2 ? 4096u : W <= 4 ? 2048u : 1024u;
                    for (; r >= 256; r >>= 1)
                        if (solve_smem_bytes(W, I.n, I.G, I.max_len, j.seg_cap, j.gt_in_smem, warps, r) <= F.smem_cap)
                            break;
                    if (r >= 256) j.small_rows = r;
                }
                ok = j.cache_alloc >= 1 && j.chunk_max >= 1 &&
                     solve_smem_bytes(W, I.n, I.G, I.max_len, j.seg_cap, j.gt_in_smem, warps, j.small_rows) <=
                         F.smem_cap;
            }
            J = j;  // (CTA 0 keeps the job in shared memory)
            if (!ok) st->status = ST_RESTAGE;
            s_go = ok ? 1u : 0u;
        }
        __syncthreads();
        // the job for the other CTAs, written by every thread; then the
        // release: the job and the fresh state are in place
        {
            const unsigned long long *src = reinterpret_cast<const unsigned long long *>(&J);
            unsigned long long *dst = reinterpret_cast<unsigned long long *>(F.job);
            for (uint32_t i = threadIdx.x; i < sizeof(SolveJob) / 8; i += blockDim.x) dst[i] = src[i];
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();
            atomicExch(&st->launch, F.launch_id);
        }
        if (!s_go) {
            state_out(F);
            return;
        }
    } else {
        // the other CTAs wait for CTA 0's release of this launch (a stale id
        // in the state is always smaller: ids only grow), then take the job
        if (threadIdx.x == 0) {
            const unsigned long long t0 = globaltimer_ns();
            uint32_t nap = 64, go = 0;
            for (;;) {
                if (ld_acquire_u64(&st->launch) == F.launch_id) {
                    go = 1;
                    break;
                }
                if (globaltimer_ns() - t0 > kBarrierWaitNs) break;
                __nanosleep(nap);
                if (nap < REI_CMD_NAP) nap <<= 1;
            }
            __threadfence();
            if (go && ld_relaxed_u32(&st->status) != ST_RUNNING) go = 0;
            if (!go && ld_acquire_u64(&st->launch) != F.launch_id) {
                // (never released: the launch ends with an error for the host)
                atomicCAS(&st->err, 0u, 4u);
                atomicExch(&st->status, (uint32_t)ST_TIMEOUT);
            }
            s_go = go;
        }
        __syncthreads();
        if (!s_go) return;
        const unsigned long long *src = reinterpret_cast<const unsigned long long *>(F.job);
        unsigned long long *dst = reinterpret_cast<unsigned long long *>(&J);
        for (uint32_t i = threadIdx.x; i < sizeof(SolveJob) / 8; i += blockDim.x) dst[i] = ld_relaxed_u64(src + i);
        __syncthreads();
    }
#ifdef REI_TIMING
    if (blockIdx.x == 0 && threadIdx.x == 0) st->t_sub[10] = globaltimer_ns() - t_begin;
#endif
    solve_body(J, bar_epoch);
#ifdef REI_TIMING
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        st->t_sub[11] = globaltimer_ns() - t_begin;
        st->t_sub[38] = (unsigned long long)(clock64() - c_begin);
    }
#endif
    if (blockIdx.x == 0) state_out(F);
}

// ---------------------------------------------------------------------------
// the batched search: one launch for many staged problems; every CTA takes
// problems from a queue and solves each one on its own (its own memory slot,
// no grid-wide synchronisation), with the same leader code as k_solve.

// Solve the problem whose job (staged data, costs) is in shared memory J,
// in memory slot `slot`, on this CTA alone; the report goes to *out and the
// tree to J.tree.  Returns the search's status (every thread).  With
// ST_NEED_MEM (the time allowance ran out or the slot is too small) the slot
// keeps the cache rows, back-pointers, level table and state for the host to
// continue from; its uniqueness table and survivor bitmap are emptied.
// a problem's search in memory slot `slot`: its cache, table, chunk
// workspace, level table, state and answer-walk stack (one CTA's share)
__device__ void bind_slot(SolveJob &J, const SlotMem &m, uint32_t slot) {
    const uint64_t so = slot;
    J.cs = m.cs + so * m.cs_words;
    J.bp_op = m.bp_op + so * m.rows;
    J.bp_l = m.bp_l + so * m.rows;
    J.bp_r = m.bp_r + so * m.rows;
    J.used = m.used + so * m.rows;
    J.cache_alloc = umin64(J.cap, m.cs_words / J.W < m.rows ? m.cs_words / J.W : m.rows);
    J.table = m.table + so * m.table_slots;
    J.table_mask = m.table_slots - 1;
    J.tmp = m.tmp + so * m.tmp_words;
    J.chunk_max = umin64(m.chunk, m.tmp_words / J.W);
    J.pending = m.pending + so * m.chunk;
    J.slotpos = m.slotpos + so * m.chunk;
    J.bitmap = m.bitmap + so * ((m.chunk + 31) / 32);
    J.blk = m.blk + so;
    J.lvl_start = m.lvl + so * 2 * (kMaxCost + 2);
    J.lvl_count = J.lvl_start + (kMaxCost + 2);
    J.st = m.state + so;
    J.tstack = m.tstack + so * 4 * (kMaxCost + 2);
    J.trace = nullptr;
}

// a slot search's report (thread 0)
__device__ void report_slot(const SolveJob &J, uint32_t status, uint32_t slot, unsigned long long ns, BatchOut &o) {
    const SolveState *st = J.st;
    o.status = status;
    o.cost = st->ans_cost;
    o.tree_len = st->tree_len;
    o.candidates = st->candidates;
    o.unique = st->unique_done;
    o.levels = st->level;
    for (int k = 0; k < 5; k++) o.cand_op[k] = st->cand_op[k];
    o.ns = ns;
    o.slot = slot;
    o.need_rows = status == ST_NEED_MEM ? st->need_rows : 0u;
}

// keep_table: a search that parks leaves its uniqueness table in the slot
// (the batch continues it there, or empties the table when it continues
// elsewhere); else the table is emptied for the slot's next problem
__device__ uint32_t solve_in_slot(SolveJob &J, const SlotMem &m, uint32_t slot, BatchOut *out, uint8_t *smem_raw,
                              Plan *s_plan, uint32_t *s_red, uint64_t *s_tiles, unsigned long long *s_found,
                              uint32_t *s_npend, Lead *L, uint64_t yield_ns, bool keep_table) {
    const uint32_t tid = threadIdx.x;
    const unsigned long long t_start = globaltimer_ns();
    if (tid == 0) {
        J.yield_ns = yield_ns;
        J.t_start = t_start;
        bind_slot(J, m, slot);
        J.solo_tiles = 0xFFFFFFFFu;
        J.team_base = blockIdx.x;
        J.team_size = 1;
    }
    __syncthreads();
    SolveState *st = J.st;
    // fresh search state and level table for this problem
    for (uint32_t c = tid; c < 2 * (kMaxCost + 2); c += blockDim.x) J.lvl_start[c] = 0;
    if (tid == 0) {
        SolveState z{};
        z.status = ST_RUNNING;
        z.level = J.cmin;
        z.found = kNone;
        z.partial_level = J.max_cost + 1;
        *st = z;
    }
    __threadfence();
    __syncthreads();
    Shared S;
    uint32_t *wm;
    carve_shared(J, S, smem_raw, &wm);
    const Cta K{s_plan, s_red, s_tiles, s_found, s_npend, L, wm};
    uint32_t epoch = 0;
    lead_search(J, st, S, K, false, epoch);
    const uint32_t status = st->status;
    if (status == ST_FOUND || status == ST_NOT_FOUND || status == ST_OOM) {
        clean_table(J, L->smode ? 0u : L->size, st->pending_count, 1, 0);
    } else {
        // the search continues from the slot's rows and state (in the slot,
        // or on the whole GPU, where the table is rebuilt from the rows)
        if (!keep_table)
            for (uint64_t i = tid; i <= J.table_mask; i += blockDim.x) J.table[i] = kEmpty;
        for (uint64_t i = tid; i < (J.chunk_max + 31) / 32; i += blockDim.x) J.bitmap[i] = 0;
    }
    __syncthreads();
    if (tid == 0) report_slot(J, status, slot, globaltimer_ns() - t_start, *out);
    __syncthreads();
    return status;
}

__global__ void __launch_bounds__(256, 2) k_solve_batch(const BatchJob *jobs, const __grid_constant__ BatchArgs B) {
    extern __shared__ __align__(16) uint8_t smem_raw[];
    __shared__ Plan s_plan;
    __shared__ uint32_t s_red[32];
    __shared__ uint64_t s_tiles;
    __shared__ unsigned long long s_found;
    __shared__ uint32_t s_npend;
    __shared__ Lead L;
    __shared__ SolveJob J;
    __shared__ uint32_t s_prob;
    const uint32_t tid = threadIdx.x;
    for (;;) {
        if (tid == 0) s_prob = atomicAdd(B.queue, 1u);
        __syncthreads();
        const uint32_t pi = s_prob;
        __syncthreads();
        if (pi >= B.n) return;
        const BatchJob &bj = jobs[pi];
        if (tid == 0) {
            J = bj.job;
            J.tree = bj.tree;
        }
        __syncthreads();
        // a search left in this slot for the host to continue: the slot is
        // not reused, and this CTA takes no more problems (the host launches
        // again for any left in the queue)
        if (solve_in_slot(J, B.slot, blockIdx.x, bj.out, smem_raw, &s_plan, s_red, &s_tiles, &s_found, &s_npend,
                          &L, B.yield_ns, true) == ST_NEED_MEM)
            return;
    }
}

// ---------------------------------------------------------------------------
// searches a batch left in their slots at their time allowance, continued side
// by side: group g of G.group_ctas CTAs takes problem G.prob[g] in its slot and
// runs the plain search there (its first CTA leads, the others take the team
// chunks), with the slot's cache, uniqueness table and state as the batch CTA
// left them.  The leader writes the problem's report like a batch CTA.
__global__ void __launch_bounds__(256, 2) k_solve_groups(const BatchJob *jobs, const __grid_constant__ GroupArgs G) {
    __shared__ SolveJob J;
    __shared__ unsigned long long s_t0;
    const uint32_t g = blockIdx.x / G.group_ctas;
    if (g >= G.groups) return;
    const uint32_t slot = G.slot_of[g];
    const BatchJob &bj = jobs[G.prob[g]];
    if (threadIdx.x == 0) {
        J = bj.job;
        J.tree = bj.tree;
        bind_slot(J, G.slot, slot);
        J.blk = G.blk + (uint64_t)g * G.group_ctas;
        J.plan = G.plan + (uint64_t)g * G.plan_stride;
        J.tmp = G.tmp + (uint64_t)g * G.tmp_words;
        J.pending = G.pending + (uint64_t)g * G.chunk;
        J.slotpos = G.slotpos + (uint64_t)g * G.chunk;
        J.bitmap = G.bitmap + (uint64_t)g * ((G.chunk + 31) / 32);
        // (new languages of a chunk and the cached ones keep the slot's
        // table at most half full)
        J.chunk_max = umin64(umin64(G.chunk, G.tmp_words / J.W), (J.table_mask + 1) / 2 - J.cache_alloc);
        J.team_base = g * G.group_ctas;
        J.team_size = G.group_ctas;
        J.yield_ns = 0;
        J.solo_tiles = 64;
        J.small_rows = 0;
        J.handover = 0;
        s_t0 = globaltimer_ns();
        // (the leader continues the parked search; the other CTAs read no
        // state before its first command)
        if (team_rank_of(J) == 0) {
            SolveState *st = J.st;
            st->status = ST_RUNNING;
            st->need_rows = 0;
            st->pending_count = 0;
            st->bar_arrive = 0;
            st->cmd = 0;
            st->cmd_seq = 0;
            st->err = 0;
        }
    }
    __syncthreads();
    uint32_t epoch = 0;
    solve_body(J, epoch);
    if (team_rank_of(J) == 0 && threadIdx.x == 0)
        report_slot(J, ld_relaxed_u32(&J.st->status), slot, globaltimer_ns() - s_t0, *bj.out);
}

// ---------------------------------------------------------------------------
// the served search: a persistent launch whose CTAs take requests from a ring
// in mapped host memory as the host publishes them, stage each one themselves
// (scratch in their slot), solve it, and write the answer and a completion
// word back to mapped memory.  A CTA that finds nothing to do for idle_ns, or
// sees the stop word, returns; the host relaunches when work arrives.

__device__ __forceinline__ unsigned long long ld_acquire_sys_u64(const volatile unsigned long long *p) {
    unsigned long long v;
    asm volatile("ld.acquire.sys.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__global__ void __launch_bounds__(256, 2) k_serve(const __grid_constant__ ServeArgs A) {
    extern __shared__ __align__(16) uint8_t smem_raw[];
    __shared__ Plan s_plan;
    __shared__ uint32_t s_red[32];
    __shared__ uint64_t s_tiles;
    __shared__ unsigned long long s_found;
    __shared__ uint32_t s_npend;
    __shared__ Lead L;
    __shared__ SolveJob J;
    __shared__ StageJob SJ;
    __shared__ unsigned long long s_job;
    const uint32_t tid = threadIdx.x;
    const uint32_t slot = blockIdx.x;
    for (;;) {
        if (tid == 0) {
            // claim the next published request, backing off while there is none
            const unsigned long long t0 = globaltimer_ns();
            uint32_t nap = 64;
            unsigned long long job = kNone;
            for (;;) {
                if (ld_acquire_sys_u64(A.stop)) break;
                const unsigned long long h = ld_relaxed_u64(A.head);
                const unsigned long long av = ld_acquire_sys_u64(A.avail);
                if (h < av) {
                    if (atomicCAS(A.head, h, h + 1) == h) {
                        job = h;
                        break;
                    }
                    continue;
                }
                __nanosleep(nap);
                if (nap < 2048) nap <<= 1;
                if (globaltimer_ns() - t0 > A.idle_ns) break;
            }
            s_job = job;
        }
        __syncthreads();
        const unsigned long long job = s_job;
        __syncthreads();
        if (job == kNone) return;
        const uint32_t r = (uint32_t)(job % A.ring_size);
        const ServeReq &q = A.ring[r];
        ServeOut &o = A.outs[r];
        // the entry is read only once it is whole: its sequence word names
        // this job and its sizes are in range (waited for at most 2 ms; a
        // request still incomplete then is answered as invalid, never read)
        if (tid == 0) {
            const unsigned long long t0 = globaltimer_ns();
            uint32_t ok = 0, tries = 0;
            for (;;) {
                if (ld_acquire_sys_u64(&q.seq) == job + 1) {
                    const uint32_t np = q.n_pos, nn = q.n_neg, ns = q.n_sym, tb = q.total_bytes;
                    if (np + nn <= kServeMaxStrings && np <= kServeMaxStrings && ns <= 256 && tb <= kServeMaxBytes &&
                        q.offs[np + nn] == tb && q.max_cost <= REI_MAX_COST) {
                        ok = 1;
                        break;
                    }
                }
                tries++;
                if (globaltimer_ns() - t0 > 2000000ull) break;
                __nanosleep(256);
            }
            if (tries) atomicAdd(A.head + 1, 1ull);
            if (!ok) atomicAdd(A.head + 2, 1ull);
            s_red[1] = ok;
        }
        __syncthreads();
        if (!s_red[1]) {
            if (tid == 0) {
                o.out = BatchOut{};
                o.out.status = ST_BAD;
                o.info = StageInfo{};
                __threadfence_system();
                *(volatile unsigned long long *)&o.done = job + 1;
                __threadfence_system();
            }
            __syncthreads();
            continue;
        }
        // the request's offsets into this slot's buffer, then staged by this CTA
        const uint32_t n_str = q.n_pos + q.n_neg;
        uint32_t *in_o = A.in_offs + (uint64_t)slot * (kServeMaxStrings + 1);
        for (uint32_t i = tid; i <= n_str; i += blockDim.x) in_o[i] = q.offs[i];
        if (tid == 0) {
            StageJob sj{};
            sj.bytes = q.bytes;  // copied once into shared memory by the staging
            sj.offs = in_o;
            sj.n_pos = q.n_pos;
            sj.n_neg = q.n_neg;
            for (uint32_t a = 0; a < q.n_sym; a++) sj.alphabet[a] = q.alphabet[a];
            sj.n_sym = q.n_sym;
            sj.total_bytes = q.total_bytes;
            sj.info = A.sinfo + slot;
            sj.word_start = A.word_start + (uint64_t)slot * kMaxIC;
            sj.word_len = A.word_len + (uint64_t)slot * kMaxIC;
            sj.len_start = A.len_start + (uint64_t)slot * (REI_MAX_STRLEN + 2);
            sj.gt_off = A.gt_off + (uint64_t)slot * (kMaxIC + 1);
            sj.gt_pair = A.gt_pair + (uint64_t)slot * A.pair_cap;
            sj.pair_cap = A.pair_cap;
            sj.pos_mask = A.pos + (uint64_t)slot * kMaxWords;
            sj.neg_mask = A.neg + (uint64_t)slot * kMaxWords;
            sj.leaf = A.leaf + (uint64_t)slot * kMaxWords * 256;
            SJ = sj;
        }
        __threadfence();
        __syncthreads();
        {
            // the staging scratch uses the shared memory the search carves later
            StageSmem M;
            stage_layout(kServeMaxIC, kServeMaxBytes, smem_raw, &M);
            stage_run(SJ, M);
        }
        __threadfence();
        __syncthreads();
        const StageInfo I = *SJ.info;
        __syncthreads();
        uint32_t verdict = 0;  // 0 solve, 1 invalid input, 2 too large for this launch
        // the job, built in shared memory (zeroed, the leaf table by every
        // thread, the rest by thread 0)
        if (tid == 0) {
            if (I.status == SE_PAIRS || I.status == SE_IC_LARGE) verdict = 2;
            else if (I.status != SE_OK) verdict = 1;
            s_red[0] = verdict;
        }
        for (uint32_t i = tid; i < sizeof(SolveJob) / 8; i += blockDim.x)
            reinterpret_cast<unsigned long long *>(&J)[i] = 0;
        __syncthreads();
        verdict = s_red[0];
        if (!verdict) {
            for (uint32_t a = tid; a < 256; a += blockDim.x) {
                J.leaf_cost[a] = q.leaf_cost[a];
                J.leaf_sym[a] = q.leaf_sym[a];
            }
            if (tid == 0) {
                SolveJob &j = J;
                j.n = I.n;
                j.W = I.W;
                j.G = I.G;
                j.n_sym = q.n_sym;
                j.max_len = I.max_len;
                j.gt_off = SJ.gt_off;
                j.gt_pair = SJ.gt_pair;
                j.len_start = SJ.len_start;
                j.pos_mask = SJ.pos_mask;
                j.neg_mask = SJ.neg_mask;
                j.leaf = SJ.leaf;
                j.leaf_stride = kMaxWords;
                j.n_pos_set = I.n_pos_set;
                j.pos_eps = I.pos_eps;
                j.neg_eps = I.neg_eps;
                j.cmin = q.cmin;
                j.c[0] = q.costs.c_sym;
                j.c[1] = q.costs.c_opt;
                j.c[2] = q.costs.c_star;
                j.c[3] = q.costs.c_cat;
                j.c[4] = q.costs.c_alt;
                j.max_cost = q.max_cost;
                j.max_errors = q.max_errors;
                j.flags = q.flags;
                const uint64_t per = 4ull * I.W + 28;
                j.cap = umin64(q.mem_budget / per, 0x7FFF0000ull);
                j.seg_cap = 2 * q.max_cost + 4;
                j.gt_in_smem = solve_smem_bytes(I.W, I.n, I.G, I.max_len, j.seg_cap, true, blockDim.x / 32, 0) <=
                               A.smem_cap;
                if (solve_smem_bytes(I.W, I.n, I.G, I.max_len, j.seg_cap, j.gt_in_smem, blockDim.x / 32, 0) >
                        A.smem_cap ||
                    I.W > A.slot.cs_words / A.slot.rows)
                    s_red[0] = 2;
                j.tree = o.tree;
            }
        }
        __syncthreads();
        verdict = s_red[0];
        __syncthreads();
        uint32_t status = ST_BAD;
        if (verdict == 0) {
            status = solve_in_slot(J, A.slot, slot, &o.out, smem_raw, &s_plan, s_red, &s_tiles, &s_found, &s_npend,
                                   &L, A.yield_ns, true);
            // a parked search's job, for its continuation (in its slot, or on
            // the whole GPU from the slot's rows)
            if (status == ST_NEED_MEM && threadIdx.x == 0) {
                BatchJob &pj = A.parked[slot];
                pj.job = J;
                pj.tree = o.tree;
                pj.out = &o.out;
            }
        } else if (tid == 0) {
            o.out.status = verdict == 1 ? ST_BAD : ST_NEED_MEM;
            o.out.slot = kNoSlot;  // (too large for a slot: never searched here)
        }
        if (tid == 0) {
            o.info = I;
            __threadfence_system();
            *(volatile unsigned long long *)&o.done = job + 1;
            __threadfence_system();
        }
        __syncthreads();
        // a search left in this slot for the host to continue: the CTA takes
        // no more requests, so the slot stays as it is until the host has
        // copied it (the host stops the launch before it does)
        if (status == ST_NEED_MEM) return;
    }
}

// rebuild the uniqueness table after the cache grew (all entries are distinct)
__global__ void k_rehash(const __grid_constant__ SolveJob J, uint32_t count) {
    const uint32_t W = J.W;
    for (uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; k < count;
         k += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t *c = J.cs + k * W;
        const uint64_t h = cs_hash(c, W, 1);
        const unsigned long long v =
            J.exact ? exact_key(c, W) : ((uint64_t)(uint32_t)(h >> 32) << 32) | (uint32_t)k;
        uint64_t p = J.direct ? v : h & J.table_mask;
        for (uint64_t probe = 0; probe <= J.table_mask; probe++) {
            if (atomicCAS(&J.table[p], kEmpty, v) == kEmpty) {
                J.used[k] = (uint32_t)p;
                break;
            }
            p = (p + 1) & J.table_mask;
        }
        if (J.seen) atomicOr(J.seen + (c[0] >> 5), 1u << (c[0] & 31u));
    }
}

// the dynamic shared memory limit of a kernel, raised once per device to the
// opt-in maximum (so that launches need no attribute call), and occupancy
// queries remembered per (device, kernel, threads, shared memory)
static std::mutex g_attr_mu;
static std::map<std::pair<int, const void *>, bool> g_attr_set;
static std::map<std::tuple<int, const void *, uint32_t, size_t>, int> g_occ;

static cudaError_t prepare(const void *fn) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lk(g_attr_mu);
    auto key = std::make_pair(dev, fn);
    if (g_attr_set.count(key)) return cudaSuccess;
    int optin = 0;
    e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) return e;
    cudaFuncAttributes fa;
    e = cudaFuncGetAttributes(&fa, fn);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - (int)fa.sharedSizeBytes);
    if (e != cudaSuccess) return e;
    g_attr_set[key] = true;
    return cudaSuccess;
}

// the largest dynamic shared memory one launch of `fn` can take on the
// current device: the opt-in maximum per CTA less the kernel's static shared
// memory
static cudaError_t smem_max_of(const void *fn, size_t *bytes) {
    int dev = 0, optin = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) return e;
    cudaFuncAttributes fa;
    e = cudaFuncGetAttributes(&fa, fn);
    if (e != cudaSuccess) return e;
    *bytes = (size_t)optin > fa.sharedSizeBytes ? (size_t)optin - fa.sharedSizeBytes : 0;
    return cudaSuccess;
}

static cudaError_t occupancy(const void *fn, uint32_t threads, size_t smem, int *bps) {
    cudaError_t e = prepare(fn);
    if (e != cudaSuccess) return e;
    int dev = 0;
    cudaGetDevice(&dev);
    {
        std::lock_guard<std::mutex> lk(g_attr_mu);
        auto it = g_occ.find(std::make_tuple(dev, fn, threads, smem));
        if (it != g_occ.end()) {
            *bps = it->second;
            return cudaSuccess;
        }
    }
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(bps, fn, (int)threads, smem);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lk(g_attr_mu);
    g_occ[std::make_tuple(dev, fn, threads, smem)] = *bps;
    return cudaSuccess;
}

cudaError_t launch_solve(const SolveJob *job, uint32_t grid, uint32_t threads, size_t smem,
                         cudaStream_t stream) {
    cudaError_t e = prepare((const void *)k_solve);
    if (e != cudaSuccess) return e;
    void *args[] = {(void *)job};
    return cudaLaunchCooperativeKernel((const void *)k_solve, dim3(grid), dim3(threads), args, smem, stream);
}

cudaError_t launch_solve_fused(const FuseArgs *args, uint32_t grid, uint32_t threads, size_t smem,
                               cudaStream_t stream) {
    cudaError_t e = prepare((const void *)k_solve_fused);
    if (e != cudaSuccess) return e;
    void *args_[] = {(void *)args};
    return cudaLaunchCooperativeKernel((const void *)k_solve_fused, dim3(grid), dim3(threads), args_, smem, stream);
}

cudaError_t solve_fused_occupancy(uint32_t threads, size_t smem, int *blocks_per_sm) {
    return occupancy((const void *)k_solve_fused, threads, smem, blocks_per_sm);
}

cudaError_t solve_occupancy(uint32_t threads, size_t smem, int *blocks_per_sm) {
    return occupancy((const void *)k_solve, threads, smem, blocks_per_sm);
}

cudaError_t solve_smem_max(size_t *bytes) { return smem_max_of((const void *)k_solve, bytes); }

cudaError_t solve_batch_smem_max(size_t *bytes) { return smem_max_of((const void *)k_solve_batch, bytes); }

cudaError_t launch_rehash(const SolveJob *job, uint32_t count, uint32_t grid, cudaStream_t stream) {
    k_rehash<<<grid, 256, 0, stream>>>(*job, count);
    return cudaGetLastError();
}

cudaError_t launch_solve_batch(const BatchJob *jobs_dev, const BatchArgs *args, uint32_t grid, uint32_t threads,
                               size_t smem, cudaStream_t stream) {
    cudaError_t e = prepare((const void *)k_solve_batch);
    if (e != cudaSuccess) return e;
    k_solve_batch<<<grid, threads, smem, stream>>>(jobs_dev, *args);
    return cudaGetLastError();
}

cudaError_t solve_batch_occupancy(uint32_t threads, size_t smem, int *blocks_per_sm) {
    return occupancy((const void *)k_solve_batch, threads, smem, blocks_per_sm);
}

cudaError_t launch_solve_groups(const BatchJob *jobs_dev, const GroupArgs *args, uint32_t grid, uint32_t threads,
                                size_t smem, cudaStream_t stream) {
    cudaError_t e = prepare((const void *)k_solve_groups);
    if (e != cudaSuccess) return e;
    void *args_[] = {(void *)&jobs_dev, (void *)args};
    return cudaLaunchCooperativeKernel((const void *)k_solve_groups, dim3(grid), dim3(threads), args_, smem, stream);
}

cudaError_t solve_groups_occupancy(uint32_t threads, size_t smem, int *blocks_per_sm) {
    return occupancy((const void *)k_solve_groups, threads, smem, blocks_per_sm);
}

cudaError_t solve_groups_smem_max(size_t *bytes) { return smem_max_of((const void *)k_solve_groups, bytes); }

cudaError_t launch_serve(const ServeArgs *args, uint32_t grid, uint32_t threads, size_t smem, cudaStream_t stream) {
    cudaError_t e = prepare((const void *)k_serve);
    if (e != cudaSuccess) return e;
    k_serve<<<grid, threads, smem, stream>>>(*args);
    return cudaGetLastError();
}

cudaError_t serve_occupancy(uint32_t threads, size_t smem, int *blocks_per_sm) {
    return occupancy((const void *)k_serve, threads, smem, blocks_per_sm);
}

}  // namespace rei
