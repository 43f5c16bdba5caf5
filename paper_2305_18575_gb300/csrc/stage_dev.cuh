// stage_dev.cuh -- staging of one REI problem by one CTA (internal).
//
// Computes, from the packed example strings:
//   * ic(P u N), the infix closure (Sec. 2 "infix-closed"; Sec. 3 "First
//     space-time trade-off: infix-closure"), in shortlex order over the
//     caller's alphabet with eps at index 0 (Example 1 and its figure);
//   * the guide table (Sec. 3 "Staging: guide table"): for every word w, the
//     |w| + 1 pairs (u, v) with w = u v, in order of the split position, as a
//     CSR array gt_off / gt_pair with u | v << 16;
//   * the characteristic sequences of P and N (precision masks, Def.
//     "specification") and of each alphabet symbol (the leaves of Alg. 1).
//
// Distinct infixes are found with a hash set of occurrences (start, len) keyed
// by content.  Shortlex ranks come from a sort of 64-bit keys (length, then
// the symbols' ranks packed most significant first) when every word packs
// into 39 bits, else from counting the shortlex-smaller words.  All scratch
// (hash set, keys, word table, a copy of the strings when they fit) is
// shared memory the caller carves with stage_layout().
#pragma once
#include <cstdint>

#include "rei_dev.cuh"

namespace rei {


constexpr uint32_t kStageThreads = 1024;
constexpr uint64_t kTagMask = 0xFFFFFFFF00000000ull;
constexpr uint64_t kH0 = 0x9E3779B97F4A7C15ull;

__device__ __forceinline__ uint64_t stage_mix(uint64_t h, uint32_t r) {
    h ^= (uint64_t)(r + 1u);
    h *= 0xBF58476D1CE4E5B9ull;
    h ^= h >> 29;
    return h;
}

__device__ __forceinline__ uint64_t stage_final(uint64_t h, uint32_t len) {
    h ^= (uint64_t)len * 0x94D049BB133111EBull;
    h ^= h >> 31;
    h *= 0xD6E8FEB86659FD93ull;
    h ^= h >> 32;
    return h;
}

// slot = fingerprint (20 bits) << 44 | len (12 bits) << 32 | start (32 bits)
__device__ __forceinline__ uint64_t stage_tag(uint64_t f, uint32_t len) {
    return ((f >> 44) << 44) | ((uint64_t)len << 32);
}

__device__ __forceinline__ bool same_bytes(const uint8_t *b, uint32_t s1, uint32_t s2, uint32_t len) {
    for (uint32_t i = 0; i < len; i++)
        if (b[s1 + i] != b[s2 + i]) return false;
    return true;
}

// scratch of one staging CTA (shared memory)
struct StageSmem {
    uint64_t *hset;            // hcap slots: fingerprint | len | start of one occurrence
    uint16_t *rank_of;         // hcap: shortlex rank of the word in each slot
    unsigned long long *keys;  // ic_cap: the words' slots, then their sort keys
    uint32_t *wstart;          // ic_cap: an occurrence of the word of each rank
    uint16_t *wlen;            // ic_cap: its length
    uint16_t *dfirst, *dlast;  // ic_cap: rank of the word without its first / last symbol
    uint32_t *masks;           // 2 * kMaxWords: P and N characteristic sequences
    uint32_t *offs;            // offs_cap: the string offsets, when they fit
    int16_t *rank_tab;         // 256: rank of each byte in the alphabet, -1 if none
    uint8_t *bytes;            // bytes_cap: the strings, when they fit
    uint32_t hcap, ic_cap, bytes_cap, offs_cap;
};

// bytes of shared memory the scratch takes; carves it from `base` when given.
// ic_cap (a power of two) bounds |ic|; strings longer in total than bytes_cap
// are read from global memory
__host__ __device__ inline size_t stage_layout(uint32_t ic_cap, uint32_t bytes_cap, uint8_t *base,
                                               StageSmem *out) {
    uint32_t hcap = 1;
    while (hcap < 2 * ic_cap) hcap <<= 1;
    size_t o = 0;
    auto carve = [&](size_t bytes) {
        const size_t at = o;
        o += (bytes + 15) & ~size_t(15);
        return at;
    };
    const uint32_t offs_cap = 1024;
    const size_t o_hset = carve(8ull * hcap), o_keys = carve(8ull * ic_cap), o_ws = carve(4ull * ic_cap);
    const size_t o_masks = carve(4ull * 2 * kMaxWords), o_offs = carve(4ull * offs_cap);
    const size_t o_rank = carve(2ull * hcap), o_wl = carve(2ull * ic_cap), o_df = carve(2ull * ic_cap);
    const size_t o_dl = carve(2ull * ic_cap), o_tab = carve(2 * 256);
    const size_t o_bytes = carve(bytes_cap);
    if (base && out) {
        out->hset = reinterpret_cast<uint64_t *>(base + o_hset);
        out->keys = reinterpret_cast<unsigned long long *>(base + o_keys);
        out->wstart = reinterpret_cast<uint32_t *>(base + o_ws);
        out->masks = reinterpret_cast<uint32_t *>(base + o_masks);
        out->offs = reinterpret_cast<uint32_t *>(base + o_offs);
        out->rank_of = reinterpret_cast<uint16_t *>(base + o_rank);
        out->wlen = reinterpret_cast<uint16_t *>(base + o_wl);
        out->dfirst = reinterpret_cast<uint16_t *>(base + o_df);
        out->dlast = reinterpret_cast<uint16_t *>(base + o_dl);
        out->rank_tab = reinterpret_cast<int16_t *>(base + o_tab);
        out->bytes = base + o_bytes;
        out->hcap = hcap;
        out->ic_cap = ic_cap;
        out->bytes_cap = bytes_cap;
        out->offs_cap = offs_cap;
    }
    return o;
}

// hash of the infix bytes[start, start + len)
__device__ __forceinline__ uint64_t stage_hash(const uint8_t *bytes, const int16_t *rank_tab, uint32_t start,
                                               uint32_t len) {
    uint64_t h = kH0;
    for (uint32_t i = 0; i < len; i++) h = stage_mix(h, (uint32_t)rank_tab[bytes[start + i]]);
    return stage_final(h, len);
}

// rank of the infix bytes[start, start + len) with hash f, or 0xFFFFFFFF
__device__ inline uint32_t stage_find(const StageSmem &M, const uint8_t *bytes, uint64_t f, uint32_t start,
                                      uint32_t len) {
    if (len == 0) return 0;
    const uint64_t tag = stage_tag(f, len);
    const uint32_t mask = M.hcap - 1;
    uint32_t q = (uint32_t)f & mask;
    for (uint32_t probe = 0; probe < M.hcap; probe++) {
        const uint64_t v = M.hset[q];
        if (v == kEmpty) return 0xFFFFFFFFu;
        if ((v & kTagMask) == tag && same_bytes(bytes, (uint32_t)v, start, len)) return M.rank_of[q];
        q = (q + 1) & mask;
    }
    return 0xFFFFFFFFu;
}

__device__ inline uint32_t stage_lookup(const StageSmem &M, const uint8_t *bytes, uint32_t start, uint32_t len) {
    if (len == 0) return 0;
    return stage_find(M, bytes, stage_hash(bytes, M.rank_tab, start, len), start, len);
}

// rank of the one-symbol word `a` (alphabet rank `rank`), or 0xFFFFFFFF
__device__ inline uint32_t stage_lookup_symbol(const StageSmem &M, const uint8_t *bytes, uint32_t rank,
                                               uint8_t a) {
    const uint64_t f = stage_final(stage_mix(kH0, rank), 1);
    const uint64_t tag = stage_tag(f, 1);
    const uint32_t mask = M.hcap - 1;
    uint32_t q = (uint32_t)f & mask;
    for (uint32_t probe = 0; probe < M.hcap; probe++) {
        const uint64_t v = M.hset[q];
        if (v == kEmpty) return 0xFFFFFFFFu;
        if ((v & kTagMask) == tag && bytes[(uint32_t)v] == a) return M.rank_of[q];
        q = (q + 1) & mask;
    }
    return 0xFFFFFFFFu;
}

// shortlex: length first, then symbol ranks left to right
__device__ __forceinline__ bool shortlex_less(const uint8_t *bytes, const int16_t *rank_tab,
                                              uint32_t s1, uint32_t l1, uint32_t s2, uint32_t l2) {
    if (l1 != l2) return l1 < l2;
    for (uint32_t i = 0; i < l1; i++) {
        const int16_t a = rank_tab[bytes[s1 + i]], b = rank_tab[bytes[s2 + i]];
        if (a != b) return a < b;
    }
    return false;
}

// exclusive scan of one value per thread over the CTA; returns the prefix
__device__ inline uint32_t block_exclusive_scan(uint32_t v, uint32_t *warp_sums, uint32_t *total) {
    const uint32_t lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    uint32_t x = v;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, d);
        if (lane >= (uint32_t)d) x += y;
    }
    if (lane == 31) warp_sums[wid] = x;
    __syncthreads();
    if (wid == 0) {
        const uint32_t nw = blockDim.x >> 5;
        uint32_t s = lane < nw ? warp_sums[lane] : 0;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, s, d);
            if (lane >= (uint32_t)d) s += y;
        }
        if (lane < nw) warp_sums[lane] = s;
        if (lane == nw - 1) *total = s;
    }
    __syncthreads();
    const uint32_t before = wid ? warp_sums[wid - 1] : 0;
    const uint32_t r = before + x - v;
    __syncthreads();
    return r;
}

// ascending sort of m (a power of two) 64-bit keys in shared memory by the
// calling CTA (blockDim.x a multiple of 32); element i is handled by thread
// i % blockDim.x, so compare-exchanges closer than 32 stay within a warp and
// need only a warp barrier before the next one of the same kind
__device__ inline void block_bitonic_sort(unsigned long long *key, uint32_t m) {
    const uint32_t tid = threadIdx.x, nt = blockDim.x;
    for (uint32_t k = 2; k <= m; k <<= 1) {
        for (uint32_t jj = k >> 1; jj > 0; jj >>= 1) {
            for (uint32_t i = tid; i < m; i += nt) {
                const uint32_t ix = i ^ jj;
                if (ix > i) {
                    const unsigned long long x = key[i], y = key[ix];
                    if ((x > y) == ((i & k) == 0)) {
                        key[i] = y;
                        key[ix] = x;
                    }
                }
            }
            // the next exchange distance: jj / 2, or k at the next k
            const uint32_t next = jj > 1 ? jj >> 1 : k;
            if (next >= 32) __syncthreads();
            else __syncwarp();
        }
    }
    __syncthreads();
}

// step timing (ns, in StageInfo::pad), compiled in with -DREI_TIMING only
#ifdef REI_TIMING
#define STAGE_MARK(k)                                                              \
    do {                                                                           \
        if (threadIdx.x == 0) {                                                    \
            unsigned long long t_now;                                              \
            asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t_now));               \
            J.info->pad[k] = (uint32_t)(t_now - t_prev);                           \
            t_prev = t_now;                                                        \
        }                                                                          \
    } while (0)
#else
#define STAGE_MARK(k) \
    do {              \
    } while (0)
#endif

// stage problem J with the calling CTA, in the scratch M
__device__ inline void stage_run(const StageJob &J, const StageSmem &M) {
#ifdef REI_TIMING
    unsigned long long t_prev;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t_prev));
#endif
    __shared__ uint32_t s_err, s_count, s_maxlen, s_total, s_ov, s_np, s_nn;
    __shared__ uint32_t warp_sums[32];

    const uint32_t tid = threadIdx.x, nt = blockDim.x;
    const uint32_t n_str = J.n_pos + J.n_neg;
    uint64_t *hset = M.hset;
    int16_t *rank_tab = M.rank_tab;

    // the offsets into shared memory when they fit
    const uint32_t *offs = J.offs;
    if (n_str + 1 <= M.offs_cap) {
        for (uint32_t k = tid; k <= n_str; k += nt) M.offs[k] = J.offs[k];
        offs = M.offs;
    }
    for (uint32_t q = tid; q < M.hcap; q += nt) hset[q] = kEmpty;
    for (uint32_t i = tid; i < 256; i += nt) rank_tab[i] = -1;
    for (uint32_t i = tid; i < 2 * kMaxWords; i += nt) M.masks[i] = 0;
    for (uint32_t i = tid; i < J.n_sym * kMaxWords; i += nt) J.leaf[i] = 0;
    if (tid == 0) {
        s_err = SE_OK;
        s_count = 0;
        s_maxlen = 0;
        s_ov = 0;
        s_np = 0;
        s_nn = 0;
    }
    __syncthreads();
    for (uint32_t a = tid; a < J.n_sym; a += nt) rank_tab[J.alphabet[a]] = (int16_t)a;
    const uint32_t total = offs[n_str];
    STAGE_MARK(0);

    // offsets start at 0, never decrease and end at the declared total (device
    // inputs are not checked on the host); every byte must be a symbol;
    // strings must fit the length field
    if (offs[0] != 0 || total != J.total_bytes) s_err = SE_OFFSETS;
    for (uint32_t k = tid; k < n_str; k += nt)
        if (offs[k + 1] < offs[k]) s_err = SE_OFFSETS;
    __syncthreads();
    if (s_err != SE_OK) {
        if (tid == 0) J.info->status = s_err;
        return;
    }
    // the strings into shared memory when they fit
    const uint8_t *bytes = J.bytes;
    if (total <= M.bytes_cap) {
        for (uint32_t p = tid; p < total; p += nt) M.bytes[p] = J.bytes[p];
        bytes = M.bytes;
    }
    __syncthreads();
    for (uint32_t p = tid; p < total; p += nt)
        if (rank_tab[bytes[p]] < 0) s_err = SE_SYMBOL;
    for (uint32_t k = tid; k < n_str; k += nt) atomicMax(&s_maxlen, offs[k + 1] - offs[k]);
    __syncthreads();
    if (s_err == SE_OK && s_maxlen > REI_MAX_STRLEN) s_err = SE_STRLEN;
    __syncthreads();
    STAGE_MARK(1);

    // every occurrence (start p, length len) of every string goes into the
    // set; the first occurrence of each word also records its slot.  The
    // lengths from one start are split into up to four runs of consecutive
    // lengths, one thread each (a run hashes its start's shorter prefix
    // first), so that no thread inserts more than a quarter of a string's
    // infixes from one start
    if (s_err == SE_OK) {
        const uint32_t mask = M.hcap - 1;
        const uint32_t nb = s_maxlen < 8 ? (s_maxlen + 1) / 2 : 4u;  // runs per start (0 when every string is empty)
        const uint32_t run = nb ? (s_maxlen + nb - 1) / nb : 1u;     // lengths per run
        for (uint64_t item = tid; item < (uint64_t)total * nb; item += nt) {
            const uint32_t p = (uint32_t)(item / nb), b = (uint32_t)(item - (uint64_t)p * nb);
            // string k with offs[k] <= p < offs[k+1] (strings may be empty)
            uint32_t lo = 0, hi = n_str;  // invariant: offs[lo] <= p < offs[hi]
            while (hi - lo > 1) {
                const uint32_t mid = (lo + hi) >> 1;
                if (offs[mid] <= p) lo = mid;
                else hi = mid;
            }
            const uint32_t end = offs[lo + 1];
            const uint32_t e0 = p + b * run, e1 = min(end, e0 + run);  // this run's lengths: e0 - p + 1 .. e1 - p
            if (e0 >= end) continue;
            uint64_t h = kH0;
            for (uint32_t e = p + 1; e <= e0; e++) h = stage_mix(h, (uint32_t)rank_tab[bytes[e - 1]]);
            for (uint32_t e = e0 + 1; e <= e1; e++) {
                const uint32_t len = e - p;
                h = stage_mix(h, (uint32_t)rank_tab[bytes[e - 1]]);
                const uint64_t f = stage_final(h, len);
                const uint64_t tag = stage_tag(f, len);
                const uint64_t want = tag | p;
                uint32_t q = (uint32_t)f & mask;
                for (uint32_t probe = 0; probe < M.hcap; probe++) {
                    uint64_t v = *(volatile const uint64_t *)&hset[q];  // (shared memory: CTA-coherent)
                    if (v == kEmpty) {
                        const unsigned long long old =
                            atomicCAS((unsigned long long *)&hset[q], kEmpty, want);
                        if (old == kEmpty) {
                            const uint32_t u = atomicAdd(&s_count, 1u);
                            if (u + 2 > M.ic_cap) s_err = SE_IC_LARGE;
                            else M.keys[u] = q;
                            break;
                        }
                        v = old;
                    }
                    if ((v & kTagMask) == tag && same_bytes(bytes, (uint32_t)v, p, len)) break;
                    q = (q + 1) & mask;
                }
                if (*(volatile uint32_t *)&s_err != SE_OK) break;
            }
            if (*(volatile uint32_t *)&s_err != SE_OK) break;
        }
    }
    __syncthreads();
    if (s_err != SE_OK) {
        if (tid == 0) J.info->status = s_err;
        return;
    }
    STAGE_MARK(2);

    // shortlex ranks (eps = 0).  Packed keys (length << 52 | symbol ranks
    // << 13 | slot) when every word packs into 39 bits: counted for a few
    // words, sorted for many; else counted with byte comparisons
    const uint32_t U = s_count, n = U + 1;
    uint32_t bsym = 1;
    while ((1u << bsym) < J.n_sym) bsym++;
    const bool packed = s_maxlen * bsym <= 39;
    if (packed) {
        for (uint32_t i = tid; i < U; i += nt) {
            const uint32_t q = (uint32_t)M.keys[i];
            const uint64_t v = hset[q];
            const uint32_t st = (uint32_t)v, len = (uint32_t)(v >> 32) & 0xFFFu;
            uint64_t c = 0;
            for (uint32_t k = 0; k < len; k++) c = (c << bsym) | (uint32_t)rank_tab[bytes[st + k]];
            M.keys[i] = ((unsigned long long)len << 52) | (c << 13) | q;
        }
        __syncthreads();
    }
    STAGE_MARK(3);
    if (packed && U > 256) {
        // bitonic sort of the keys (padded to a power of two with ~0)
        uint32_t m = 1;
        while (m < U) m <<= 1;
        for (uint32_t i = U + tid; i < m; i += nt) M.keys[i] = ~0ull;
        __syncthreads();
        block_bitonic_sort(M.keys, m);
        for (uint32_t i = tid; i < U; i += nt) {
            const uint32_t q = (uint32_t)(M.keys[i] & 0x1FFFu), r = i + 1;
            const uint64_t v = hset[q];
            M.rank_of[q] = (uint16_t)r;
            M.wstart[r] = (uint32_t)v;
            M.wlen[r] = (uint16_t)((v >> 32) & 0xFFFu);
        }
    } else {
        for (uint32_t i = tid; i < U; i += nt) {
            const unsigned long long ki = M.keys[i];
            const uint32_t qi = packed ? (uint32_t)(ki & 0x1FFFu) : (uint32_t)ki;
            const uint64_t vi = hset[qi];
            const uint32_t si = (uint32_t)vi, li = (uint32_t)(vi >> 32) & 0xFFFu;
            uint32_t r = 1;
            if (packed) {
                for (uint32_t j = 0; j < U; j++) r += M.keys[j] < ki;
            } else {
                for (uint32_t j = 0; j < U; j++) {
                    const uint64_t vj = hset[(uint32_t)M.keys[j]];
                    if (shortlex_less(bytes, rank_tab, (uint32_t)vj, (uint32_t)(vj >> 32) & 0xFFFu, si, li)) r++;
                }
            }
            M.rank_of[qi] = (uint16_t)r;
            M.wstart[r] = si;
            M.wlen[r] = (uint16_t)li;
        }
    }
    if (tid == 0) {
        M.wstart[0] = 0;
        M.wlen[0] = 0;
        M.dfirst[0] = 0;
        M.dlast[0] = 0;
    }
    __syncthreads();
    STAGE_MARK(4);
    // the word table, and each word without its first / last symbol (infixes:
    // in ic); first rank of every length (all lengths 0..max_len occur)
    for (uint32_t r = tid; r < n; r += nt) {
        const uint32_t st = M.wstart[r], L = M.wlen[r];
        J.word_start[r] = st;
        J.word_len[r] = L;
        if (r == 0 || M.wlen[r - 1] != L) J.len_start[L] = r;
        if (r) {
            const uint32_t a = stage_lookup(M, bytes, st + 1, L - 1), b = stage_lookup(M, bytes, st, L - 1);
            if (a >= n || b >= n) s_err = SE_INTERNAL;
            M.dfirst[r] = (uint16_t)a;
            M.dlast[r] = (uint16_t)b;
        }
    }
    const uint32_t max_len = M.wlen[n - 1];
    if (tid == 0) J.len_start[max_len + 1] = n;
    // a failed lookup (not expected: every infix of every example is in the
    // set) leaves no valid rank to walk the splits with: stop here
    __syncthreads();
    if (s_err != SE_OK) {
        if (tid == 0) J.info->status = s_err;
        return;
    }

    // guide-table offsets: exclusive scan of |w| + 1 over words in rank order
    const uint32_t per = (n + nt - 1) / nt;
    const uint32_t r0 = min(n, tid * per), r1 = min(n, r0 + per);
    uint32_t local = 0;
    for (uint32_t r = r0; r < r1; r++) local += M.wlen[r] + 1u;
    uint32_t off = block_exclusive_scan(local, warp_sums, &s_total);  // (synchronises the CTA)
    const uint32_t G = s_total;
    if (G > J.pair_cap) {
        if (tid == 0) {
            J.info->status = SE_PAIRS;
            J.info->n = n;
            J.info->G = G;
            J.info->max_len = max_len;
        }
        return;
    }
    // pairs of word r: split k is (prefix of length k, the rest); prefixes by
    // dropping last symbols from r, suffixes by dropping first symbols.  Each
    // half of a pair word is stored on its own (16-bit stores: the halves
    // are written, never read back from global memory)
    for (uint32_t r = r0; r < r1; r++) {
        J.gt_off[r] = off;
        const uint32_t len = M.wlen[r];
        // (little-endian words: pair k's low half, the prefix, is out[2k])
        uint16_t *out = reinterpret_cast<uint16_t *>(J.gt_pair + off);
        uint32_t v = r;
        for (uint32_t k = 0; k <= len; k++) {
            out[2 * k + 1] = (uint16_t)v;
            v = M.dfirst[v];
        }
        uint32_t u = r;
        for (uint32_t k = len + 1; k-- > 0;) {
            out[2 * k] = (uint16_t)u;
            u = M.dlast[u];
        }
        off += len + 1;
    }
    if (tid == 0) J.gt_off[n] = G;
    STAGE_MARK(5);

    // characteristic sequences of P and N (shared), and of every symbol
    for (uint32_t k = tid; k < n_str; k += nt) {
        const uint32_t r = stage_lookup(M, bytes, offs[k], offs[k + 1] - offs[k]);
        if (r >= n) {
            s_err = SE_INTERNAL;
            continue;
        }
        atomicOr(&M.masks[(k < J.n_pos ? 0 : kMaxWords) + (r >> 5)], 1u << (r & 31));
    }
    for (uint32_t a = tid; a < J.n_sym; a += nt) {
        const uint32_t r = stage_lookup_symbol(M, bytes, a, J.alphabet[a]);
        if (r < n) J.leaf[a * kMaxWords + (r >> 5)] = 1u << (r & 31);
    }
    __syncthreads();
    const uint32_t W = padded_words(n);
    for (uint32_t b = tid; b < kMaxWords; b += nt) {
        const uint32_t p = M.masks[b], q = M.masks[kMaxWords + b];
        J.pos_mask[b] = p;
        J.neg_mask[b] = q;
        if (p & q) s_ov = 1;
        if (p) atomicAdd(&s_np, (uint32_t)__popc(p));
        if (q) atomicAdd(&s_nn, (uint32_t)__popc(q));
    }
    __syncthreads();
    STAGE_MARK(6);
    if (tid == 0) {
        StageInfo *I = J.info;
        I->status = s_err != SE_OK ? s_err : s_ov ? SE_OVERLAP : SE_OK;
        I->n = n;
        I->W = W;
        I->max_len = max_len;
        I->G = G;
        I->n_pos_set = s_np;
        I->n_neg_set = s_nn;
        I->pos_eps = M.masks[0] & 1u;
        I->neg_eps = M.masks[kMaxWords] & 1u;
    }
}


}  // namespace rei
