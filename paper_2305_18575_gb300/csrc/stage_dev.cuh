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
// by content; ranks come from counting the shortlex-smaller words.  The hash
// set and its side arrays live wherever the caller puts them: in shared
// memory for the staging kernel, in global scratch for a server CTA that
// stages the requests it takes.
#pragma once
#include <cstdint>

#include "rei_dev.cuh"

namespace rei {


constexpr uint32_t kHsetCap = 4 * kMaxIC;  // slots; at most kMaxIC + in-flight entries
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

// rank of the infix bytes[start, start + len) in ic, or 0xFFFFFFFF if absent
__device__ inline uint32_t stage_lookup(const uint8_t *bytes, const uint64_t *hset, const uint16_t *rank_of,
                                 const int16_t *rank_tab, uint32_t start, uint32_t len) {
    if (len == 0) return 0;
    uint64_t h = kH0;
    for (uint32_t i = 0; i < len; i++) h = stage_mix(h, (uint32_t)rank_tab[bytes[start + i]]);
    const uint64_t f = stage_final(h, len);
    const uint64_t tag = stage_tag(f, len);
    uint32_t q = (uint32_t)f & (kHsetCap - 1);
    for (uint32_t probe = 0; probe < kHsetCap; probe++) {
        const uint64_t v = hset[q];
        if (v == kEmpty) return 0xFFFFFFFFu;
        if ((v & kTagMask) == tag && same_bytes(bytes, (uint32_t)v, start, len)) return rank_of[q];
        q = (q + 1) & (kHsetCap - 1);
    }
    return 0xFFFFFFFFu;
}

// rank of the one-symbol word `a`, or 0xFFFFFFFF
__device__ inline uint32_t stage_lookup_symbol(const uint8_t *bytes, const uint64_t *hset,
                                        const uint16_t *rank_of, uint32_t rank, uint8_t a) {
    const uint64_t f = stage_final(stage_mix(kH0, rank), 1);
    const uint64_t tag = stage_tag(f, 1);
    uint32_t q = (uint32_t)f & (kHsetCap - 1);
    for (uint32_t probe = 0; probe < kHsetCap; probe++) {
        const uint64_t v = hset[q];
        if (v == kEmpty) return 0xFFFFFFFFu;
        if ((v & kTagMask) == tag && bytes[(uint32_t)v] == a) return rank_of[q];
        q = (q + 1) & (kHsetCap - 1);
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

// a coherent 64-bit load through a generic address (shared or global)
__device__ __forceinline__ uint64_t ld_strong_u64(const uint64_t *p) {
    uint64_t v;
    asm volatile("ld.relaxed.gpu.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

// stage problem J with the calling CTA; hset[kHsetCap], rank_of[kHsetCap],
// uniq[kMaxIC] and rank_tab[256] are the caller's scratch
__device__ inline void stage_run(const StageJob &J, uint64_t *hset, uint16_t *rank_of, uint16_t *uniq,
                                 int16_t *rank_tab) {
    __shared__ uint32_t s_err, s_count, s_maxlen, s_total, s_ov, s_np, s_nn;
    __shared__ uint32_t warp_sums[32];

    const uint32_t tid = threadIdx.x, nt = blockDim.x;
    const uint32_t n_str = J.n_pos + J.n_neg;
    const uint8_t *bytes = J.bytes;
    const uint32_t *offs = J.offs;
    const uint32_t total = offs[n_str];

    for (uint32_t q = tid; q < kHsetCap; q += nt) hset[q] = kEmpty;
    for (uint32_t i = tid; i < 256; i += nt) rank_tab[i] = -1;
    for (uint32_t i = tid; i < kMaxWords; i += nt) {
        J.pos_mask[i] = 0;
        J.neg_mask[i] = 0;
    }
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
    __syncthreads();

    // offsets start at 0 and never decrease (device inputs are not checked on
    // the host); every byte must be a symbol; strings must fit the length field
    if (offs[0] != 0) s_err = SE_OFFSETS;
    for (uint32_t k = tid; k < n_str; k += nt)
        if (offs[k + 1] < offs[k]) s_err = SE_OFFSETS;
    __syncthreads();
    if (s_err != SE_OK) {
        if (tid == 0) J.info->status = s_err;
        return;
    }
    for (uint32_t p = tid; p < total; p += nt)
        if (rank_tab[bytes[p]] < 0) s_err = SE_SYMBOL;
    for (uint32_t k = tid; k < n_str; k += nt) atomicMax(&s_maxlen, offs[k + 1] - offs[k]);
    __syncthreads();
    if (s_err == SE_OK && s_maxlen > REI_MAX_STRLEN) s_err = SE_STRLEN;
    __syncthreads();

    // every occurrence (start p, length len) of every string goes into the set
    if (s_err == SE_OK) {
        for (uint32_t p = tid; p < total; p += nt) {
            // string k with offs[k] <= p < offs[k+1] (strings may be empty)
            uint32_t lo = 0, hi = n_str;  // invariant: offs[lo] <= p < offs[hi]
            while (hi - lo > 1) {
                const uint32_t mid = (lo + hi) >> 1;
                if (offs[mid] <= p) lo = mid;
                else hi = mid;
            }
            const uint32_t end = offs[lo + 1];
            uint64_t h = kH0;
            for (uint32_t e = p + 1; e <= end; e++) {
                const uint32_t len = e - p;
                h = stage_mix(h, (uint32_t)rank_tab[bytes[e - 1]]);
                const uint64_t f = stage_final(h, len);
                const uint64_t tag = stage_tag(f, len);
                const uint64_t want = tag | p;
                uint32_t q = (uint32_t)f & (kHsetCap - 1);
                for (uint32_t probe = 0; probe < kHsetCap; probe++) {
                    uint64_t v = ld_strong_u64(&hset[q]);
                    if (v == kEmpty) {
                        const unsigned long long old =
                            atomicCAS((unsigned long long *)&hset[q], kEmpty, want);
                        if (old == kEmpty) {
                            if (atomicAdd(&s_count, 1u) + 2 > kMaxIC) s_err = SE_IC_LARGE;
                            break;
                        }
                        v = old;
                    }
                    if ((v & kTagMask) == tag && same_bytes(bytes, (uint32_t)v, p, len)) break;
                    q = (q + 1) & (kHsetCap - 1);
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

    // the distinct words (unordered), then their shortlex ranks (eps = 0)
    if (tid == 0) s_count = 0;
    __syncthreads();
    for (uint32_t q = tid; q < kHsetCap; q += nt)
        if (hset[q] != kEmpty) uniq[atomicAdd(&s_count, 1u)] = (uint16_t)q;
    __syncthreads();
    const uint32_t U = s_count, n = U + 1;
    for (uint32_t i = tid; i < U; i += nt) {
        const uint64_t vi = hset[uniq[i]];
        const uint32_t si = (uint32_t)vi, li = (uint32_t)(vi >> 32) & 0xFFFu;
        uint32_t r = 1;
        for (uint32_t j = 0; j < U; j++) {
            const uint64_t vj = hset[uniq[j]];
            if (shortlex_less(bytes, rank_tab, (uint32_t)vj, (uint32_t)(vj >> 32) & 0xFFFu, si, li)) r++;
        }
        J.word_start[r] = si;
        J.word_len[r] = li;
        rank_of[uniq[i]] = (uint16_t)r;
    }
    if (tid == 0) {
        J.word_start[0] = 0;
        J.word_len[0] = 0;
    }
    __syncthreads();

    // first rank of every length (all lengths 0..max_len occur: ic is infix-closed)
    uint32_t max_len = 0;
    for (uint32_t r = tid; r < n; r += nt) {
        const uint32_t L = J.word_len[r];
        if (r == 0 || J.word_len[r - 1] != L) J.len_start[L] = r;
    }
    max_len = J.word_len[n - 1];
    if (tid == 0) J.len_start[max_len + 1] = n;

    // guide-table offsets: exclusive scan of |w| + 1 over words in rank order
    const uint32_t per = (n + nt - 1) / nt;
    const uint32_t r0 = min(n, tid * per), r1 = min(n, r0 + per);
    uint32_t local = 0;
    for (uint32_t r = r0; r < r1; r++) local += J.word_len[r] + 1;
    uint32_t off = block_exclusive_scan(local, warp_sums, &s_total);
    for (uint32_t r = r0; r < r1; r++) {
        J.gt_off[r] = off;
        off += J.word_len[r] + 1;
    }
    const uint32_t G = s_total;
    if (tid == 0) J.gt_off[n] = G;
    __syncthreads();
    if (G > J.pair_cap) {
        if (tid == 0) {
            J.info->status = SE_PAIRS;
            J.info->n = n;
            J.info->G = G;
            J.info->max_len = max_len;
        }
        return;
    }

    // guide-table pairs: split k of word r is (prefix of length k, the rest)
    for (uint32_t g = tid; g < G; g += nt) {
        uint32_t lo = 0, hi = n;  // gt_off[lo] <= g < gt_off[hi]
        while (hi - lo > 1) {
            const uint32_t mid = (lo + hi) >> 1;
            if (J.gt_off[mid] <= g) lo = mid;
            else hi = mid;
        }
        const uint32_t k = g - J.gt_off[lo], len = J.word_len[lo], st = J.word_start[lo];
        const uint32_t u = stage_lookup(bytes, hset, rank_of, rank_tab, st, k);
        const uint32_t v = stage_lookup(bytes, hset, rank_of, rank_tab, st + k, len - k);
        if (u >= n || v >= n) s_err = SE_INTERNAL;  // infixes of ic words are in ic
        J.gt_pair[g] = (u & 0xFFFFu) | (v << 16);
    }

    // characteristic sequences of P and N, and of every symbol
    for (uint32_t k = tid; k < n_str; k += nt) {
        const uint32_t r = stage_lookup(bytes, hset, rank_of, rank_tab, offs[k], offs[k + 1] - offs[k]);
        if (r >= n) {
            s_err = SE_INTERNAL;
            continue;
        }
        uint32_t *mask = k < J.n_pos ? J.pos_mask : J.neg_mask;
        atomicOr(&mask[r >> 5], 1u << (r & 31));
    }
    for (uint32_t a = tid; a < J.n_sym; a += nt) {
        const uint32_t r = stage_lookup_symbol(bytes, hset, rank_of, a, J.alphabet[a]);
        if (r < n) J.leaf[a * kMaxWords + (r >> 5)] = 1u << (r & 31);
    }
    __syncthreads();
    const uint32_t W = padded_words(n);
    for (uint32_t b = tid; b < W; b += nt) {
        const uint32_t p = J.pos_mask[b], q = J.neg_mask[b];
        if (p & q) s_ov = 1;
        atomicAdd(&s_np, (uint32_t)__popc(p));
        atomicAdd(&s_nn, (uint32_t)__popc(q));
    }
    __syncthreads();
    if (tid == 0) {
        StageInfo *I = J.info;
        I->status = s_err != SE_OK ? s_err : s_ov ? SE_OVERLAP : SE_OK;
        I->n = n;
        I->W = W;
        I->max_len = max_len;
        I->G = G;
        I->n_pos_set = s_np;
        I->n_neg_set = s_nn;
        I->pos_eps = J.pos_mask[0] & 1u;
        I->neg_eps = J.neg_mask[0] & 1u;
    }
}


}  // namespace rei
