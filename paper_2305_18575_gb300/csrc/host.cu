// host.cu -- host runtime of the REI library: contexts, device memory, the
// solve driver, result formatting, inspection calls, and the batched and
// served forms.  Every step of the search itself runs in the kernels of
// stage.cu and solve.cu; this file only moves inputs and results, sizes
// buffers, and launches.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <deque>
#include <map>
#include <set>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "rei_dev.cuh"
#include "stage_dev.cuh"
#include "args.h"

namespace rei {
cudaError_t launch_solve_batch(const BatchJob *jobs_dev, const BatchArgs *args, uint32_t grid, uint32_t threads,
                               size_t smem, cudaStream_t stream);
cudaError_t solve_batch_occupancy(uint32_t threads, size_t smem, int *blocks_per_sm);
cudaError_t launch_stage(const StageJob *jobs_dev, uint32_t n_jobs, cudaStream_t stream);
cudaError_t launch_serve(const ServeArgs *args, uint32_t grid, uint32_t threads, size_t smem, cudaStream_t stream);
cudaError_t launch_solve_fused(const FuseArgs *args, uint32_t grid, uint32_t threads, size_t smem,
                               cudaStream_t stream);
cudaError_t solve_fused_occupancy(uint32_t threads, size_t smem, int *blocks_per_sm);
cudaError_t serve_occupancy(uint32_t threads, size_t smem, int *blocks_per_sm);
size_t stage_smem_bytes();
cudaError_t launch_solve(const SolveJob *job, uint32_t grid, uint32_t threads, size_t smem,
                         cudaStream_t stream);
cudaError_t solve_occupancy(uint32_t threads, size_t smem, int *blocks_per_sm);
cudaError_t solve_smem_max(size_t *bytes);
cudaError_t solve_batch_smem_max(size_t *bytes);
cudaError_t launch_solve_groups(const BatchJob *jobs_dev, const GroupArgs *args, uint32_t grid, uint32_t threads,
                                size_t smem, cudaStream_t stream);
cudaError_t solve_groups_occupancy(uint32_t threads, size_t smem, int *blocks_per_sm);
cudaError_t solve_groups_smem_max(size_t *bytes);
cudaError_t launch_rehash(const SolveJob *job, uint32_t count, uint32_t grid, cudaStream_t stream);
size_t solve_smem_bytes(uint32_t W, uint32_t n, uint32_t G, uint32_t max_len, uint32_t seg_cap,
                        bool gt_in_smem, uint32_t warps, uint32_t small_rows = 0);
}  // namespace rei

using namespace rei;


namespace {

double now_ms() {
    return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

struct DevBuf {
    void *p = nullptr;
    size_t bytes = 0;
};

}  // namespace

struct rei_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    rei_alloc alloc{};
    bool has_alloc = false;
    int sm_count = 0;
    size_t smem_optin = 0;
    uint64_t launches = 0;

    int64_t opt_chunk = 0, opt_grid = 0, opt_keep = 0, opt_cache_init = 0, opt_solo_tiles = -1, opt_small_rows = -1;
    int64_t opt_fused = 1, opt_exact = 1;
    uint64_t opt_handover = 1ull << 22;  // levels of more candidates leave the fused launch
    uint64_t opt_yield_us = 500;         // batched / served problems longer than this continue on the whole GPU
    bool phases = getenv("REI_PHASES") != nullptr;  // per-solve timing report on stderr (diagnostics)
    unsigned long long fused_launch_id = 0;         // ids of this context's fused launches (only grow)
    size_t smem_sm = 0;  // shared memory per SM

    // staging
    DevBuf in_bytes, in_offs, stage_job, stage_info, word_start, word_len, len_start, gt_off, gt_pair,
        pos, neg, leaf;
    uint32_t pair_cap = 1u << 16;
    // search
    DevBuf cs, bp_op, bp_l, bp_r, table, minidx, tmp, pending, slotpos, bitmap, blk, lvl_start, lvl_count,
        state, solve_job, tstack, trace, used, plan;
    DevBuf seen;               // bitmap of cached 1-word languages (2^kSeenBits bits)
    bool table_clean = false;  // the search kernel leaves the table (and seen) empty after a normal end
    uint64_t table_extent = 0; // slots of the table (and minidx) that may hold entries: beyond, all empty
    // batched form
    DevBuf b_in, b_sjobs, b_sinfo, b_stage, b_jobs, b_out, b_tree, b_queue;
    DevBuf s_cs, s_bp_op, s_bp_l, s_bp_r, s_used, s_table, s_tmp, s_pend, s_slotpos, s_bitmap, s_blk, s_lvl,
        s_state, s_tstack;
    DevBuf g_idx, g_blk, g_plan, g_tmp, g_pend, g_slotpos, g_bitmap;  // parked searches continued in their slots
    uint64_t slot_rows = 0, slot_cs_words = 0, slot_table = 0, slot_tmp_words = 0, slot_chunk = 0;
    uint32_t slot_count = 0;
    bool slots_clean = false;
    int batch_warps = 0;       // autotuned warps per CTA of the batched launch (0 = not yet)
    uint32_t batch_chunk = 0;  // autotuned candidates per dedup chunk in a slot (0 = not yet)
    // pinned host scratch (and its device address, or null)
    uint8_t *h_pin = nullptr, *h_pin_dev = nullptr;
    size_t h_pin_bytes = 0;
    bool pin_clean = false;  // no copy from or to h_pin is in flight (the last user synchronised)

    // last solve (for rei_cache_dump)
    bool last_valid = false;
    uint32_t last_W = 0, last_size = 0, last_max_cost = 0;

    // contexts of its own (streams, buffers) on which a batch continues its
    // parked searches side by side, each launch on a share of the GPU
    std::vector<rei_ctx *> helpers;

    cudaEvent_t ev[2] = {nullptr, nullptr};
    std::mutex mu;
};

namespace {

#define CK(x)                                                                                     \
    do {                                                                                          \
        cudaError_t _e = (x);                                                                     \
        if (_e != cudaSuccess) {                                                                  \
            fprintf(stderr, "rei: %s failed: %s (%s:%d)\n", #x, cudaGetErrorString(_e), __FILE__, \
                    __LINE__);                                                                    \
            return REI_ECUDA;                                                                     \
        }                                                                                         \
    } while (0)

void *dev_alloc(rei_ctx *c, size_t bytes) {
    if (bytes == 0) bytes = 16;
    void *p = nullptr;
    if (c->has_alloc) return c->alloc.alloc(c->alloc.user, bytes, (void *)c->stream);
    if (cudaMallocAsync(&p, bytes, c->stream) != cudaSuccess) return nullptr;
    return p;
}

void dev_free(rei_ctx *c, DevBuf &b) {
    if (!b.p) return;
    if (c->has_alloc) c->alloc.free(c->alloc.user, b.p, b.bytes, (void *)c->stream);
    else cudaFreeAsync(b.p, c->stream);
    b.p = nullptr;
    b.bytes = 0;
}

// grow-only buffer; contents are not kept
rei_status ensure(rei_ctx *c, DevBuf &b, size_t bytes) {
    if (b.bytes >= bytes && b.p) return REI_OK;
    dev_free(c, b);
    size_t want = std::max<size_t>(bytes, 256);
    b.p = dev_alloc(c, want);
    if (!b.p) return REI_OOM;
    b.bytes = want;
    return REI_OK;
}

// grow keeping the first `keep` bytes
rei_status grow_keep(rei_ctx *c, DevBuf &b, size_t bytes, size_t keep) {
    if (b.bytes >= bytes && b.p) return REI_OK;
    void *np = dev_alloc(c, bytes);
    if (!np) return REI_OOM;
    if (b.p && keep) {
        if (cudaMemcpyAsync(np, b.p, std::min(keep, b.bytes), cudaMemcpyDeviceToDevice, c->stream) != cudaSuccess)
            return REI_ECUDA;
    }
    dev_free(c, b);
    b.p = np;
    b.bytes = bytes;
    return REI_OK;
}

// Empty the uniqueness table and its first-candidate array where they may
// hold entries (the first max(table_extent, at_least) slots; beyond them they
// are empty), so that a context that once solved a large problem does not
// clear its whole table for every small one.
rei_status clear_table(rei_ctx *c, uint64_t at_least) {
    const uint64_t ext = std::max(c->table_extent, at_least);
    const uint64_t t = std::min<uint64_t>(ext, c->table.bytes / 8), m = std::min<uint64_t>(ext, c->minidx.bytes / 4);
    if (t) CK(cudaMemsetAsync(c->table.p, 0xFF, 8 * t, c->stream));
    if (m) CK(cudaMemsetAsync(c->minidx.p, 0xFF, 4 * m, c->stream));
    c->table_extent = 0;
    return REI_OK;
}

rei_status ensure_pinned(rei_ctx *c, size_t bytes) {
    c->pin_clean = false;  // the caller is about to use it
    if (c->h_pin_bytes >= bytes) return REI_OK;
    if (c->h_pin) {
        cudaStreamSynchronize(c->stream);
        cudaFreeHost(c->h_pin);
        c->h_pin = nullptr;
    }
    size_t want = std::max<size_t>(bytes, 1 << 16);
    if (cudaMallocHost((void **)&c->h_pin, want) != cudaSuccess) return REI_ECUDA;
    c->h_pin_bytes = want;
    // (the device's address of the buffer, for kernels that write results there)
    void *dev = nullptr;
    c->h_pin_dev = cudaHostGetDevicePointer(&dev, c->h_pin, 0) == cudaSuccess ? (uint8_t *)dev : nullptr;
    if (!c->h_pin_dev) cudaGetLastError();
    return REI_OK;
}

uint64_t budget_cap(uint64_t budget, uint32_t n) {
    const uint64_t per = 4ull * padded_words(n) + 28;
    return std::min<uint64_t>(budget / per, 0x7FFF0000ull);
}

uint64_t pow2_at_least(uint64_t x) {
    uint64_t p = 1;
    while (p < x) p <<= 1;
    return p;
}

// ---------------------------------------------------------------------------
// result formatting (host): postfix tokens -> pretty string with the
// precedence * ? > concatenation > +, parentheses only where needed

struct PNode {
    uint8_t k, a;
    int l, r;
};

int prec(uint8_t k) { return k == '+' ? 0 : k == '.' ? 1 : 2; }

void print_node(const std::vector<PNode> &T, int x, const uint8_t *alpha, std::string &out, int need) {
    const PNode &t = T[x];
    const bool par = prec(t.k) < need;
    if (par) out += '(';
    switch (t.k) {
    case 'a': out += (char)alpha[t.a]; break;
    case 'e': out += "\xce\xb5"; break;
    case '0': out += "\xe2\x88\x85"; break;
    case '?':
    case '*':
        print_node(T, t.l, alpha, out, 2);
        out += (char)t.k;
        break;
    case '.':
        print_node(T, t.l, alpha, out, 1);
        print_node(T, t.r, alpha, out, 1);
        break;
    default:
        print_node(T, t.l, alpha, out, 0);
        out += '+';
        print_node(T, t.r, alpha, out, 0);
        break;
    }
    if (par) out += ')';
}

std::string format_regex(const uint8_t *tok, uint32_t ntok, const uint8_t *alpha) {
    std::vector<PNode> T;
    std::vector<int> st;
    for (uint32_t i = 0; i < ntok; i++) {
        const uint8_t k = tok[2 * i], a = tok[2 * i + 1];
        if (k == 'a' || k == 'e' || k == '0') {
            T.push_back({k, a, -1, -1});
        } else if (k == '?' || k == '*') {
            if (st.empty()) return "";
            T.push_back({k, 0, st.back(), -1});
            st.pop_back();
        } else {
            if (st.size() < 2) return "";
            const int r = st.back();
            st.pop_back();
            const int l = st.back();
            st.pop_back();
            T.push_back({k, 0, l, r});
        }
        st.push_back((int)T.size() - 1);
    }
    if (st.size() != 1) return "";
    std::string out;
    print_node(T, st[0], alpha, out, 0);
    return out;
}

// ---------------------------------------------------------------------------
// argument checks and input upload

struct Staged {
    StageInfo info;
    uint64_t h2d = 0, d2h = 0;
    double ms_kernel = 0;
};

// stage problem p on the device; inputs end up in ctx buffers
rei_status stage_problem(rei_ctx *c, const rei_problem *p, Staged &out) {
    const uint32_t n_str = p->n_pos + p->n_neg;
    uint64_t total;
    const uint8_t *dbytes;
    const uint32_t *doffs;
    if (p->flags & REI_F_DEVICE_INPUT) {
        total = p->total_bytes;
        dbytes = p->bytes;
        doffs = p->offsets;
        if (n_str == 0) {
            // still need an offsets array with one zero entry
            rei_status s = ensure(c, c->in_offs, 4);
            if (s) return s;
            CK(cudaMemsetAsync(c->in_offs.p, 0, 4, c->stream));
            doffs = (const uint32_t *)c->in_offs.p;
        }
    } else {
        total = n_str ? p->offsets[n_str] : 0;
        const size_t ob = 4ull * (n_str + 1);
        rei_status s = ensure_pinned(c, total + ob + 16);
        if (s) return s;
        s = ensure(c, c->in_bytes, total + 16);
        if (s) return s;
        s = ensure(c, c->in_offs, ob);
        if (s) return s;
        CK(cudaStreamSynchronize(c->stream));  // pinned buffer reuse
        uint32_t *ho = (uint32_t *)c->h_pin;
        uint8_t *hb = c->h_pin + ob;
        if (n_str) {
            memcpy(ho, p->offsets, ob);
            if (total) memcpy(hb, p->bytes, total);
        } else {
            ho[0] = 0;
        }
        CK(cudaMemcpyAsync(c->in_offs.p, ho, ob, cudaMemcpyHostToDevice, c->stream));
        if (total) CK(cudaMemcpyAsync(c->in_bytes.p, hb, total, cudaMemcpyHostToDevice, c->stream));
        out.h2d += ob + total;
        dbytes = (const uint8_t *)c->in_bytes.p;
        doffs = (const uint32_t *)c->in_offs.p;
    }
    if (total > 0xFFFFFFF0ull) return REI_EINVAL;

    for (int attempt = 0; attempt < 2; attempt++) {
        rei_status s;
        if ((s = ensure(c, c->stage_job, sizeof(StageJob) + sizeof(StageInfo)))) return s;
        if ((s = ensure(c, c->word_start, 4ull * kMaxIC))) return s;
        if ((s = ensure(c, c->word_len, 4ull * kMaxIC))) return s;
        if ((s = ensure(c, c->len_start, 4ull * (REI_MAX_STRLEN + 2)))) return s;
        if ((s = ensure(c, c->gt_off, 4ull * (kMaxIC + 1)))) return s;
        if ((s = ensure(c, c->gt_pair, 4ull * c->pair_cap))) return s;
        if ((s = ensure(c, c->pos, 4ull * kMaxWords))) return s;
        if ((s = ensure(c, c->neg, 4ull * kMaxWords))) return s;
        if ((s = ensure(c, c->leaf, 4ull * kMaxWords * p->n_sym))) return s;
        if ((s = ensure_pinned(c, sizeof(StageJob) + sizeof(StageInfo)))) return s;
        CK(cudaStreamSynchronize(c->stream));
        StageJob *hj = (StageJob *)c->h_pin;
        memset(hj, 0, sizeof(StageJob));
        hj->bytes = dbytes;
        hj->offs = doffs;
        hj->n_pos = p->n_pos;
        hj->n_neg = p->n_neg;
        memcpy(hj->alphabet, p->alphabet, p->n_sym);
        hj->n_sym = p->n_sym;
        hj->total_bytes = (uint32_t)total;
        StageJob *dj = (StageJob *)c->stage_job.p;
        hj->info = (StageInfo *)(dj + 1);
        hj->word_start = (uint32_t *)c->word_start.p;
        hj->word_len = (uint32_t *)c->word_len.p;
        hj->len_start = (uint32_t *)c->len_start.p;
        hj->gt_off = (uint32_t *)c->gt_off.p;
        hj->gt_pair = (uint32_t *)c->gt_pair.p;
        hj->pair_cap = c->pair_cap;
        hj->pos_mask = (uint32_t *)c->pos.p;
        hj->neg_mask = (uint32_t *)c->neg.p;
        hj->leaf = (uint32_t *)c->leaf.p;
        CK(cudaMemcpyAsync(dj, hj, sizeof(StageJob), cudaMemcpyHostToDevice, c->stream));
        CK(cudaMemsetAsync(hj->info, 0, sizeof(StageInfo), c->stream));
        out.h2d += sizeof(StageJob);
        CK(cudaEventRecord(c->ev[0], c->stream));
        CK(launch_stage(dj, 1, c->stream));
        CK(cudaEventRecord(c->ev[1], c->stream));
        c->launches++;
        StageInfo *hi = (StageInfo *)(c->h_pin + sizeof(StageJob));
        CK(cudaMemcpyAsync(hi, hj->info, sizeof(StageInfo), cudaMemcpyDeviceToHost, c->stream));
        CK(cudaStreamSynchronize(c->stream));
        out.d2h += sizeof(StageInfo);
        out.info = *hi;
        float ms = 0;
        CK(cudaEventElapsedTime(&ms, c->ev[0], c->ev[1]));
        out.ms_kernel = ms;
        if (out.info.status == SE_PAIRS) {
            c->pair_cap = (uint32_t)pow2_at_least(out.info.G);
            continue;
        }
        break;
    }
    return out.info.status == SE_OK ? REI_OK : REI_EINVAL;
}

void fill_stats(rei_result *r, const StageInfo &I) {
    r->stats.n_ic = I.n;
    r->stats.words = I.W;
    r->stats.max_len = I.max_len;
    r->stats.guide_pairs = I.G;
}

rei_status write_outputs(rei_result *out, const uint8_t *tok, uint32_t ntok, const uint8_t *alpha) {
    const std::string s = format_regex(tok, ntok, alpha);
    out->regex_len = s.size();
    out->tree_len = 2ull * ntok;
    rei_status st = REI_OK;
    if (out->regex) {
        if (out->regex_cap >= s.size() + 1) {
            memcpy(out->regex, s.data(), s.size());
            out->regex[s.size()] = 0;
        } else {
            st = REI_EBUFSZ;
        }
    } else if (out->regex_cap) {
        st = REI_EINVAL;
    }
    if (out->tree) {
        if (out->tree_cap >= 2ull * ntok) memcpy(out->tree, tok, 2ull * ntok);
        else st = REI_EBUFSZ;
    }
    return st;
}

// ---------------------------------------------------------------------------
// the plain solve, staged inside its search launch

// Pinned host layout of a plain solve: the job of a relaunch, then the state,
// the answer's tokens and the staging report (the device state buffer holds
// the same three, so one copy brings them back), then the inputs.
size_t state_bytes(uint32_t max_cost) {
    return (sizeof(SolveState) + 2ull * (max_cost + 1) + 15) & ~size_t(15);
}

// Stage and search in one cooperative launch (k_solve_fused).  REI_OK: the
// launch ran; *hst holds its final state (an answer, not found, out of
// memory, a timeout, or a request for more memory that the caller's relaunch
// loop serves) and sg.info the staging report.  REI_EBUSY: the problem needs
// the separate staging launch (|ic| beyond what the launch stages, a guide
// table beyond the pair buffer, shared memory, or an invalid input, which the
// staging launch reports).
rei_status run_fused(rei_ctx *c, const rei_problem *p, Staged &sg, double &ms_search, uint32_t &grid_out,
                     uint64_t &h2d, uint64_t &d2h) {
    rei_status s;
    const double th0 = now_ms();
    const uint32_t n_str = p->n_pos + p->n_neg, max_cost = p->max_cost;
    const bool dev_in = (p->flags & REI_F_DEVICE_INPUT) != 0;
    const uint64_t total = dev_in ? p->total_bytes : (n_str ? p->offsets[n_str] : 0);
    if (total > kServeMaxBytes) return REI_EBUSY;
    const size_t sb = state_bytes(max_cost);
    const size_t ob = (4ull * (n_str + 1) + 15) & ~size_t(15);
    const size_t pin_in = sizeof(SolveJob) + sb + sizeof(StageInfo);
    const bool pin_was_clean = c->pin_clean;
    if ((s = ensure_pinned(c, pin_in + (dev_in ? 0 : ob + total + 16)))) return s;
    if (!pin_was_clean) CK(cudaStreamSynchronize(c->stream));  // pinned buffer reuse

    // inputs
    const uint8_t *dbytes;
    const uint32_t *doffs;
    if (dev_in) {
        dbytes = p->bytes;
        doffs = p->offsets;
        if (n_str == 0) {
            if ((s = ensure(c, c->in_offs, 16))) return s;
            CK(cudaMemsetAsync(c->in_offs.p, 0, 4, c->stream));
            doffs = (const uint32_t *)c->in_offs.p;
        }
    } else {
        if ((s = ensure(c, c->in_bytes, ob + total + 16))) return s;
        uint8_t *hp = c->h_pin + pin_in;
        uint32_t *ho = (uint32_t *)hp;
        if (n_str) memcpy(ho, p->offsets, 4ull * (n_str + 1));
        else ho[0] = 0;
        if (total) memcpy(hp + ob, p->bytes, total);
        CK(cudaMemcpyAsync(c->in_bytes.p, hp, ob + total, cudaMemcpyHostToDevice, c->stream));
        h2d += ob + total;
        doffs = (const uint32_t *)c->in_bytes.p;
        dbytes = (const uint8_t *)c->in_bytes.p + ob;
    }

    // staged-problem buffers
    if ((s = ensure(c, c->word_start, 4ull * kMaxIC))) return s;
    if ((s = ensure(c, c->word_len, 4ull * kMaxIC))) return s;
    if ((s = ensure(c, c->len_start, 4ull * (REI_MAX_STRLEN + 2)))) return s;
    if ((s = ensure(c, c->gt_off, 4ull * (kMaxIC + 1)))) return s;
    if ((s = ensure(c, c->gt_pair, 4ull * c->pair_cap))) return s;
    if ((s = ensure(c, c->pos, 4ull * kMaxWords))) return s;
    if ((s = ensure(c, c->neg, 4ull * kMaxWords))) return s;
    if ((s = ensure(c, c->leaf, 4ull * kMaxWords * p->n_sym))) return s;

    // search buffers, sized before the staged sizes are known: the rows a
    // previous solve allocated (at least 64 Ki), languages of up to the
    // previous solve's width; the launch derives its cache and chunk sizes
    // from what is there
    uint64_t rows = c->opt_cache_init > 0 ? (uint64_t)c->opt_cache_init : (1ull << 16);
    if (c->opt_cache_init <= 0 && c->bp_l.p && c->bp_r.p && c->bp_op.p && c->used.p) {
        const uint64_t have = std::min<uint64_t>({(uint64_t)(c->bp_l.bytes / 4), (uint64_t)(c->bp_r.bytes / 4),
                                                  (uint64_t)c->bp_op.bytes, (uint64_t)(c->used.bytes / 4)});
        rows = std::max<uint64_t>(rows, std::min<uint64_t>(have, 1ull << 20));
    }
    const uint64_t wguess = std::max<uint32_t>(2u, c->last_W);
    if ((s = ensure(c, c->cs, 4ull * wguess * rows))) return s;
    if ((s = ensure(c, c->bp_op, rows))) return s;
    if ((s = ensure(c, c->bp_l, 4ull * rows))) return s;
    if ((s = ensure(c, c->bp_r, 4ull * rows))) return s;
    if ((s = ensure(c, c->used, 4ull * rows))) return s;
    const uint64_t tslots = pow2_at_least(std::max<uint64_t>(4 * rows, 1024));
    {
        // a reallocated table (even at the same address) holds garbage
        const void *before = c->table.p, *mbefore = c->minidx.p;
        const size_t before_bytes = c->table.bytes, mbefore_bytes = c->minidx.bytes;
        if ((s = ensure(c, c->table, 8ull * tslots))) return s;
        if ((s = ensure(c, c->minidx, 4ull * tslots))) return s;
        if (c->table.p != before || c->table.bytes != before_bytes || c->minidx.p != mbefore ||
            c->minidx.bytes != mbefore_bytes) {
            c->table_clean = false;
            c->table_extent = std::max<uint64_t>(c->table.bytes / 8, c->minidx.bytes / 4);
        }
    }
    const uint64_t chunk_words = c->opt_chunk > 0 ? (uint64_t)c->opt_chunk : (1ull << 22);
    if ((s = ensure(c, c->tmp, std::max<uint64_t>(4ull * 2 * chunk_words, 4ull * 64 * 4096)))) return s;
    if ((s = ensure(c, c->pending, 4ull * chunk_words))) return s;
    if ((s = ensure(c, c->slotpos, 4ull * chunk_words))) return s;
    {
        const void *before = c->bitmap.p;
        const size_t before_bytes = c->bitmap.bytes;
        if ((s = ensure(c, c->bitmap, 4ull * ((chunk_words + 31) / 32)))) return s;
        if (c->bitmap.p != before || c->bitmap.bytes != before_bytes) c->table_clean = false;
    }
    const uint32_t threads = 512;  // (the launch bounds of k_solve_fused: one 16-warp CTA per SM)
    const size_t smem = c->smem_optin > 8192 ? c->smem_optin - 8192 : 0;  // (its static shared memory and a reserve)
    int bps = 0;
    CK(solve_fused_occupancy(threads, smem, &bps));
    if (bps < 1) return REI_EBUSY;
    uint32_t grid = std::min<uint32_t>((uint32_t)(c->sm_count * bps), kMaxTeam);
    if (c->opt_grid > 0 && (uint32_t)c->opt_grid < grid) grid = (uint32_t)c->opt_grid;
    if ((s = ensure(c, c->blk, 4ull * grid))) return s;
    if ((s = ensure(c, c->lvl_start, 8ull * (max_cost + 2)))) return s;
    if ((s = ensure(c, c->lvl_count, 8ull * (max_cost + 2)))) return s;
    {
        // a new state buffer starts zeroed: the launch id it holds is then
        // always below the next launch's (the launch resets the rest itself)
        const void *before = c->state.p;
        if ((s = ensure(c, c->state, sb + sizeof(StageInfo)))) return s;
        if (c->state.p != before) CK(cudaMemsetAsync(c->state.p, 0, c->state.bytes, c->stream));
    }
    if ((s = ensure(c, c->solve_job, sizeof(SolveJob)))) return s;
    if ((s = ensure(c, c->tstack, 16ull * (max_cost + 2)))) return s;
    if ((s = ensure(c, c->trace, 4ull * grid))) return s;
    if ((s = ensure(c, c->plan, 8 * plan_words(2 * max_cost + 4)))) return s;
    if (c->opt_exact && !c->seen.p) {
        if ((s = ensure(c, c->seen, (1ull << kSeenBits) / 8))) return s;
        c->table_clean = false;
    }
    if (!c->table_clean) {
        if ((s = clear_table(c, 0))) return s;
        CK(cudaMemsetAsync(c->bitmap.p, 0, c->bitmap.bytes, c->stream));
        if (c->seen.p) CK(cudaMemsetAsync(c->seen.p, 0, c->seen.bytes, c->stream));
    }
    c->table_clean = false;
    c->table_extent = std::max(c->table_extent, tslots);

    FuseArgs F;
    memset(&F, 0, sizeof F);
    StageJob &sj = F.sj;
    sj.bytes = dbytes;
    sj.offs = doffs;
    sj.n_pos = p->n_pos;
    sj.n_neg = p->n_neg;
    memcpy(sj.alphabet, p->alphabet, p->n_sym);
    sj.n_sym = p->n_sym;
    sj.total_bytes = (uint32_t)total;
    sj.info = (StageInfo *)((uint8_t *)c->state.p + sb);
    sj.word_start = (uint32_t *)c->word_start.p;
    sj.word_len = (uint32_t *)c->word_len.p;
    sj.len_start = (uint32_t *)c->len_start.p;
    sj.gt_off = (uint32_t *)c->gt_off.p;
    sj.gt_pair = (uint32_t *)c->gt_pair.p;
    sj.pair_cap = c->pair_cap;
    sj.pos_mask = (uint32_t *)c->pos.p;
    sj.neg_mask = (uint32_t *)c->neg.p;
    sj.leaf = (uint32_t *)c->leaf.p;
    SolveJob &j = F.tmpl;
    j.n_sym = p->n_sym;
    j.gt_off = (const uint32_t *)c->gt_off.p;
    j.gt_pair = (const uint32_t *)c->gt_pair.p;
    j.len_start = (const uint32_t *)c->len_start.p;
    j.pos_mask = (const uint32_t *)c->pos.p;
    j.neg_mask = (const uint32_t *)c->neg.p;
    j.leaf = (const uint32_t *)c->leaf.p;
    j.leaf_stride = kMaxWords;
    fill_leaves(p, &j.cmin, j.leaf_cost, j.leaf_sym);
    j.c[0] = p->costs.c_sym;
    j.c[1] = p->costs.c_opt;
    j.c[2] = p->costs.c_star;
    j.c[3] = p->costs.c_cat;
    j.c[4] = p->costs.c_alt;
    j.max_cost = max_cost;
    j.max_errors = p->max_errors;
    j.flags = p->flags & ~REI_F_DEVICE_INPUT;
    j.cs = (uint32_t *)c->cs.p;
    j.bp_op = (uint8_t *)c->bp_op.p;
    j.bp_l = (uint32_t *)c->bp_l.p;
    j.bp_r = (uint32_t *)c->bp_r.p;
    j.used = (uint32_t *)c->used.p;
    j.table = (unsigned long long *)c->table.p;
    j.table_mask = tslots - 1;
    j.minidx = (uint32_t *)c->minidx.p;
    j.exact = c->opt_exact ? 1u : 0u;  // allowed; the launch decides from the staged size
    j.tmp = (uint32_t *)c->tmp.p;
    j.pending = (uint32_t *)c->pending.p;
    j.slotpos = (uint32_t *)c->slotpos.p;
    j.bitmap = (uint32_t *)c->bitmap.p;
    j.blk = (uint32_t *)c->blk.p;
    j.lvl_start = (int64_t *)c->lvl_start.p;
    j.lvl_count = (int64_t *)c->lvl_count.p;
    j.seg_cap = 2 * max_cost + 4;
    j.plan = (uint64_t *)c->plan.p;
    j.st = (SolveState *)c->state.p;
    j.tree = (uint8_t *)c->state.p + sizeof(SolveState);
    j.tstack = (uint32_t *)c->tstack.p;
    j.trace = (uint32_t *)c->trace.p;
    j.solo_tiles = c->opt_solo_tiles >= 0 ? (uint32_t)c->opt_solo_tiles : 64;
    F.job = (SolveJob *)c->solve_job.p;
    F.mem_budget = p->mem_budget;
    F.rows_alloc = rows;
    F.cs_words = c->cs.bytes / 4;
    F.tmp_words = c->tmp.bytes / 4;
    F.pend_cap = std::min<uint64_t>({(uint64_t)(c->pending.bytes / 4), (uint64_t)(c->slotpos.bytes / 4),
                                     (uint64_t)c->bitmap.bytes * 8});
    F.table_slots = tslots;
    F.chunk_opt = c->opt_chunk > 0 ? (uint64_t)c->opt_chunk : 0;
    F.small_opt = c->opt_small_rows < 0 ? 0xFFFFFFFFu : (uint32_t)c->opt_small_rows;
    F.smem_cap = (uint32_t)smem;
    F.handover = c->opt_handover;
    F.seen = (uint32_t *)c->seen.p;
    F.seen_bits = c->seen.p ? kSeenBits : 0;
    F.launch_id = ++c->fused_launch_id;
    // the launch writes its final state into the pinned buffer itself
    F.host_out = c->h_pin_dev ? (unsigned long long *)(c->h_pin_dev + sizeof(SolveJob)) : nullptr;
    F.out_words = (sb + sizeof(StageInfo)) / 8;

    const double th1 = now_ms();
    CK(cudaEventRecord(c->ev[0], c->stream));
    CK(launch_solve_fused(&F, grid, threads, smem, c->stream));
    CK(cudaEventRecord(c->ev[1], c->stream));
    const double th2 = now_ms();
    c->launches++;
    uint8_t *hs = c->h_pin + sizeof(SolveJob);
    if (!F.host_out) CK(cudaMemcpyAsync(hs, c->state.p, sb + sizeof(StageInfo), cudaMemcpyDeviceToHost, c->stream));
    const double th3 = now_ms();
    CK(cudaStreamSynchronize(c->stream));
    if (c->phases)
        fprintf(stderr, "rei host (fused): setup %.1f us, launch %.1f us, read-back issue %.1f us, wait %.1f us\n",
                (th1 - th0) * 1e3, (th2 - th1) * 1e3, (th3 - th2) * 1e3, (now_ms() - th3) * 1e3);
    c->pin_clean = true;
    d2h += sb + sizeof(StageInfo);
    float ms = 0;
    CK(cudaEventElapsedTime(&ms, c->ev[0], c->ev[1]));
    ms_search += ms;
    grid_out = grid;
    memcpy(&sg.info, hs + sb, sizeof(StageInfo));
    const SolveState *hst = (const SolveState *)hs;
    if (hst->status == ST_RESTAGE) {
        // nothing entered the table: it is still clean
        c->table_clean = true;
        return REI_EBUSY;
    }
    return REI_OK;
}

// ---------------------------------------------------------------------------
// the plain solve

// A search that a batched or served CTA left in its memory slot (ST_NEED_MEM:
// its time allowance ran out, or it outgrew the slot), continued on the whole
// GPU from the slot's cached levels instead of solved again from level 1.
struct SlotResume {
    const SlotMem *m;
    uint32_t slot;
};

constexpr uint32_t kBatchHelpers = 8;  // parked searches of a batch continued side by side, at most

// Copy a parked slot's search into the context: the state into the pinned
// state area, the cached rows, back-pointers and level table into the
// context's buffers; clear what the continued search needs cleared.  The
// caller has staged the problem into the context (same |ic| and W).
rei_status load_slot(rei_ctx *c, const rei_problem *p, const StageInfo &I, const SlotResume &rs, uint64_t &d2h) {
    const SlotMem &m = *rs.m;
    const uint64_t so = rs.slot;
    const uint32_t W = I.W, max_cost = p->max_cost;
    rei_status s;
    if ((s = ensure_pinned(c, sizeof(SolveJob) + state_bytes(max_cost) + sizeof(StageInfo)))) return s;
    CK(cudaStreamSynchronize(c->stream));  // pinned buffer reuse
    SolveState *hst = (SolveState *)(c->h_pin + sizeof(SolveJob));
    CK(cudaMemcpyAsync(hst, m.state + so, sizeof(SolveState), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    d2h += sizeof(SolveState);
    if (hst->status != ST_NEED_MEM || W > m.cs_words / m.rows || hst->size > m.rows) return REI_ECUDA;
    const uint64_t rows = hst->size, alloc = std::max<uint64_t>(rows, 1);
    if ((s = ensure(c, c->cs, 4ull * W * alloc))) return s;
    if ((s = ensure(c, c->bp_op, alloc))) return s;
    if ((s = ensure(c, c->bp_l, 4ull * alloc))) return s;
    if ((s = ensure(c, c->bp_r, 4ull * alloc))) return s;
    if ((s = ensure(c, c->used, 4ull * alloc))) return s;
    if ((s = ensure(c, c->lvl_start, 8ull * (max_cost + 2)))) return s;
    if ((s = ensure(c, c->lvl_count, 8ull * (max_cost + 2)))) return s;
    if (rows) {
        CK(cudaMemcpyAsync(c->cs.p, m.cs + so * m.cs_words, 4ull * W * rows, cudaMemcpyDeviceToDevice, c->stream));
        CK(cudaMemcpyAsync(c->bp_op.p, m.bp_op + so * m.rows, rows, cudaMemcpyDeviceToDevice, c->stream));
        CK(cudaMemcpyAsync(c->bp_l.p, m.bp_l + so * m.rows, 4ull * rows, cudaMemcpyDeviceToDevice, c->stream));
        CK(cudaMemcpyAsync(c->bp_r.p, m.bp_r + so * m.rows, 4ull * rows, cudaMemcpyDeviceToDevice, c->stream));
    }
    const int64_t *lv = m.lvl + so * 2 * (kMaxCost + 2);
    CK(cudaMemcpyAsync(c->lvl_start.p, lv, 8ull * (max_cost + 2), cudaMemcpyDeviceToDevice, c->stream));
    CK(cudaMemcpyAsync(c->lvl_count.p, lv + (kMaxCost + 2), 8ull * (max_cost + 2), cudaMemcpyDeviceToDevice,
                       c->stream));
    // the continued search rebuilds the table from the rows; its survivor
    // bitmap and seen bitmap must start empty
    // (a bitmap allocated later is cleared when it is allocated)
    if (!c->table_clean) {
        if (c->bitmap.p) CK(cudaMemsetAsync(c->bitmap.p, 0, c->bitmap.bytes, c->stream));
        if (c->seen.p) CK(cudaMemsetAsync(c->seen.p, 0, c->seen.bytes, c->stream));
    }
    c->table_clean = false;
    return REI_OK;
}

rei_status solve_one(rei_ctx *c, const rei_problem *p, rei_result *out, const SlotResume *rs = nullptr) {
    const double t0 = now_ms();
    const uint64_t l0 = c->launches;
    memset(&out->stats, 0, sizeof(out->stats));
    out->status = REI_EINVAL;
    out->cost = 0;
    out->regex_len = 0;
    out->tree_len = 0;
    c->last_valid = false;
    rei_status s = check_problem(p);
    if (s) return s;
    if (!p->offsets && p->n_pos + p->n_neg) return REI_EINVAL;

    Staged sg;
    double ms_search = 0;
    uint32_t search_launches = 0, grid = 0;
    uint64_t h2d = 0, d2h = 0;
    // staging inside the search launch when the launch can hold the problem;
    // a search continued from a memory slot stages on its own, then starts
    // from the slot's state as if a first launch had run its first part
    bool fused = false;
    if (rs) {
        s = stage_problem(c, p, sg);
        h2d += sg.h2d;
        d2h += sg.d2h;
        fill_stats(out, sg.info);
        if (s == REI_OK) s = load_slot(c, p, sg.info, *rs, d2h);
        if (s) {
            out->status = s;
            return s;
        }
        fused = true;
    } else if (c->opt_fused) {
        s = run_fused(c, p, sg, ms_search, grid, h2d, d2h);
        if (s == REI_OK) {
            fused = true;
            search_launches = 1;
        } else if (s != REI_EBUSY) {
            out->status = s;
            return s;
        }
    }
    if (!fused) {
        s = stage_problem(c, p, sg);
        h2d += sg.h2d;
        d2h += sg.d2h;
    }
    if (!rs) fill_stats(out, sg.info);
    if (!fused && s) {
        out->status = s;
        return s;
    }
    const double t_stage = now_ms();
    const StageInfo &I = sg.info;
    const uint32_t n = I.n, W = I.W, G = I.G, max_len = I.max_len;
    const uint64_t cap = budget_cap(p->mem_budget, n);
    const uint32_t max_cost = p->max_cost;
    const size_t tree_bytes = 2ull * (max_cost + 1);
    SolveState *hst = (SolveState *)(c->h_pin + sizeof(SolveJob));
    if (!fused || hst->status == ST_NEED_MEM) {

    // 1-word languages with exact keys: a bitmap of the cached languages in
    // front of the uniqueness table
    const bool use_seen = c->opt_exact && W == 1 && n <= kSeenBits;
    const bool use_direct = c->opt_exact && W == 1 && n <= kDirectBits;

    // launch shape
    const uint32_t seg_cap = 2 * max_cost + 4;
    size_t smem_max = 0;  // dynamic shared memory a k_solve launch can take
    CK(solve_smem_max(&smem_max));
    bool gt_smem = 4ull * (n + 1 + G + max_len + 2) <= 96 * 1024;
    uint32_t warps = 16;  // (the launch bounds of k_solve)
    size_t smem = solve_smem_bytes(W, n, G, max_len, seg_cap, gt_smem, warps);
    while (smem > smem_max && warps > 1) {
        warps /= 2;
        smem = solve_smem_bytes(W, n, G, max_len, seg_cap, gt_smem, warps);
    }
    if (smem > smem_max && gt_smem) {
        gt_smem = false;
        warps = 16;
        smem = solve_smem_bytes(W, n, G, max_len, seg_cap, gt_smem, warps);
        while (smem > smem_max && warps > 1) {
            warps /= 2;
            smem = solve_smem_bytes(W, n, G, max_len, seg_cap, gt_smem, warps);
        }
    }
    if (smem > smem_max) return REI_EINVAL;
    // the search's start in CTA 0's shared memory: as many languages as keep
    // the launch at two CTAs per SM (one, if it already has only one)
    uint32_t small_rows = 0;
    if (c->opt_small_rows != 0 && W <= 8) {
        const size_t half = c->smem_sm / 2 > 4096 ? c->smem_sm / 2 - 4096 : 0;  // static smem + reserve
        const size_t limit = smem <= half ? half : smem_max;
        uint32_t r = c->opt_small_rows > 0 ? (uint32_t)c->opt_small_rows : W <= 2 ? 4096u : W <= 4 ? 2048u : 1024u;
        for (; r >= 256; r >>= 1)
            if (solve_smem_bytes(W, n, G, max_len, seg_cap, gt_smem, warps, r) <= limit) break;
        if (r >= 256) {
            small_rows = r;
            smem = solve_smem_bytes(W, n, G, max_len, seg_cap, gt_smem, warps, r);
        }
    }
    const uint32_t threads = 32 * warps;
    int bps = 0;
    CK(solve_occupancy(threads, smem, &bps));
    if (bps < 1) return REI_ECUDA;
    grid = std::min<uint32_t>((uint32_t)(c->sm_count * bps), kMaxTeam);
    if (c->opt_grid > 0 && (uint32_t)c->opt_grid < grid) grid = (uint32_t)c->opt_grid;

    // a chunk costs a fixed ~15 us of barriers and bookkeeping, so the
    // large levels this launch runs take chunks of up to 32 Mi candidates
    // (at most 1 GiB of candidate rows in tmp; the chunk that holds the
    // answer still runs to its end, which bounds the size from above)
    // (with the seen bitmap, 256 Mi: most candidates end at one bit, so
    // chunks are quicker and their fixed phases and barriers weigh more)
    uint64_t chunk_max = c->opt_chunk > 0 ? (uint64_t)c->opt_chunk
                         : use_seen      ? (1ull << 28)
                                         : std::min<uint64_t>(1ull << 25, std::max<uint64_t>(1ull << 16, (1ull << 30) / (4ull * W)));
    chunk_max = std::min<uint64_t>(chunk_max, use_seen ? (1ull << 28) : (1ull << 26));
    uint64_t cache_alloc = c->opt_cache_init > 0 ? (uint64_t)c->opt_cache_init : (1ull << 16);
    if (c->opt_cache_init <= 0 && c->cs.p && c->bp_l.p && c->bp_r.p && c->bp_op.p) {
        // rows a previous solve already allocated (the table is cleared only
        // where a search filled it, so a large one costs nothing here)
        const uint64_t have = std::min<uint64_t>({(uint64_t)(c->cs.bytes / (4ull * W)), (uint64_t)(c->bp_l.bytes / 4),
                                                  (uint64_t)(c->bp_r.bytes / 4), (uint64_t)c->bp_op.bytes,
                                                  (uint64_t)(c->used.bytes / 4)});
        cache_alloc = std::max<uint64_t>(cache_alloc, have);
    }
    // (no more than 2^n distinct languages exist: rows beyond that are never used)
    const uint64_t cap_rows = n < 63 ? std::min<uint64_t>(cap, 1ull << n) : cap;
    cache_alloc = std::max<uint64_t>(1, std::min<uint64_t>(cache_alloc, cap_rows));

    auto table_slots = [&](uint64_t alloc_rows) {
        uint64_t need = alloc_rows + (alloc_rows >= cap ? chunk_max : 0);
        // (the table holds distinct languages: at most 2^n of them; with
        // 1-word exact keys up to 2^26 it has a slot for every language, the
        // language itself, and is never probed twice)
        if (n < 40) need = std::min<uint64_t>(need, 1ull << n);
        const uint64_t t = pow2_at_least(std::max<uint64_t>(2 * need, 1024));
        return use_direct ? std::max<uint64_t>(t, 1ull << n) : t;
    };
    uint64_t tslots = table_slots(cache_alloc);
    // after a fused launch the cache holds its rows: grow keeping them
    auto ensure_rows = [&](DevBuf &b, size_t bytes) {
        return fused ? grow_keep(c, b, bytes, b.bytes) : ensure(c, b, bytes);
    };
    if ((s = ensure_rows(c->cs, 4ull * W * cache_alloc))) return s;
    if ((s = ensure_rows(c->bp_op, cache_alloc))) return s;
    if ((s = ensure_rows(c->bp_l, 4ull * cache_alloc))) return s;
    if ((s = ensure_rows(c->bp_r, 4ull * cache_alloc))) return s;
    if ((s = ensure(c, c->used, 4ull * cache_alloc))) return s;  // (rebuilt with the table)
    {
        const void *before = c->table.p, *mbefore = c->minidx.p;
        const size_t before_bytes = c->table.bytes, mbefore_bytes = c->minidx.bytes;
        if ((s = ensure(c, c->table, 8ull * tslots))) return s;
        if ((s = ensure(c, c->minidx, 4ull * tslots))) return s;
        if (c->table.p != before || c->table.bytes != before_bytes || c->minidx.p != mbefore ||
            c->minidx.bytes != mbefore_bytes) {
            c->table_clean = false;
            c->table_extent = std::max<uint64_t>(c->table.bytes / 8, c->minidx.bytes / 4);
        }
    }
    // (candidate rows wait in tmp only when the keys are fingerprints)
    const bool exact_keys = W <= 2 && n <= 62 && c->opt_exact;
    if ((s = ensure(c, c->tmp, exact_keys ? 4096 : 4ull * W * chunk_max))) return s;
    if ((s = ensure(c, c->pending, 4ull * chunk_max))) return s;
    if ((s = ensure(c, c->slotpos, 4ull * chunk_max))) return s;
    {
        // a reallocated bitmap holds garbage: the search needs it zero
        const void *before = c->bitmap.p;
        const size_t before_bytes = c->bitmap.bytes;
        if ((s = ensure(c, c->bitmap, 4ull * ((chunk_max + 31) / 32)))) return s;
        if (c->bitmap.p != before || c->bitmap.bytes != before_bytes) {
            if (fused) CK(cudaMemsetAsync(c->bitmap.p, 0, c->bitmap.bytes, c->stream));
            else c->table_clean = false;
        }
    }
    if ((s = ensure(c, c->blk, 4ull * grid))) return s;
    if ((s = ensure(c, c->lvl_start, 8ull * (max_cost + 2)))) return s;
    if ((s = ensure(c, c->lvl_count, 8ull * (max_cost + 2)))) return s;
    {
        const void *before = c->state.p;  // (a new state buffer starts zeroed, as in run_fused)
        if ((s = ensure(c, c->state, sizeof(SolveState) + tree_bytes))) return s;
        if (c->state.p != before) CK(cudaMemsetAsync(c->state.p, 0, c->state.bytes, c->stream));
    }
    if ((s = ensure(c, c->solve_job, sizeof(SolveJob)))) return s;
    if ((s = ensure(c, c->tstack, 16ull * (max_cost + 2)))) return s;
    if ((s = ensure(c, c->trace, 4ull * grid))) return s;
    if ((s = ensure(c, c->plan, 8 * plan_words(seg_cap)))) return s;
    if ((s = ensure_pinned(c, sizeof(SolveJob) + sizeof(SolveState) + tree_bytes))) return s;
    hst = (SolveState *)(c->h_pin + sizeof(SolveJob));  // (the pinned buffer may have moved)

    if (use_seen && !c->seen.p) {
        if ((s = ensure(c, c->seen, (1ull << kSeenBits) / 8))) return s;
        CK(cudaMemsetAsync(c->seen.p, 0, c->seen.bytes, c->stream));
    }
    if (!fused) {
        if (!c->table_clean) {
            // a new table, or the last search ended abnormally: clear it once
            if ((s = clear_table(c, 0))) return s;
            CK(cudaMemsetAsync(c->bitmap.p, 0, c->bitmap.bytes, c->stream));
            if (c->seen.p) CK(cudaMemsetAsync(c->seen.p, 0, c->seen.bytes, c->stream));
        }
        c->table_clean = false;
        c->table_extent = std::max(c->table_extent, tslots);
        uint32_t hj_cmin;
        {
            uint16_t lc[256];
            uint8_t ls[256];
            fill_leaves(p, &hj_cmin, lc, ls);
        }
        CK(cudaMemsetAsync(c->lvl_start.p, 0, 8ull * (max_cost + 2), c->stream));
        CK(cudaMemsetAsync(c->lvl_count.p, 0, 8ull * (max_cost + 2), c->stream));
        memset(hst, 0, sizeof(SolveState));
        hst->status = ST_RUNNING;
        hst->level = hj_cmin;
        hst->found = kNone;
        hst->partial_level = max_cost + 1;
        CK(cudaMemcpyAsync(c->state.p, hst, sizeof(SolveState), cudaMemcpyHostToDevice, c->stream));
        h2d += sizeof(SolveState);
    }

    SolveJob *hj = (SolveJob *)c->h_pin;
    auto fill_job = [&]() {
        memset(hj, 0, sizeof(SolveJob));
        hj->n = n;
        hj->W = W;
        hj->G = G;
        hj->n_sym = p->n_sym;
        hj->max_len = max_len;
        hj->gt_off = (const uint32_t *)c->gt_off.p;
        hj->gt_pair = (const uint32_t *)c->gt_pair.p;
        hj->len_start = (const uint32_t *)c->len_start.p;
        hj->pos_mask = (const uint32_t *)c->pos.p;
        hj->neg_mask = (const uint32_t *)c->neg.p;
        hj->leaf = (const uint32_t *)c->leaf.p;
        hj->leaf_stride = kMaxWords;
        hj->n_pos_set = I.n_pos_set;
        hj->pos_eps = I.pos_eps;
        hj->neg_eps = I.neg_eps;
        fill_leaves(p, &hj->cmin, hj->leaf_cost, hj->leaf_sym);
        hj->c[0] = p->costs.c_sym;
        hj->c[1] = p->costs.c_opt;
        hj->c[2] = p->costs.c_star;
        hj->c[3] = p->costs.c_cat;
        hj->c[4] = p->costs.c_alt;
        hj->max_cost = max_cost;
        hj->max_errors = p->max_errors;
        hj->flags = p->flags;
        hj->cap = cap;
        hj->cs = (uint32_t *)c->cs.p;
        hj->bp_op = (uint8_t *)c->bp_op.p;
        hj->bp_l = (uint32_t *)c->bp_l.p;
        hj->bp_r = (uint32_t *)c->bp_r.p;
        hj->used = (uint32_t *)c->used.p;
        hj->cache_alloc = cache_alloc;
        hj->table = (unsigned long long *)c->table.p;
        hj->minidx = (uint32_t *)c->minidx.p;
        hj->exact = (W <= 2 && n <= 62 && c->opt_exact) ? 1u : 0u;
        hj->seen = use_seen ? (uint32_t *)c->seen.p : nullptr;
        hj->direct = use_direct && tslots >= (1ull << n) ? 1u : 0u;
        hj->table_mask = tslots - 1;
        hj->tmp = (uint32_t *)c->tmp.p;
        hj->pending = (uint32_t *)c->pending.p;
        hj->slotpos = (uint32_t *)c->slotpos.p;
        hj->bitmap = (uint32_t *)c->bitmap.p;
        hj->blk = (uint32_t *)c->blk.p;
        hj->chunk_max = chunk_max;
        hj->lvl_start = (int64_t *)c->lvl_start.p;
        hj->lvl_count = (int64_t *)c->lvl_count.p;
        hj->seg_cap = seg_cap;
        hj->plan = (uint64_t *)c->plan.p;
        hj->st = (SolveState *)c->state.p;
        hj->tree = (uint8_t *)c->state.p + sizeof(SolveState);
        hj->tstack = (uint32_t *)c->tstack.p;
        hj->trace = (uint32_t *)c->trace.p;
        hj->gt_in_smem = gt_smem ? 1 : 0;
        hj->solo_tiles = c->opt_solo_tiles >= 0 ? (uint32_t)c->opt_solo_tiles : 64;
        hj->small_rows = small_rows;
    };
    fill_job();

    for (int relaunch = 0;; relaunch++) {
        // (a fused launch already ran the first part of this search)
        if (!fused || relaunch > 0) {
            CK(cudaEventRecord(c->ev[0], c->stream));
            CK(launch_solve(hj, grid, threads, smem, c->stream));
            CK(cudaEventRecord(c->ev[1], c->stream));
            c->launches++;
            search_launches++;
            CK(cudaMemcpyAsync(hst, c->state.p, sizeof(SolveState) + tree_bytes, cudaMemcpyDeviceToHost,
                               c->stream));
            CK(cudaStreamSynchronize(c->stream));
            {
                float ms = 0;
                CK(cudaEventElapsedTime(&ms, c->ev[0], c->ev[1]));
                ms_search += ms;
            }
            d2h += sizeof(SolveState) + tree_bytes;
        }
        if (hst->status != ST_NEED_MEM) break;
        // grow the cache (keeping its rows) and rebuild the table
        // (a search handed over by a first launch, or continued from a memory
        // slot, may already fit: then only the table is rebuilt at this size)
        const uint64_t want = hst->need_rows > cache_alloc
                                  ? std::min<uint64_t>(cap_rows, std::max<uint64_t>(cache_alloc * 4, hst->need_rows))
                                  : cache_alloc;
        const uint64_t rows = hst->size;
        if ((s = grow_keep(c, c->cs, 4ull * W * want, 4ull * W * rows))) return s;
        if ((s = grow_keep(c, c->bp_op, want, rows))) return s;
        if ((s = grow_keep(c, c->bp_l, 4ull * want, 4ull * rows))) return s;
        if ((s = grow_keep(c, c->bp_r, 4ull * want, 4ull * rows))) return s;
        if ((s = grow_keep(c, c->used, 4ull * want, 0))) return s;
        cache_alloc = want;
        tslots = table_slots(cache_alloc);
        {
            const void *before = c->table.p, *mbefore = c->minidx.p;
            if ((s = ensure(c, c->table, 8ull * tslots))) return s;
            if ((s = ensure(c, c->minidx, 4ull * tslots))) return s;
            if (c->table.p != before || c->minidx.p != mbefore)
                c->table_extent = std::max<uint64_t>(c->table.bytes / 8, c->minidx.bytes / 4);
        }
        if ((s = clear_table(c, tslots))) return s;  // (the rehash refills it)
        c->table_extent = tslots;
        fill_job();
        if (rows) {
            CK(launch_rehash(hj, (uint32_t)rows, (uint32_t)(c->sm_count * 8), c->stream));
            c->launches++;
        }
        hst->status = ST_RUNNING;
        hst->bar_arrive = 0;
        hst->cmd = 0;
        hst->cmd_seq = 0;
        CK(cudaMemcpyAsync(c->state.p, hst, sizeof(SolveState), cudaMemcpyHostToDevice, c->stream));
        CK(cudaStreamSynchronize(c->stream));
        h2d += sizeof(SolveState);
        if (relaunch > 64) return REI_ECUDA;
    }
    }

    if (c->phases) {
        fprintf(stderr, "rei phases: plan %.1f us, solo %.1f us (%llu chunks), team %.1f us (%llu chunks), "
                "level-end %.1f us (%llu levels); search kernel %.1f us\n", hst->t_phase[0] / 1e3,
                hst->t_phase[1] / 1e3, (unsigned long long)hst->n_phase[0], hst->t_phase[2] / 1e3,
                (unsigned long long)hst->n_phase[1], hst->t_phase[3] / 1e3, (unsigned long long)hst->n_phase[2],
                ms_search * 1e3);
        fprintf(stderr, "rei staging steps (timing builds): init %.1f us, checks %.1f us, insert %.1f us, keys %.1f us, "
                "ranks %.1f us, guide table %.1f us, masks %.1f us\n", sg.info.pad[0] / 1e3, sg.info.pad[1] / 1e3,
                sg.info.pad[2] / 1e3, sg.info.pad[3] / 1e3, sg.info.pad[4] / 1e3, sg.info.pad[5] / 1e3,
                sg.info.pad[6] / 1e3);
        fprintf(stderr, "rei chunk steps (timing builds): tiles %.1f us, read %.1f us, append %.1f us; "
                "in append: keys %.1f us, sort %.1f us, copy %.1f us\n", hst->t_sub[0] / 1e3, hst->t_sub[1] / 1e3,
                hst->t_sub[2] / 1e3, hst->t_sub[3] / 1e3, hst->t_sub[4] / 1e3, hst->t_sub[5] / 1e3);
        fprintf(stderr, "rei tile steps of warp 0 (timing builds): load %.1f us, build %.1f us, precision %.1f us, "
                "dedup %.1f us\n", hst->t_sub[6] / 1e3, hst->t_sub[7] / 1e3, hst->t_sub[8] / 1e3, hst->t_sub[9] / 1e3);
        fprintf(stderr, "rei CTA 0 (timing builds): staging to job %.1f us, whole launch %.1f us\n",
                hst->t_sub[10] / 1e3, hst->t_sub[11] / 1e3);
        fprintf(stderr, "rei team chunks on CTA 0 (timing builds): tiles+barrier %.1f us, mark+barrier %.1f us, "
                "count+barrier %.1f us, append+barrier %.1f us; leader appends: keys %.1f sort %.1f copy %.1f us\n",
                hst->t_sub[12] / 1e3, hst->t_sub[13] / 1e3, hst->t_sub[14] / 1e3, hst->t_sub[15] / 1e3,
                hst->t_sub[3] / 1e3, hst->t_sub[4] / 1e3, hst->t_sub[5] / 1e3);
        fprintf(stderr, "rei CTA 0 spans (timing builds): staging run %.1f us, lead init %.1f us, plan_level %.1f us, "
                "tile_setup %.1f us, to global %.1f us, answer %.1f us, cleanup %.1f us\n", hst->t_sub[22] / 1e3,
                hst->t_sub[17] / 1e3, hst->t_sub[18] / 1e3, hst->t_sub[19] / 1e3, hst->t_sub[16] / 1e3,
                hst->t_sub[20] / 1e3, hst->t_sub[21] / 1e3);
        fprintf(stderr, "rei solo chunks (timing builds): tile loop slowest warp %.1f us, tiles %.0f count, "
                "before loop %.1f us\n", hst->t_sub[23] / 1e3, (double)hst->t_sub[24], hst->t_sub[25] / 1e3);
        fprintf(stderr, "rei team phase A (timing builds): publish %.1f us, last CTA starts tiles %.1f us, "
                "slowest tile loop %.1f us, last arrival %.1f us, CTA 0 leaves barrier %.1f us, CTA 0 tile loop %.1f us "
                "(after publish, summed over team chunks)\n", hst->t_sub[40] / 1e3, hst->t_sub[41] / 1e3,
                hst->t_sub[42] / 1e3, hst->t_sub[43] / 1e3, hst->t_sub[39] / 1e3, hst->t_sub[37] / 1e3);
        fprintf(stderr, "rei CTA 0 clock (timing builds): %.0f MHz\n",
                hst->t_sub[11] ? 1e3 * (double)hst->t_sub[38] / (double)hst->t_sub[11] : 0.0);
        for (int k = 0; k < 5; k++)
            fprintf(stderr, "rei solo tiles op%d (timing builds): %.1f us, %.0f count\n", k, hst->t_sub[26 + k] / 1e3,
                    (double)hst->t_sub[32 + k]);
    }
    if (hst->status == ST_TIMEOUT && getenv("REI_DEBUG")) {
        std::vector<uint32_t> tr(grid);
        cudaMemcpyAsync(tr.data(), c->trace.p, 4ull * grid, cudaMemcpyDeviceToHost, c->stream);
        cudaStreamSynchronize(c->stream);
        std::map<uint32_t, uint32_t> hist;
        for (uint32_t v : tr) hist[v]++;
        fprintf(stderr, "rei: barrier wait ran out: cta %u epoch %u site %u seen %u (grid %u); "
                "level %u pos %llu size %u found %llx\n", hst->dbg_cta, hst->dbg_epoch, hst->dbg_site,
                hst->dbg_seen, grid, hst->level, (unsigned long long)hst->chunk_pos, hst->size,
                (unsigned long long)hst->found);
        for (auto &kv : hist) fprintf(stderr, "rei:   %u CTAs last passed epoch %u site %u\n", kv.second, kv.first >> 8, kv.first & 255);
    }
    c->table_clean = hst->status == ST_FOUND || hst->status == ST_NOT_FOUND || hst->status == ST_OOM;
    if (c->table_clean) c->table_extent = 0;  // (the search emptied every slot it filled)
    c->last_valid = true;
    c->last_W = W;
    c->last_size = hst->size;
    c->last_max_cost = max_cost;

    rei_status result;
    switch (hst->status) {
    case ST_FOUND: result = REI_OK; break;
    case ST_NOT_FOUND: result = REI_NOT_FOUND; break;
    case ST_OOM: result = REI_OOM; break;
    case ST_TIMEOUT: result = REI_ETIMEOUT; break;
    default: result = REI_ECUDA; break;
    }
    out->status = result;
    out->stats.candidates = hst->candidates;
    out->stats.unique = result == REI_OK ? hst->unique_done : hst->unique_done;
    out->stats.levels = hst->level;
    rei_status ws = REI_OK;
    if (result == REI_OK) {
        out->cost = hst->ans_cost;
        const uint8_t *tok = (const uint8_t *)(hst + 1);
        ws = write_outputs(out, tok, hst->tree_len, p->alphabet);
    }
    const double t1 = now_ms();
    out->stats.ms_stage = t_stage - t0;
    out->stats.ms_total = t1 - t0;
    if (c->phases) fprintf(stderr, "rei host: solve call %.1f us (after the search %.1f us)\n", (t1 - t0) * 1e3,
                           (t1 - t_stage) * 1e3);
    out->stats.launches = c->launches - l0;
    out->stats.bytes_h2d = h2d;
    out->stats.bytes_d2h = d2h;
    for (int k = 0; k < 5; k++) out->stats.cand_op[k] = hst->cand_op[k];
    out->stats.star_pairs = (uint64_t)G - n;  // sum of |w| over all words: G - n
    out->stats.ms_search_kernel = ms_search;
    out->stats.ms_stage_kernel = sg.ms_kernel;
    out->stats.search_launches = search_launches;
    out->stats.grid = grid;
    if (ws != REI_OK) return ws;
    return result;
}

}  // namespace

// ---------------------------------------------------------------------------
// C ABI

extern "C" {

rei_status rei_ctx_create(rei_ctx **out, int device, const rei_alloc *alloc, void *stream) {
    if (!out) return REI_EINVAL;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) return REI_EINVAL;
    rei_ctx *c = new rei_ctx();
    c->device = device;
    if (cudaSetDevice(device) != cudaSuccess) {
        delete c;
        return REI_ECUDA;
    }
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) {
        delete c;
        return REI_ECUDA;
    }
    c->sm_count = prop.multiProcessorCount;
    c->smem_optin = prop.sharedMemPerBlockOptin;
    c->smem_sm = prop.sharedMemPerMultiprocessor;
    if (alloc && alloc->alloc && alloc->free) {
        c->alloc = *alloc;
        c->has_alloc = true;
    }
    if (cudaEventCreate(&c->ev[0]) != cudaSuccess || cudaEventCreate(&c->ev[1]) != cudaSuccess) {
        delete c;
        return REI_ECUDA;
    }
    if (stream) {
        c->stream = (cudaStream_t)stream;
    } else {
        if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess) {
            delete c;
            return REI_ECUDA;
        }
        c->own_stream = true;
    }
    *out = c;
    return REI_OK;
}

void rei_ctx_destroy(rei_ctx *c) {
    if (!c) return;
    for (rei_ctx *h : c->helpers) rei_ctx_destroy(h);
    c->helpers.clear();
    cudaSetDevice(c->device);
    cudaStreamSynchronize(c->stream);
    DevBuf *bufs[] = {&c->in_bytes, &c->in_offs, &c->stage_job, &c->stage_info, &c->word_start, &c->word_len,
                      &c->len_start, &c->gt_off, &c->gt_pair, &c->pos, &c->neg, &c->leaf, &c->cs,
                      &c->bp_op, &c->bp_l, &c->bp_r, &c->table, &c->minidx, &c->tmp, &c->pending, &c->slotpos,
                      &c->bitmap, &c->blk, &c->lvl_start, &c->lvl_count, &c->state, &c->solve_job,
                      &c->tstack, &c->trace, &c->used, &c->plan, &c->seen, &c->b_in, &c->b_sjobs, &c->b_sinfo, &c->b_stage,
                      &c->b_jobs, &c->b_out, &c->b_tree, &c->b_queue, &c->s_cs, &c->s_bp_op, &c->s_bp_l,
                      &c->s_bp_r, &c->s_used, &c->s_table, &c->s_tmp, &c->s_pend, &c->s_slotpos, &c->s_bitmap,
                      &c->s_blk, &c->s_lvl, &c->s_state, &c->s_tstack, &c->g_idx, &c->g_blk, &c->g_plan,
                      &c->g_tmp, &c->g_pend, &c->g_slotpos, &c->g_bitmap};
    for (DevBuf *b : bufs) dev_free(c, *b);
    cudaStreamSynchronize(c->stream);
    if (c->h_pin) cudaFreeHost(c->h_pin);
    for (cudaEvent_t e : c->ev)
        if (e) cudaEventDestroy(e);
    if (c->own_stream) cudaStreamDestroy(c->stream);
    delete c;
}

rei_status rei_ctx_set_option(rei_ctx *c, int option, int64_t value) {
    if (!c || (value < 0 && option != REI_OPT_SOLO_TILES && option != REI_OPT_SMALL_ROWS)) return REI_EINVAL;
    switch (option) {
    case REI_OPT_CHUNK: c->opt_chunk = value; return REI_OK;
    case REI_OPT_GRID: c->opt_grid = value; return REI_OK;
    case REI_OPT_KEEP_CACHE: c->opt_keep = value; return REI_OK;
    case REI_OPT_CACHE_INIT: c->opt_cache_init = value; return REI_OK;
    case REI_OPT_SOLO_TILES: c->opt_solo_tiles = value; return REI_OK;
    case REI_OPT_FUSED_STAGE: c->opt_fused = value ? 1 : 0; return REI_OK;
    case REI_OPT_EXACT_KEYS: c->opt_exact = value ? 1 : 0; return REI_OK;
    case REI_OPT_HANDOVER: c->opt_handover = (uint64_t)value; return REI_OK;
    case REI_OPT_YIELD_US: c->opt_yield_us = (uint64_t)value; return REI_OK;
    case REI_OPT_SMALL_ROWS:
        if (value > 16384 || (value > 0 && (value < 256 || (value & (value - 1))))) return REI_EINVAL;
        c->opt_small_rows = value < 0 ? -1 : value;
        return REI_OK;
    default: return REI_EINVAL;
    }
}

uint64_t rei_ctx_launches(const rei_ctx *c) { return c ? c->launches : 0; }

rei_status rei_solve_problem(rei_ctx *c, const rei_problem *prob, rei_result *out) {
    if (!c || !prob || !out) return REI_EINVAL;
    std::lock_guard<std::mutex> g(c->mu);
    if (cudaSetDevice(c->device) != cudaSuccess) return REI_ECUDA;
    return solve_one(c, prob, out);
}

rei_status rei_solve(rei_ctx *c, const uint8_t *alphabet, uint32_t n_sym, const rei_str *P, uint32_t nP,
                     const rei_str *N, uint32_t nN, rei_costs costs, uint32_t max_cost, uint64_t mem_budget,
                     rei_result *out) {
    if (!c || !out || (nP && !P) || (nN && !N)) return REI_EINVAL;
    std::vector<uint32_t> offs(1, 0);
    std::vector<uint8_t> bytes;
    for (uint32_t i = 0; i < nP + nN; i++) {
        const rei_str &s = i < nP ? P[i] : N[i - nP];
        if (s.len && !s.ptr) return REI_EINVAL;
        bytes.insert(bytes.end(), s.ptr, s.ptr + s.len);
        offs.push_back((uint32_t)bytes.size());
    }
    rei_problem p{};
    p.alphabet = alphabet;
    p.n_sym = n_sym;
    p.bytes = bytes.data();
    p.offsets = offs.data();
    p.n_pos = nP;
    p.n_neg = nN;
    p.total_bytes = bytes.size();
    p.costs = costs;
    p.max_cost = max_cost;
    p.mem_budget = mem_budget;
    return rei_solve_problem(c, &p, out);
}

rei_status rei_stage(rei_ctx *c, const rei_problem *prob, rei_staged *out) {
    if (!c || !prob || !out) return REI_EINVAL;
    std::lock_guard<std::mutex> g(c->mu);
    if (cudaSetDevice(c->device) != cudaSuccess) return REI_ECUDA;
    rei_status s = check_problem(prob);
    if (s) return s;
    Staged sg;
    s = stage_problem(c, prob, sg);
    if (s) return s;
    const StageInfo &I = sg.info;
    out->n_ic = I.n;
    out->words = I.W;
    out->max_len = I.max_len;
    out->guide_pairs = I.G;
    if (out->cap_words < I.n || out->cap_pairs < I.G || out->cap_w < I.W) return REI_EBUFSZ;
    auto cp = [&](void *dst, const void *src, size_t b) -> cudaError_t {
        if (!dst) return cudaSuccess;
        return cudaMemcpyAsync(dst, src, b, cudaMemcpyDeviceToHost, c->stream);
    };
    CK(cp(out->word_start, c->word_start.p, 4ull * I.n));
    CK(cp(out->word_len, c->word_len.p, 4ull * I.n));
    CK(cp(out->gt_off, c->gt_off.p, 4ull * (I.n + 1)));
    CK(cp(out->gt_pair, c->gt_pair.p, 4ull * I.G));
    CK(cp(out->pos_mask, c->pos.p, 4ull * I.W));
    CK(cp(out->neg_mask, c->neg.p, 4ull * I.W));
    if (out->leaf)
        for (uint32_t a = 0; a < prob->n_sym; a++)
            CK(cudaMemcpyAsync(out->leaf + (size_t)a * out->cap_w, (uint32_t *)c->leaf.p + (size_t)a * kMaxWords,
                               4ull * I.W, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return REI_OK;
}

rei_status rei_cache_dump(rei_ctx *c, uint32_t *cs, uint8_t *op, uint32_t *left, uint32_t *right,
                          uint64_t *count, uint64_t *level_start, uint64_t *level_count, uint32_t n_levels) {
    if (!c || !count) return REI_EINVAL;
    std::lock_guard<std::mutex> g(c->mu);
    if (!c->last_valid) return REI_EINVAL;
    const uint64_t k = c->last_size;
    const uint64_t capn = *count;
    *count = k;
    if (capn < k) return REI_EBUFSZ;
    const uint32_t W = c->last_W;
    if (cs) CK(cudaMemcpyAsync(cs, c->cs.p, 4ull * W * k, cudaMemcpyDeviceToHost, c->stream));
    if (op) CK(cudaMemcpyAsync(op, c->bp_op.p, k, cudaMemcpyDeviceToHost, c->stream));
    if (left) CK(cudaMemcpyAsync(left, c->bp_l.p, 4ull * k, cudaMemcpyDeviceToHost, c->stream));
    if (right) CK(cudaMemcpyAsync(right, c->bp_r.p, 4ull * k, cudaMemcpyDeviceToHost, c->stream));
    const uint32_t nl = std::min<uint32_t>(n_levels, c->last_max_cost + 1);
    if (level_start) CK(cudaMemcpyAsync(level_start, c->lvl_start.p, 8ull * nl, cudaMemcpyDeviceToHost, c->stream));
    if (level_count) CK(cudaMemcpyAsync(level_count, c->lvl_count.p, 8ull * nl, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return REI_OK;
}

// ---- batched form: one staging launch and one persistent search launch ----

}  // extern "C"

namespace {

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

struct BatchPlan {
    std::vector<uint32_t> idx;          // outs index of every problem in the launch
    std::vector<size_t> off_in, off_offs, off_stage;
    std::vector<uint32_t> n_bound, g_bound, l_bound;
    size_t in_bytes = 0, stage_bytes = 0;
};

// Run problems `sel` of `probs` in one batched launch with `warps` warps per
// CTA, dedup chunks of `chunk` candidates in each slot and a time allowance of
// `yield_us` per problem (~0 = none).  Searches that pass the allowance or
// outgrow their slot continue on the whole GPU afterwards.
rei_status run_batch(rei_ctx *c, const rei_problem *probs, const std::vector<uint32_t> &sel, rei_result *outs,
                     uint32_t warps, uint32_t chunk_sz, uint32_t yield_us, double *kernel_ms) {
    const uint32_t nb = (uint32_t)sel.size();
    if (kernel_ms) *kernel_ms = 0;
    if (nb == 0) return REI_OK;
    const double tb0 = now_ms();
    double tb_up = 0, tb_launch = 0;
    BatchPlan P;
    // host-side bounds of every problem's staged sizes (exact upper bounds)
    for (uint32_t t = 0; t < nb; t++) {
        const rei_problem &p = probs[sel[t]];
        const uint32_t n_str = p.n_pos + p.n_neg;
        uint64_t occ = 1, pairs = 1;
        uint32_t maxl = 0;
        for (uint32_t k = 0; k < n_str; k++) {
            const uint64_t L = p.offsets[k + 1] - p.offsets[k];
            occ += L * (L + 1) / 2;
            for (uint64_t len = 1; len <= L; len++) pairs += (L - len + 1) * (len + 1);
            maxl = std::max<uint32_t>(maxl, (uint32_t)L);
        }
        const uint32_t nbd = (uint32_t)std::min<uint64_t>(occ, kMaxIC);
        P.n_bound.push_back(nbd);
        P.g_bound.push_back((uint32_t)std::min<uint64_t>(pairs, (uint64_t)nbd * (maxl + 1)));
        P.l_bound.push_back(maxl);
        P.off_offs.push_back(P.in_bytes);
        P.in_bytes = align256(P.in_bytes + 4ull * (n_str + 1));
        P.off_in.push_back(P.in_bytes);
        P.in_bytes = align256(P.in_bytes + (n_str ? p.offsets[n_str] : 0) + 1);
        P.off_stage.push_back(P.stage_bytes);
        P.stage_bytes += align256(8ull * nbd) + align256(4ull * (maxl + 2)) + align256(4ull * (nbd + 1)) +
                         align256(4ull * P.g_bound.back()) + 2 * align256(4ull * kMaxWords) +
                         align256(4ull * kMaxWords * p.n_sym);
    }
    rei_status s;
    const size_t tree_bytes = 2ull * (REI_MAX_COST + 1);
    if ((s = ensure(c, c->b_in, P.in_bytes))) return s;
    if ((s = ensure(c, c->b_stage, P.stage_bytes))) return s;
    if ((s = ensure(c, c->b_sjobs, sizeof(StageJob) * nb))) return s;
    if ((s = ensure(c, c->b_sinfo, sizeof(StageInfo) * nb))) return s;
    if ((s = ensure(c, c->b_jobs, sizeof(BatchJob) * nb))) return s;
    if ((s = ensure(c, c->b_out, sizeof(BatchOut) * nb))) return s;
    if ((s = ensure(c, c->b_tree, tree_bytes * nb))) return s;
    if ((s = ensure(c, c->b_queue, 16))) return s;
    const size_t host_bytes = std::max(P.in_bytes, std::max(sizeof(StageJob), sizeof(BatchJob)) * nb) +
                              (sizeof(StageInfo) + sizeof(BatchOut) + tree_bytes + 8) * nb + 4096;
    if ((s = ensure_pinned(c, host_bytes))) return s;
    CK(cudaStreamSynchronize(c->stream));
    uint8_t *hp = c->h_pin;
    // inputs: one upload
    for (uint32_t t = 0; t < nb; t++) {
        const rei_problem &p = probs[sel[t]];
        const uint32_t n_str = p.n_pos + p.n_neg;
        if (n_str) memcpy(hp + P.off_offs[t], p.offsets, 4ull * (n_str + 1));
        else memset(hp + P.off_offs[t], 0, 4);
        if (n_str && p.offsets[n_str]) memcpy(hp + P.off_in[t], p.bytes, p.offsets[n_str]);
    }
    CK(cudaMemcpyAsync(c->b_in.p, hp, P.in_bytes, cudaMemcpyHostToDevice, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    // staging jobs
    StageJob *sj = (StageJob *)hp;
    uint8_t *din = (uint8_t *)c->b_in.p, *dst = (uint8_t *)c->b_stage.p;
    std::vector<uint32_t *> ws(nb), wl(nb), ls(nb), go(nb), gp(nb), pm(nb), nm(nb), lf(nb);
    for (uint32_t t = 0; t < nb; t++) {
        const rei_problem &p = probs[sel[t]];
        StageJob &j = sj[t];
        memset(&j, 0, sizeof j);
        j.bytes = din + P.off_in[t];
        j.offs = (const uint32_t *)(din + P.off_offs[t]);
        j.n_pos = p.n_pos;
        j.n_neg = p.n_neg;
        memcpy(j.alphabet, p.alphabet, p.n_sym);
        j.n_sym = p.n_sym;
        j.total_bytes = (p.n_pos + p.n_neg) ? p.offsets[p.n_pos + p.n_neg] : 0;
        j.info = (StageInfo *)c->b_sinfo.p + t;
        uint8_t *q = dst + P.off_stage[t];
        ws[t] = (uint32_t *)q;
        wl[t] = ws[t] + P.n_bound[t];
        q += align256(8ull * P.n_bound[t]);
        ls[t] = (uint32_t *)q;
        q += align256(4ull * (P.l_bound[t] + 2));
        go[t] = (uint32_t *)q;
        q += align256(4ull * (P.n_bound[t] + 1));
        gp[t] = (uint32_t *)q;
        q += align256(4ull * P.g_bound[t]);
        pm[t] = (uint32_t *)q;
        q += align256(4ull * kMaxWords);
        nm[t] = (uint32_t *)q;
        q += align256(4ull * kMaxWords);
        lf[t] = (uint32_t *)q;
        j.word_start = ws[t];
        j.word_len = wl[t];
        j.len_start = ls[t];
        j.gt_off = go[t];
        j.gt_pair = gp[t];
        j.pair_cap = P.g_bound[t];
        j.pos_mask = pm[t];
        j.neg_mask = nm[t];
        j.leaf = lf[t];
    }
    CK(cudaMemcpyAsync(c->b_sjobs.p, sj, sizeof(StageJob) * nb, cudaMemcpyHostToDevice, c->stream));
    CK(cudaMemsetAsync(c->b_sinfo.p, 0, sizeof(StageInfo) * nb, c->stream));
    tb_up = now_ms();
    CK(launch_stage((const StageJob *)c->b_sjobs.p, nb, c->stream));
    c->launches++;
    StageInfo *si = (StageInfo *)(hp + std::max(sizeof(StageJob), sizeof(BatchJob)) * nb);
    CK(cudaMemcpyAsync(si, c->b_sinfo.p, sizeof(StageInfo) * nb, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));

    // search jobs; the launch's shared memory fits the largest problem
    std::vector<uint32_t> live;
    uint32_t wmax = 1;
    size_t smem = 0;
    BatchJob *bj = (BatchJob *)hp;  // reuses the staging-job area (already uploaded)
    // the CTAs take problems in queue order: the widest first, so that the
    // longest searches start early and the short ones fill in around them
    std::vector<uint32_t> order(nb);
    for (uint32_t t = 0; t < nb; t++) order[t] = t;
    std::stable_sort(order.begin(), order.end(), [&](uint32_t x, uint32_t y) {
        if (si[x].W != si[y].W) return si[x].W > si[y].W;
        return si[x].n > si[y].n;
    });
    for (uint32_t t : order) {
        const rei_problem &p = probs[sel[t]];
        const StageInfo &I = si[t];
        rei_result &o = outs[sel[t]];
        o.stats.n_ic = I.n;
        o.stats.words = I.W;
        o.stats.max_len = I.max_len;
        o.stats.guide_pairs = I.G;
        if (I.status != SE_OK) {
            o.status = REI_EINVAL;
            continue;
        }
        BatchJob &b = bj[live.size()];
        memset(&b, 0, sizeof b);
        SolveJob &J = b.job;
        J.n = I.n;
        J.W = I.W;
        J.G = I.G;
        J.n_sym = p.n_sym;
        J.max_len = I.max_len;
        J.gt_off = go[t];
        J.gt_pair = gp[t];
        J.len_start = ls[t];
        J.pos_mask = pm[t];
        J.neg_mask = nm[t];
        J.leaf = lf[t];
        J.leaf_stride = kMaxWords;
        J.n_pos_set = I.n_pos_set;
        J.pos_eps = I.pos_eps;
        J.neg_eps = I.neg_eps;
        fill_leaves(&p, &J.cmin, J.leaf_cost, J.leaf_sym);
        J.c[0] = p.costs.c_sym;
        J.c[1] = p.costs.c_opt;
        J.c[2] = p.costs.c_star;
        J.c[3] = p.costs.c_cat;
        J.c[4] = p.costs.c_alt;
        J.max_cost = p.max_cost;
        J.max_errors = p.max_errors;
        J.flags = p.flags & ~REI_F_DEVICE_INPUT;
        J.cap = budget_cap(p.mem_budget, I.n);
        J.seg_cap = 2 * p.max_cost + 4;
        J.gt_in_smem = 4ull * (I.n + 1 + I.G + I.max_len + 2) <= 48 * 1024;
        b.tree = (uint8_t *)c->b_tree.p + tree_bytes * live.size();
        b.out = (BatchOut *)c->b_out.p + live.size();
        smem = std::max(smem, solve_smem_bytes(I.W, I.n, I.G, I.max_len, J.seg_cap, J.gt_in_smem, warps));
        wmax = std::max(wmax, I.W);
        live.push_back(t);
    }
    const uint32_t nl = (uint32_t)live.size();
    if (nl == 0) return REI_OK;
    size_t smem_max = 0;
    CK(solve_batch_smem_max(&smem_max));
    if (smem > smem_max) return REI_EINVAL;
    int bps = 0;
    CK(solve_batch_occupancy(32 * warps, smem, &bps));
    if (bps < 1) return REI_ECUDA;
    const uint32_t slots = std::min<uint32_t>(nl, (uint32_t)(c->sm_count * bps));

    // per-slot memory (grow-only; tables and bitmaps kept empty between uses)
    const uint64_t rows = 1ull << 18, chunk = chunk_sz;
    const uint64_t cs_words = rows * wmax, tmp_words = chunk * wmax;
    const uint64_t tslots = pow2_at_least(2 * (rows + chunk));
    bool fresh = !c->slots_clean || c->slot_count < slots || c->slot_rows != rows || c->slot_cs_words < cs_words ||
                 c->slot_table != tslots || c->slot_tmp_words < tmp_words || c->slot_chunk != chunk;
    if (fresh) {
        const uint64_t sl = std::max<uint32_t>(slots, c->slot_count);
        const uint64_t csw = std::max(cs_words, c->slot_cs_words), tw = std::max(tmp_words, c->slot_tmp_words);
        if ((s = ensure(c, c->s_cs, 4 * sl * csw))) return s;
        if ((s = ensure(c, c->s_bp_op, sl * rows))) return s;
        if ((s = ensure(c, c->s_bp_l, 4 * sl * rows))) return s;
        if ((s = ensure(c, c->s_bp_r, 4 * sl * rows))) return s;
        if ((s = ensure(c, c->s_used, 4 * sl * rows))) return s;
        if ((s = ensure(c, c->s_table, 8 * sl * tslots))) return s;
        if ((s = ensure(c, c->s_tmp, 4 * sl * tw))) return s;
        if ((s = ensure(c, c->s_pend, 4 * sl * chunk))) return s;
        if ((s = ensure(c, c->s_slotpos, 4 * sl * chunk))) return s;
        if ((s = ensure(c, c->s_bitmap, 4 * sl * ((chunk + 31) / 32)))) return s;
        if ((s = ensure(c, c->s_blk, 4 * sl))) return s;
        if ((s = ensure(c, c->s_lvl, 8 * sl * 2 * (kMaxCost + 2)))) return s;
        if ((s = ensure(c, c->s_state, sizeof(SolveState) * sl))) return s;
        if ((s = ensure(c, c->s_tstack, 16 * sl * (kMaxCost + 2)))) return s;
        CK(cudaMemsetAsync(c->s_table.p, 0xFF, 8 * sl * tslots, c->stream));
        CK(cudaMemsetAsync(c->s_bitmap.p, 0, 4 * sl * ((chunk + 31) / 32), c->stream));
        c->slot_count = (uint32_t)sl;
        c->slot_rows = rows;
        c->slot_cs_words = csw;
        c->slot_table = tslots;
        c->slot_tmp_words = tw;
        c->slot_chunk = chunk;
    }
    BatchArgs A{};
    A.slot.cs = (uint32_t *)c->s_cs.p;
    A.slot.bp_op = (uint8_t *)c->s_bp_op.p;
    A.slot.bp_l = (uint32_t *)c->s_bp_l.p;
    A.slot.bp_r = (uint32_t *)c->s_bp_r.p;
    A.slot.used = (uint32_t *)c->s_used.p;
    A.slot.table = (unsigned long long *)c->s_table.p;
    A.slot.tmp = (uint32_t *)c->s_tmp.p;
    A.slot.pending = (uint32_t *)c->s_pend.p;
    A.slot.slotpos = (uint32_t *)c->s_slotpos.p;
    A.slot.bitmap = (uint32_t *)c->s_bitmap.p;
    A.slot.blk = (uint32_t *)c->s_blk.p;
    A.slot.lvl = (int64_t *)c->s_lvl.p;
    A.slot.state = (SolveState *)c->s_state.p;
    A.slot.tstack = (uint32_t *)c->s_tstack.p;
    A.slot.rows = rows;
    A.slot.cs_words = c->slot_cs_words;
    A.slot.table_slots = tslots;
    A.slot.tmp_words = c->slot_tmp_words;
    A.slot.chunk = chunk;
    A.n = nl;
    A.queue = (uint32_t *)c->b_queue.p;
    A.yield_ns = yield_us == 0xFFFFFFFFu ? 0 : (uint64_t)yield_us * 1000ull;
    CK(cudaMemcpyAsync(c->b_jobs.p, bj, sizeof(BatchJob) * nl, cudaMemcpyHostToDevice, c->stream));
    CK(cudaMemsetAsync(c->b_queue.p, 0, 16, c->stream));
    // (a problem no CTA took keeps status 0, ST_RUNNING)
    CK(cudaMemsetAsync(c->b_out.p, 0, sizeof(BatchOut) * nl, c->stream));
    c->slots_clean = false;
    CK(cudaEventRecord(c->ev[0], c->stream));
    tb_launch = now_ms();
    CK(launch_solve_batch((const BatchJob *)c->b_jobs.p, &A, slots, 32 * warps, smem, c->stream));
    CK(cudaEventRecord(c->ev[1], c->stream));
    c->launches++;
    BatchOut *bo = (BatchOut *)(hp + std::max(sizeof(StageJob), sizeof(BatchJob)) * nb + sizeof(StageInfo) * nb);
    uint8_t *tr = (uint8_t *)(bo + nb);
    CK(cudaMemcpyAsync(bo, c->b_out.p, sizeof(BatchOut) * nl, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaMemcpyAsync(tr, c->b_tree.p, tree_bytes * nl, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    c->slots_clean = true;
    float ms = 0;
    CK(cudaEventElapsedTime(&ms, c->ev[0], c->ev[1]));
    if (kernel_ms) *kernel_ms = ms;
    if (c->phases)
        fprintf(stderr, "rei batch of %u: upload %.3f ms, staging+jobs %.3f ms, search launch to answers %.3f ms "
                "(kernel %.3f ms), total %.3f ms\n", nb, tb_up - tb0, tb_launch - tb_up, now_ms() - tb_launch, ms,
                now_ms() - tb0);

    // parked searches (continued from their slots, before a launch reuses the
    // slots) and problems no CTA took (a CTA that parks a search takes no
    // more problems): launched again
    struct Parked {
        uint32_t prob, slot;
        double ms;           // time the search spent on its CTA (and in its slot group)
        uint32_t k;          // its entry among the launch's problems
        uint32_t need_rows;  // 0: parked at its time allowance
    };
    std::vector<Parked> redo;
    std::vector<uint32_t> again;
    // a finished search's report into its result
    auto finish = [&](uint32_t k, const BatchOut &b, double ms) {
        const uint32_t t = live[k];
        const rei_problem &p = probs[sel[t]];
        rei_result &o = outs[sel[t]];
        o.stats.candidates = b.candidates;
        o.stats.unique = b.unique;
        o.stats.levels = b.levels;
        for (int q = 0; q < 5; q++) o.stats.cand_op[q] = b.cand_op[q];
        o.stats.star_pairs = o.stats.guide_pairs - o.stats.n_ic;
        o.stats.ms_search_kernel = ms;
        o.stats.ms_total = ms;
        o.stats.launches += 2;
        o.stats.search_launches += 1;
        o.stats.grid = slots;
        switch (b.status) {
        case ST_FOUND: o.status = REI_OK; break;
        case ST_NOT_FOUND: o.status = REI_NOT_FOUND; break;
        case ST_OOM: o.status = REI_OOM; break;
        default: o.status = REI_ECUDA; break;
        }
        o.regex_len = o.tree_len = 0;
        if (o.status == REI_OK) {
            o.cost = b.cost;
            if (write_outputs(&o, tr + tree_bytes * k, b.tree_len, p.alphabet) != REI_OK) o.status = REI_EBUFSZ;
        }
    };
    for (uint32_t k = 0; k < nl; k++) {
        const uint32_t t = live[k];
        const BatchOut &b = bo[k];
        if (b.status == ST_RUNNING) {
            again.push_back(sel[t]);
            continue;
        }
        if (b.status == ST_NEED_MEM) {
            redo.push_back({sel[t], b.slot, b.ns / 1e6, k, b.need_rows});
            continue;
        }
        finish(k, b, b.ns / 1e6);
    }

    // searches parked at their time allowance (their slot holds their cache
    // and table): continued side by side in one launch, a group of CTAs per
    // search in its slot
    std::vector<Parked> rest;
    {
        std::vector<Parked> grp;
        for (const Parked &pk : redo) (pk.slot < slots && pk.need_rows == 0 ? grp : rest).push_back(pk);
        const uint32_t threads_g = 256;
        size_t smem_g = 0, smem_gmax = 0;
        uint32_t seg_cap_g = 0, wmax_g = 1;
        for (const Parked &pk : grp) {
            const SolveJob &J = bj[pk.k].job;
            smem_g = std::max(smem_g, solve_smem_bytes(J.W, J.n, J.G, J.max_len, J.seg_cap, J.gt_in_smem, threads_g / 32));
            seg_cap_g = std::max(seg_cap_g, J.seg_cap);
            wmax_g = std::max(wmax_g, J.W);
        }
        int bps_g = 0;
        if (!grp.empty()) {
            CK(solve_groups_smem_max(&smem_gmax));
            if (smem_g <= smem_gmax) CK(solve_groups_occupancy(threads_g, smem_g, &bps_g));
        }
        const uint32_t cap = (uint32_t)std::max(0, bps_g) * (uint32_t)c->sm_count;
        const uint32_t ng = (uint32_t)std::min<size_t>(grp.size(), cap / 2);
        for (uint32_t q = ng; q < grp.size(); q++) rest.push_back(grp[q]);
        if (ng > 0) {
            const uint32_t gctas = std::min<uint32_t>(cap / ng, kMaxTeam);
            const uint64_t pstride = plan_words(seg_cap_g);
            if ((s = ensure(c, c->g_idx, 8ull * ng))) return s;
            if ((s = ensure(c, c->g_blk, 4ull * ng * gctas))) return s;
            if ((s = ensure(c, c->g_plan, 8ull * ng * pstride))) return s;
            // chunks of up to 2^18 candidates (the slot tables' room), rows of
            // the widest group's languages; about 1 GiB of rows at most
            uint64_t chunk_g = 1ull << 18;
            while (chunk_g > 4096 && chunk_g * wmax_g * ng > (1ull << 28)) chunk_g >>= 1;
            const uint64_t tmp_g = chunk_g * wmax_g, bmw_g = (chunk_g + 31) / 32;
            if ((s = ensure(c, c->g_tmp, 4ull * ng * tmp_g))) return s;
            if ((s = ensure(c, c->g_pend, 4ull * ng * chunk_g))) return s;
            if ((s = ensure(c, c->g_slotpos, 4ull * ng * chunk_g))) return s;
            if ((s = ensure(c, c->g_bitmap, 4ull * ng * bmw_g))) return s;
            CK(cudaMemsetAsync(c->g_bitmap.p, 0, 4ull * ng * bmw_g, c->stream));
            uint32_t *gidx = (uint32_t *)(((uintptr_t)(tr + tree_bytes * nb) + 7) & ~(uintptr_t)7);
            for (uint32_t g = 0; g < ng; g++) {
                gidx[g] = grp[g].k;
                gidx[ng + g] = grp[g].slot;
            }
            CK(cudaMemcpyAsync(c->g_idx.p, gidx, 8ull * ng, cudaMemcpyHostToDevice, c->stream));
            GroupArgs G{};
            G.slot = A.slot;
            G.prob = (const uint32_t *)c->g_idx.p;
            G.slot_of = (const uint32_t *)c->g_idx.p + ng;
            G.groups = ng;
            G.group_ctas = gctas;
            G.blk = (uint32_t *)c->g_blk.p;
            G.plan = (uint64_t *)c->g_plan.p;
            G.plan_stride = pstride;
            G.tmp = (uint32_t *)c->g_tmp.p;
            G.pending = (uint32_t *)c->g_pend.p;
            G.slotpos = (uint32_t *)c->g_slotpos.p;
            G.bitmap = (uint32_t *)c->g_bitmap.p;
            G.chunk = chunk_g;
            G.tmp_words = tmp_g;
            c->slots_clean = false;
            CK(launch_solve_groups((const BatchJob *)c->b_jobs.p, &G, ng * gctas, threads_g, smem_g, c->stream));
            c->launches++;
            CK(cudaMemcpyAsync(bo, c->b_out.p, sizeof(BatchOut) * nl, cudaMemcpyDeviceToHost, c->stream));
            CK(cudaMemcpyAsync(tr, c->b_tree.p, tree_bytes * nl, cudaMemcpyDeviceToHost, c->stream));
            CK(cudaStreamSynchronize(c->stream));
            if (c->phases)
                fprintf(stderr, "rei batch: %u parked searches continued in their slots, %u CTAs each\n", ng, gctas);
            for (uint32_t g = 0; g < ng; g++) {
                Parked pk = grp[g];
                const BatchOut &b = bo[pk.k];
                pk.ms += b.ns / 1e6;
                if (b.status == ST_FOUND || b.status == ST_NOT_FOUND || b.status == ST_OOM) {
                    finish(pk.k, b, pk.ms);
                    outs[pk.prob].stats.launches += 1;
                    outs[pk.prob].stats.search_launches += 1;
                } else {
                    // (outgrew its slot again, or failed: continued on the whole GPU)
                    pk.need_rows = b.status == ST_NEED_MEM ? b.need_rows : 1u;
                    rest.push_back(pk);
                }
            }
        }
    }
    // the rest continue on the whole GPU from their slots' rows (the table is
    // rebuilt there, so the slots' tables and chunk bitmaps are emptied for
    // later problems); then every slot is empty again
    const uint64_t bm_words = (chunk + 31) / 32;
    for (const Parked &pk : rest)
        if (pk.slot < slots) {
            CK(cudaMemsetAsync((unsigned long long *)c->s_table.p + (uint64_t)pk.slot * tslots, 0xFF, 8 * tslots,
                               c->stream));
            CK(cudaMemsetAsync((uint32_t *)c->s_bitmap.p + (uint64_t)pk.slot * bm_words, 0, 4 * bm_words, c->stream));
        }
    c->slots_clean = true;

    // each such search continues from its slot: one after another on this
    // context's whole GPU when there is one, else side by side on helper
    // contexts (own streams and buffers), each launch on an equal share of
    // the SMs (the searches are latency-bound; together they fill the GPU)
    auto continue_one = [&](rei_ctx *h, const Parked &pk) {
        const uint32_t i = pk.prob;
        const SlotResume rs{&A.slot, pk.slot};
        const rei_status r = solve_one(h, &probs[i], &outs[i], pk.slot < slots ? &rs : nullptr);
        if (r != REI_OK && r != REI_NOT_FOUND && r != REI_OOM) outs[i].status = r;
        // the problem's time: on its CTA (and group), then on its share of the GPU
        outs[i].stats.ms_total += pk.ms;
        outs[i].stats.ms_search_kernel += pk.ms;
    };
    redo = rest;
    const uint32_t nh = (uint32_t)std::min<size_t>(redo.size(), kBatchHelpers);
    if (nh <= 1) {
        for (const Parked &pk : redo) continue_one(c, pk);
    } else {
        while (c->helpers.size() < nh) {
            rei_ctx *h = nullptr;
            if (rei_ctx_create(&h, c->device, nullptr, nullptr) != REI_OK) break;
            c->helpers.push_back(h);
        }
        const uint32_t nuse = (uint32_t)std::min<size_t>(nh, c->helpers.size());
        std::atomic<size_t> next{0};
        std::vector<uint64_t> l0(nuse);
        std::vector<std::thread> th;
        for (uint32_t k = 0; k < nuse; k++) {
            rei_ctx *h = c->helpers[k];
            h->opt_chunk = c->opt_chunk;
            h->opt_cache_init = c->opt_cache_init;
            h->opt_solo_tiles = c->opt_solo_tiles;
            h->opt_small_rows = c->opt_small_rows;
            h->opt_fused = c->opt_fused;
            h->opt_exact = c->opt_exact;
            h->opt_handover = c->opt_handover;
            const int64_t share = std::max<int64_t>(1, (int64_t)c->sm_count * 2 / nuse);  // (k_solve: 2 CTAs per SM)
            h->opt_grid = c->opt_grid > 0 ? std::min<int64_t>(c->opt_grid, share) : share;
            l0[k] = h->launches;
            th.emplace_back([&, h] {
                cudaSetDevice(h->device);
                for (size_t q; (q = next.fetch_add(1)) < redo.size();) continue_one(h, redo[q]);
            });
        }
        if (nuse == 0)
            for (const Parked &pk : redo) continue_one(c, pk);
        for (std::thread &t : th) t.join();
        for (uint32_t k = 0; k < nuse; k++) c->launches += c->helpers[k]->launches - l0[k];
    }
    if (!again.empty()) return run_batch(c, probs, again, outs, warps, chunk_sz, yield_us, nullptr);
    return REI_OK;
}

}  // namespace

extern "C" {

rei_status rei_solve_batch(rei_ctx *c, const rei_problem *probs, uint32_t n, rei_result *outs,
                           const rei_tune *tune) {
    if (!c || (n && (!probs || !outs))) return REI_EINVAL;
    if (tune && ((tune->warps_per_cta && (tune->warps_per_cta > 8 || (tune->warps_per_cta & (tune->warps_per_cta - 1)))) ||
                 (tune->chunk && (tune->chunk < 256 || tune->chunk > 65536))))
        return REI_EINVAL;
    std::lock_guard<std::mutex> g(c->mu);
    if (cudaSetDevice(c->device) != cudaSuccess) return REI_ECUDA;
    std::vector<uint32_t> sel;
    for (uint32_t i = 0; i < n; i++) {
        memset(&outs[i].stats, 0, sizeof(outs[i].stats));
        outs[i].status = REI_EINVAL;
        outs[i].cost = 0;
        outs[i].regex_len = outs[i].tree_len = 0;
        if (check_problem(&probs[i]) != REI_OK) continue;
        if (probs[i].flags & REI_F_DEVICE_INPUT) {
            // device-resident inputs: solved alone (the batch packs host inputs)
            const rei_status r = solve_one(c, &probs[i], &outs[i]);
            if (r != REI_OK && r != REI_NOT_FOUND && r != REI_OOM) outs[i].status = r;
            continue;
        }
        sel.push_back(i);
    }
    // the launch shape: given, else autotuned once per context on samples of
    // the batch (each one problem per SM; every sample is solved exactly, so
    // tuning costs no work), else the default (8 warps, chunks of 2^14)
    uint32_t warps = tune && tune->warps_per_cta ? tune->warps_per_cta : (uint32_t)c->batch_warps;
    uint32_t chunk = tune && tune->chunk ? tune->chunk : c->batch_chunk;
    const uint32_t yield_us = tune && tune->yield_us ? tune->yield_us
                              : c->opt_yield_us ? (uint32_t)std::min<uint64_t>(c->opt_yield_us, 0xFFFFFFFEu) : 0xFFFFFFFFu;
    size_t done = 0;
    if (warps == 0 || chunk == 0) {
        struct Trial {
            uint32_t warps, chunk;
        };
        std::vector<Trial> trials;
        for (uint32_t w : {8u, 4u})
            for (uint32_t ch : {1u << 14, 1u << 12, 1u << 16})
                if ((!warps || w == warps) && (!chunk || ch == chunk)) trials.push_back({w, ch});
        Trial best{warps ? warps : 8u, chunk ? chunk : (1u << 14)};
        const size_t sample = (size_t)std::max(1, c->sm_count);
        double best_rate = -1;
        // (at least two samples of the batch stay untimed)
        for (const Trial &tr : trials) {
            if (sel.size() - done < 3 * sample) break;
            std::vector<uint32_t> part(sel.begin() + done, sel.begin() + done + sample);
            const double ts = now_ms();
            const rei_status r = run_batch(c, probs, part, outs, tr.warps, tr.chunk, yield_us, nullptr);
            if (r != REI_OK) return r;
            const double ms = now_ms() - ts;
            uint64_t cands = 0;
            for (uint32_t i : part) cands += outs[i].stats.candidates;
            const double rate = ms > 0 ? cands / ms : 0;
            if (rate > best_rate) {
                best_rate = rate;
                best = tr;
            }
            done += sample;
        }
        warps = best.warps;
        chunk = best.chunk;
        if (best_rate >= 0) {
            if (!tune || !tune->warps_per_cta) c->batch_warps = (int)warps;
            if (!tune || !tune->chunk) c->batch_chunk = chunk;
        }
    }
    std::vector<uint32_t> rest(sel.begin() + done, sel.end());
    return run_batch(c, probs, rest, outs, warps, chunk, yield_us, nullptr);
}

}  // extern "C"

// ---------------------------------------------------------------------------
// served form: continuous batching.  A worker thread admits queued requests
// (while the live ones' cache footprints fit the budget and fewer than
// max_live are live) into a ring of mapped host memory and publishes them; a
// persistent k_serve launch whose CTAs take them as they free up stages and
// solves each one and writes its answer back.  Requests larger than a CTA
// slot are solved alone (rei_solve_problem) while the launch is stopped.

struct rei_server {
    rei_ctx *ctx;
    uint64_t budget;
    uint32_t max_live;
    std::mutex mu;
    std::condition_variable cv, done_cv;
    struct Req {
        uint64_t ticket;
        std::vector<uint8_t> alphabet, bytes;
        std::vector<uint32_t> offs, sym_costs;
        rei_problem p;
        uint64_t footprint;
        double t_submit;  // host clock, ms
        uint32_t slot = kNoSlot;  // a search the launch left in this memory slot
        uint32_t need_rows = 0;   // the rows it asked for (0: it stopped at its time allowance)
        uint64_t job = 0;         // its ring job (its report is in outs[job % ring_size])
        double ms_slot = 0;       // time its search spent in the slot
    };
    struct Done {
        rei_result r;
        std::string regex;
        std::vector<uint8_t> tree;
    };
    std::deque<Req> queue;
    std::map<uint64_t, Done> done;
    std::set<uint64_t> open;  // issued, not yet released
    uint64_t next_ticket = 1;
    bool stop = false;
    std::thread worker;
    rei_status error = REI_OK;

    // device side
    uint32_t ring_size = 0, grid = 0, threads = 256;
    size_t smem = 0;
    ServeReq *ring_h = nullptr;
    ServeOut *outs_h = nullptr;
    unsigned long long *ctl_h = nullptr;  // [0] avail, [1] stop
    ServeArgs args{};
    std::vector<DevBuf> bufs;
    cudaStream_t kstream = nullptr;
    cudaEvent_t kdone = nullptr;
    bool running = false;
    uint64_t published = 0;
    std::map<uint64_t, Req> live;  // by job id
    uint64_t live_bytes = 0;
};

namespace {

void server_fail(rei_server *S, rei_status e) {
    std::lock_guard<std::mutex> lk(S->mu);
    if (S->error == REI_OK) S->error = e;
    S->done_cv.notify_all();
}

rei_status server_setup(rei_server *S) {
    rei_ctx *c = S->ctx;
    if (cudaSetDevice(c->device) != cudaSuccess) return REI_ECUDA;
    S->ring_size = 4096;
    S->threads = 256;
    // two CTAs per SM with their static shared memory and reserve
    S->smem = c->smem_sm / 2 > 8192 ? c->smem_sm / 2 - 4096 : 48 * 1024;
    if (stage_layout(kServeMaxIC, kServeMaxBytes, nullptr, nullptr) > S->smem) return REI_EINVAL;
    int bps = 0;
    if (serve_occupancy(S->threads, S->smem, &bps) != cudaSuccess || bps < 1) return REI_ECUDA;
    S->grid = (uint32_t)(c->sm_count * bps);
    const uint64_t slots = S->grid;
    // mapped host memory: the ring, the results, the control words
    if (cudaHostAlloc((void **)&S->ring_h, sizeof(ServeReq) * S->ring_size, cudaHostAllocMapped) != cudaSuccess)
        return REI_ECUDA;
    if (cudaHostAlloc((void **)&S->outs_h, sizeof(ServeOut) * S->ring_size, cudaHostAllocMapped) != cudaSuccess)
        return REI_ECUDA;
    if (cudaHostAlloc((void **)&S->ctl_h, 64, cudaHostAllocMapped) != cudaSuccess) return REI_ECUDA;
    memset(S->ring_h, 0, sizeof(ServeReq) * S->ring_size);  // (sequence words 0: no job yet)
    memset(S->outs_h, 0, sizeof(ServeOut) * S->ring_size);
    memset(S->ctl_h, 0, 64);
    ServeArgs &A = S->args;
    void *dp = nullptr;
    if (cudaHostGetDevicePointer(&dp, S->ring_h, 0) != cudaSuccess) return REI_ECUDA;
    A.ring = (const ServeReq *)dp;
    if (cudaHostGetDevicePointer(&dp, S->outs_h, 0) != cudaSuccess) return REI_ECUDA;
    A.outs = (ServeOut *)dp;
    if (cudaHostGetDevicePointer(&dp, S->ctl_h, 0) != cudaSuccess) return REI_ECUDA;
    A.avail = (const volatile unsigned long long *)dp;
    A.stop = (const volatile unsigned long long *)dp + 1;
    A.ring_size = S->ring_size;
    A.idle_ns = 200ull * 1000 * 1000;
    A.yield_ns = c->opt_yield_us * 1000ull;
    A.smem_cap = S->smem;
    // device memory per slot (rows of up to 64 words: |ic| <= 2048)
    const uint64_t rows = 1ull << 17, chunk = 1ull << 14, wmax = 64;
    const uint64_t tslots = pow2_at_least(2 * (rows + chunk));
    bool oom = false;
    auto take = [&](size_t bytes) -> void * {
        DevBuf b;
        b.p = dev_alloc(c, bytes);
        b.bytes = bytes;
        if (b.p) S->bufs.push_back(b);
        else oom = true;
        return b.p;
    };
    SlotMem &m = A.slot;
    m.rows = rows;
    m.chunk = chunk;
    m.cs_words = rows * wmax;
    m.tmp_words = chunk * wmax;
    m.table_slots = tslots;
    m.cs = (uint32_t *)take(4 * slots * m.cs_words);
    m.bp_op = (uint8_t *)take(slots * rows);
    m.bp_l = (uint32_t *)take(4 * slots * rows);
    m.bp_r = (uint32_t *)take(4 * slots * rows);
    m.used = (uint32_t *)take(4 * slots * rows);
    m.table = (unsigned long long *)take(8 * slots * tslots);
    m.tmp = (uint32_t *)take(4 * slots * m.tmp_words);
    m.pending = (uint32_t *)take(4 * slots * chunk);
    m.slotpos = (uint32_t *)take(4 * slots * chunk);
    m.bitmap = (uint32_t *)take(4 * slots * ((chunk + 31) / 32));
    m.blk = (uint32_t *)take(4 * slots);
    m.lvl = (int64_t *)take(8 * slots * 2 * (kMaxCost + 2));
    m.state = (SolveState *)take(sizeof(SolveState) * slots);
    m.tstack = (uint32_t *)take(16 * slots * (kMaxCost + 2));
    A.in_offs = (uint32_t *)take(4 * slots * (kServeMaxStrings + 1));
    A.word_start = (uint32_t *)take(4 * slots * kMaxIC);
    A.word_len = (uint32_t *)take(4 * slots * kMaxIC);
    A.len_start = (uint32_t *)take(4 * slots * (REI_MAX_STRLEN + 2));
    A.gt_off = (uint32_t *)take(4 * slots * (kMaxIC + 1));
    A.pair_cap = kServePairCap;
    A.gt_pair = (uint32_t *)take(4 * slots * A.pair_cap);
    A.pos = (uint32_t *)take(4 * slots * kMaxWords);
    A.neg = (uint32_t *)take(4 * slots * kMaxWords);
    A.leaf = (uint32_t *)take(4 * slots * kMaxWords * 256);
    A.sinfo = (StageInfo *)take(sizeof(StageInfo) * slots);
    A.head = (unsigned long long *)take(64);
    A.parked = (BatchJob *)take(sizeof(BatchJob) * slots);
    if (oom) return REI_OOM;
    if (cudaStreamCreateWithFlags(&S->kstream, cudaStreamNonBlocking) != cudaSuccess) return REI_ECUDA;
    if (cudaEventCreateWithFlags(&S->kdone, cudaEventDisableTiming) != cudaSuccess) return REI_ECUDA;
    // allocations from the context allocator are stream-ordered on its stream.
    // The slot tables, bitmaps and queue heads are emptied on the launch's own
    // stream and waited for: both streams are non-blocking, so a memset
    // without a stream (legacy default stream) would not be ordered before the
    // first launch, which could then read the memory's previous contents as
    // table entries (row indices from another allocation).
    if (cudaStreamSynchronize(c->stream) != cudaSuccess) return REI_ECUDA;
    if (cudaMemsetAsync(m.table, 0xFF, 8 * slots * tslots, S->kstream) != cudaSuccess) return REI_ECUDA;
    if (cudaMemsetAsync(m.bitmap, 0, 4 * slots * ((chunk + 31) / 32), S->kstream) != cudaSuccess) return REI_ECUDA;
    if (cudaMemsetAsync(A.head, 0, 64, S->kstream) != cudaSuccess) return REI_ECUDA;
    if (cudaStreamSynchronize(S->kstream) != cudaSuccess) return REI_ECUDA;
    return REI_OK;
}

// whether the persistent launch is still running; *err is set when the
// launch (or the context) reported an error instead of finishing
bool kernel_running(rei_server *S, bool *err) {
    *err = false;
    if (!S->running) return false;
    const cudaError_t e = cudaEventQuery(S->kdone);
    if (e == cudaErrorNotReady) return true;
    S->running = false;
    *err = e != cudaSuccess;
    return false;
}

rei_status ensure_kernel(rei_server *S) {
    bool err = false;
    if (kernel_running(S, &err)) return REI_OK;
    if (err) return REI_ECUDA;
    if (launch_serve(&S->args, S->grid, S->threads, S->smem, S->kstream) != cudaSuccess) return REI_ECUDA;
    if (cudaEventRecord(S->kdone, S->kstream) != cudaSuccess) return REI_ECUDA;
    S->ctx->launches++;
    S->running = true;
    return REI_OK;
}

void stop_kernel(rei_server *S) {
    volatile unsigned long long *ctl = S->ctl_h;
    ctl[1] = 1;
    std::atomic_thread_fence(std::memory_order_seq_cst);
    if (S->running) cudaEventSynchronize(S->kdone);
    S->running = false;
    ctl[1] = 0;
    std::atomic_thread_fence(std::memory_order_seq_cst);
}

void finish(rei_server *S, uint64_t ticket, const rei_result &r, const char *regex, size_t rlen,
            const uint8_t *tree, size_t tlen) {
    rei_server::Done d{};
    d.r = r;
    d.regex.assign(regex, rlen);
    d.tree.assign(tree, tree + tlen);
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->done[ticket] = std::move(d);
    }
    S->done_cv.notify_all();
}

// a served search's report (from its slot, or its slot group) as its result
void finish_served(rei_server *S, const rei_server::Req &req, const ServeOut &o, const BatchOut &b, double ms,
                   uint32_t launches) {
    rei_result r{};
    r.stats.n_ic = o.info.n;
    r.stats.words = o.info.W;
    r.stats.max_len = o.info.max_len;
    r.stats.guide_pairs = o.info.G;
    r.stats.candidates = b.candidates;
    r.stats.unique = b.unique;
    r.stats.levels = b.levels;
    for (int k = 0; k < 5; k++) r.stats.cand_op[k] = b.cand_op[k];
    r.stats.ms_search_kernel = ms;
    r.stats.ms_total = now_ms() - req.t_submit;
    r.stats.search_launches = launches;
    switch (b.status) {
    case ST_FOUND: r.status = REI_OK; break;
    case ST_NOT_FOUND: r.status = REI_NOT_FOUND; break;
    case ST_OOM: r.status = REI_OOM; break;
    case ST_BAD: r.status = REI_EINVAL; break;
    default: r.status = REI_ECUDA; break;
    }
    std::string text;
    uint32_t ntok = 0;
    if (r.status == REI_OK) {
        r.cost = b.cost;
        ntok = b.tree_len;
        text = format_regex(o.tree, ntok, req.alphabet.data());
    }
    r.regex_len = text.size();
    r.tree_len = 2ull * ntok;
    finish(S, req.ticket, r, text.data(), text.size(), o.tree, 2ull * ntok);
}

// a slot whose search continues elsewhere: its table and chunk bitmap are
// emptied for its next request (ordered before the next launch)
void empty_slot(rei_server *S, uint32_t slot) {
    const SlotMem &m = S->args.slot;
    const uint64_t bmw = (m.chunk + 31) / 32;
    cudaMemsetAsync(m.table + (uint64_t)slot * m.table_slots, 0xFF, 8 * m.table_slots, S->kstream);
    cudaMemsetAsync(m.bitmap + (uint64_t)slot * bmw, 0, 4 * bmw, S->kstream);
}

// the searches in `alone` that stopped at their time allowance continue in
// their slots, side by side in one launch (a group of CTAs each, as in the
// batched form); those that finish are answered and leave `alone`
void continue_in_slots(rei_server *S, std::vector<rei_server::Req> &alone) {
    rei_ctx *c = S->ctx;
    std::vector<size_t> gi;
    for (size_t i = 0; i < alone.size(); i++)
        if (alone[i].slot < S->grid && alone[i].need_rows == 0) gi.push_back(i);
    if (gi.empty()) return;
    const uint32_t threads_g = 256;
    size_t smem_g = 0, smem_gmax = 0;
    uint32_t seg_cap_g = 0, wmax_g = 1;
    for (size_t i : gi) {
        const StageInfo &I = S->outs_h[alone[i].job % S->ring_size].info;
        const uint32_t seg_cap = 2 * alone[i].p.max_cost + 4;
        // (the guide table in shared memory as the served CTA decided it)
        const bool gt = solve_smem_bytes(I.W, I.n, I.G, I.max_len, seg_cap, true, threads_g / 32) <= S->smem;
        smem_g = std::max(smem_g, solve_smem_bytes(I.W, I.n, I.G, I.max_len, seg_cap, gt, threads_g / 32));
        seg_cap_g = std::max(seg_cap_g, seg_cap);
        wmax_g = std::max(wmax_g, I.W);
    }
    if (solve_groups_smem_max(&smem_gmax) != cudaSuccess || smem_g > smem_gmax) return;
    int bps = 0;
    if (solve_groups_occupancy(threads_g, smem_g, &bps) != cudaSuccess || bps < 1) return;
    const uint32_t cap = (uint32_t)bps * (uint32_t)c->sm_count;
    const uint32_t ng = (uint32_t)std::min<size_t>(gi.size(), cap / 2);
    if (ng == 0) return;
    const uint32_t gctas = std::min<uint32_t>(cap / ng, kMaxTeam);
    const uint64_t pstride = plan_words(seg_cap_g);
    uint64_t chunk_g = 1ull << 18;
    while (chunk_g > 4096 && chunk_g * wmax_g * ng > (1ull << 28)) chunk_g >>= 1;
    const uint64_t tmp_g = chunk_g * wmax_g, bmw_g = (chunk_g + 31) / 32;
    if (ensure(c, c->g_idx, 8ull * ng) || ensure(c, c->g_blk, 4ull * ng * gctas) ||
        ensure(c, c->g_plan, 8ull * ng * pstride) || ensure(c, c->g_tmp, 4ull * ng * tmp_g) ||
        ensure(c, c->g_pend, 4ull * ng * chunk_g) || ensure(c, c->g_slotpos, 4ull * ng * chunk_g) ||
        ensure(c, c->g_bitmap, 4ull * ng * bmw_g) || ensure_pinned(c, 8ull * ng))
        return;
    // (allocations on the context's stream; and no copy uses the pinned buffer)
    if (cudaStreamSynchronize(c->stream) != cudaSuccess) return;
    uint32_t *gidx = (uint32_t *)c->h_pin;
    for (uint32_t g = 0; g < ng; g++) gidx[g] = gidx[ng + g] = alone[gi[g]].slot;
    GroupArgs G{};
    G.slot = S->args.slot;
    G.prob = (const uint32_t *)c->g_idx.p;
    G.slot_of = (const uint32_t *)c->g_idx.p + ng;
    G.groups = ng;
    G.group_ctas = gctas;
    G.blk = (uint32_t *)c->g_blk.p;
    G.plan = (uint64_t *)c->g_plan.p;
    G.plan_stride = pstride;
    G.tmp = (uint32_t *)c->g_tmp.p;
    G.pending = (uint32_t *)c->g_pend.p;
    G.slotpos = (uint32_t *)c->g_slotpos.p;
    G.bitmap = (uint32_t *)c->g_bitmap.p;
    G.chunk = chunk_g;
    G.tmp_words = tmp_g;
    if (cudaMemcpyAsync(c->g_idx.p, gidx, 8ull * ng, cudaMemcpyHostToDevice, S->kstream) != cudaSuccess ||
        cudaMemsetAsync(c->g_bitmap.p, 0, 4ull * ng * bmw_g, S->kstream) != cudaSuccess ||
        launch_solve_groups(S->args.parked, &G, ng * gctas, threads_g, smem_g, S->kstream) != cudaSuccess ||
        cudaStreamSynchronize(S->kstream) != cudaSuccess) {
        // (nothing was answered: every search continues alone, from its slot)
        return;
    }
    c->launches++;
    c->pin_clean = true;
    std::vector<rei_server::Req> rest;
    std::vector<bool> grouped(alone.size(), false);
    for (uint32_t g = 0; g < ng; g++) grouped[gi[g]] = true;
    for (size_t i = 0; i < alone.size(); i++) {
        rei_server::Req &req = alone[i];
        if (!grouped[i]) {
            rest.push_back(std::move(req));
            continue;
        }
        const ServeOut &o = S->outs_h[req.job % S->ring_size];
        std::atomic_thread_fence(std::memory_order_acquire);  // (the launch has finished: its writes are in)
        const BatchOut b = o.out;
        const double ms = req.ms_slot + b.ns / 1e6;
        if (b.status == ST_FOUND || b.status == ST_NOT_FOUND || b.status == ST_OOM) {
            finish_served(S, req, o, b, ms, 2);
        } else {
            // (outgrew its slot in the group, or failed there: continued alone)
            req.need_rows = b.status == ST_NEED_MEM ? std::max<uint32_t>(1, b.need_rows) : 1u;
            req.ms_slot = ms;
            rest.push_back(std::move(req));
        }
    }
    alone.swap(rest);
}

void solve_alone(rei_server *S, rei_server::Req &req) {
    req.p.alphabet = req.alphabet.data();
    req.p.bytes = req.bytes.data();
    req.p.offsets = req.offs.data();
    req.p.sym_costs = req.sym_costs.empty() ? nullptr : req.sym_costs.data();
    char rbuf[8192];
    uint8_t tbuf[2 * (REI_MAX_COST + 1)];
    rei_result r{};
    r.regex = rbuf;
    r.regex_cap = sizeof rbuf;
    r.tree = tbuf;
    r.tree_cap = sizeof tbuf;
    rei_status s;
    {
        // a search left in a memory slot continues from there (the launch is
        // stopped, so the slot is as the search left it)
        const SlotResume rs{&S->args.slot, req.slot};
        std::lock_guard<std::mutex> g(S->ctx->mu);
        s = solve_one(S->ctx, &req.p, &r, req.slot < S->grid ? &rs : nullptr);
    }
    if (s != REI_OK && s != REI_NOT_FOUND && s != REI_OOM) r.status = s;
    r.stats.ms_total = now_ms() - req.t_submit;
    finish(S, req.ticket, r, rbuf, r.status == REI_OK ? r.regex_len : 0, tbuf,
           r.status == REI_OK ? r.tree_len : 0);
}

void server_loop(rei_server *S) {
    cudaSetDevice(S->ctx->device);
    volatile unsigned long long *ctl = S->ctl_h;
    std::vector<rei_server::Req> alone;
    // completions of the live requests: answered ones are finished, parked
    // ones move to `alone`
    auto collect = [&]() {
        bool any = false;
        for (auto it = S->live.begin(); it != S->live.end();) {
            const uint64_t job = it->first;
            ServeOut &o = S->outs_h[job % S->ring_size];
            if (*(volatile unsigned long long *)&o.done != job + 1) {
                ++it;
                continue;
            }
            std::atomic_thread_fence(std::memory_order_acquire);
            rei_server::Req &req = it->second;
            const BatchOut b = o.out;
            any = true;
            S->live_bytes -= req.footprint;
            if (b.status == ST_NEED_MEM) {
                req.slot = b.slot;
                req.need_rows = b.need_rows;
                req.job = job;
                req.ms_slot = b.ns / 1e6;
                alone.push_back(std::move(req));
                it = S->live.erase(it);
                continue;
            }
            finish_served(S, req, o, b, b.ns / 1e6, 1);
            it = S->live.erase(it);
        }
        return any;
    };
    // searches a launch left in their slots, and requests too large for a
    // slot, once the launch has ended (and every search it parked is in
    // `alone`: a slot is reused only by a later launch): those that stopped
    // at their time allowance continue side by side in their slots, the
    // others (and any that outgrow their slot there) alone on the whole GPU
    auto handle_alone = [&]() {
        stop_kernel(S);
        collect();  // (searches parked while the launch was stopping)
        continue_in_slots(S, alone);
        for (auto &req : alone) {
            if (req.slot < S->grid) empty_slot(S, req.slot);
            solve_alone(S, req);
        }
        alone.clear();
    };
    for (;;) {
        bool progress = false;
        // 1. completions
        if (collect()) progress = true;
        // 2. parked searches and requests too large for a slot
        if (!alone.empty()) {
            handle_alone();
            progress = true;
        }
        // 3. admissions into the ring, then one publication
        uint64_t admitted = 0;
        {
            std::unique_lock<std::mutex> lk(S->mu);
            const uint64_t oldest = S->live.empty() ? S->published : S->live.begin()->first;
            while (!S->queue.empty() && S->live.size() < S->max_live &&
                   S->published + 1 - oldest <= S->ring_size &&
                   (S->live.empty() || S->live_bytes + S->queue.front().footprint <= S->budget)) {
                rei_server::Req req = std::move(S->queue.front());
                S->queue.pop_front();
                const uint32_t n_str = req.p.n_pos + req.p.n_neg;
                const uint32_t total = req.offs.back();
                if (n_str > kServeMaxStrings || total > kServeMaxBytes) {
                    alone.push_back(std::move(req));
                    continue;
                }
                const uint64_t job = S->published;
                ServeReq &q = S->ring_h[job % S->ring_size];
                q.n_pos = req.p.n_pos;
                q.n_neg = req.p.n_neg;
                q.n_sym = req.p.n_sym;
                q.total_bytes = total;
                memcpy(q.alphabet, req.alphabet.data(), req.p.n_sym);
                q.costs = req.p.costs;
                q.max_cost = req.p.max_cost;
                q.max_errors = req.p.max_errors;
                q.flags = req.p.flags & ~REI_F_DEVICE_INPUT;
                q.mem_budget = req.p.mem_budget;
                req.p.alphabet = req.alphabet.data();
                req.p.sym_costs = req.sym_costs.empty() ? nullptr : req.sym_costs.data();
                fill_leaves(&req.p, &q.cmin, q.leaf_cost, q.leaf_sym);
                memcpy(q.offs, req.offs.data(), 4ull * (n_str + 1));
                if (total) memcpy(q.bytes, req.bytes.data(), total);
                // the entry's sequence word last: a launch that sees it reads a whole entry
                std::atomic_thread_fence(std::memory_order_seq_cst);
                *(volatile unsigned long long *)&q.seq = job + 1;
                S->live_bytes += req.footprint;
                S->live[job] = std::move(req);
                S->published++;
                admitted++;
            }
        }
        if (admitted) {
            std::atomic_thread_fence(std::memory_order_seq_cst);
            ctl[0] = S->published;
            std::atomic_thread_fence(std::memory_order_seq_cst);
            progress = true;
        }
        // 4. a launch must be running while published requests wait; before
        // a new launch reuses the slots, every search the last one parked is
        // continued (its completion may have arrived after step 1)
        if (!S->live.empty()) {
            bool kerr = false;
            const bool running = kernel_running(S, &kerr);
            if (kerr) {
                server_fail(S, REI_ECUDA);
                return;
            }
            if (!running) {
                collect();
                if (!alone.empty()) handle_alone();
            }
            const rei_status s = ensure_kernel(S);
            if (s != REI_OK) {
                server_fail(S, s);
                return;
            }
        }
        // 5. wait for work, or poll completions
        std::unique_lock<std::mutex> lk(S->mu);
        if (S->stop && S->queue.empty() && S->live.empty() && alone.empty()) break;
        if (!progress) {
            if (S->live.empty()) S->cv.wait_for(lk, std::chrono::milliseconds(2));
            else {
                lk.unlock();
                std::this_thread::sleep_for(std::chrono::microseconds(20));
            }
        }
    }
    stop_kernel(S);
}

}  // namespace

extern "C" {

rei_status rei_server_create(rei_ctx *ctx, uint64_t budget_bytes, uint32_t max_live, rei_server **out) {
    if (!ctx || !out || max_live == 0) return REI_EINVAL;
    rei_server *S = new rei_server();
    S->ctx = ctx;
    S->budget = budget_bytes;
    S->max_live = max_live;
    rei_status s = server_setup(S);
    if (s != REI_OK) {
        rei_server_destroy(S);
        return s;
    }
    S->max_live = std::min<uint32_t>(max_live, S->ring_size);
    S->worker = std::thread(server_loop, S);
    *out = S;
    return REI_OK;
}

rei_status rei_server_submit(rei_server *S, const rei_problem *p, uint64_t *ticket) {
    if (!S || !p || !ticket) return REI_EINVAL;
    if (p->flags & REI_F_DEVICE_INPUT) return REI_EINVAL;
    rei_status s = check_problem(p);
    if (s) return s;
    rei_server::Req r;
    const uint32_t n_str = p->n_pos + p->n_neg;
    r.alphabet.assign(p->alphabet, p->alphabet + p->n_sym);
    if (n_str) r.offs.assign(p->offsets, p->offsets + n_str + 1);
    else r.offs.assign(1, 0);
    const uint32_t total = r.offs.back();
    r.bytes.assign(p->bytes, p->bytes + total);
    if (p->sym_costs) r.sym_costs.assign(p->sym_costs, p->sym_costs + p->n_sym);
    r.p = *p;
    r.t_submit = now_ms();
    // the cache this request may hold: its budget, at most one slot's cache
    const uint64_t slot_bytes = S->args.slot.rows * (4ull * 64 + 28);
    r.footprint = std::min<uint64_t>(p->mem_budget, slot_bytes);
    {
        std::lock_guard<std::mutex> lk(S->mu);
        if (S->error != REI_OK) return S->error;
        r.ticket = S->next_ticket++;
        *ticket = r.ticket;
        S->open.insert(r.ticket);
        S->queue.push_back(std::move(r));
    }
    S->cv.notify_one();
    return REI_OK;
}

rei_status rei_server_poll(rei_server *S, uint64_t ticket, rei_result *out, int block_ms) {
    if (!S || !out) return REI_EINVAL;
    std::unique_lock<std::mutex> lk(S->mu);
    if (!S->open.count(ticket)) return REI_EINVAL;
    auto ready = [&] { return S->done.count(ticket) > 0 || S->error != REI_OK; };
    if (!ready()) {
        if (block_ms == 0) return REI_EBUSY;
        if (block_ms < 0) S->done_cv.wait(lk, ready);
        else if (!S->done_cv.wait_for(lk, std::chrono::milliseconds(block_ms), ready)) return REI_EBUSY;
    }
    if (!S->done.count(ticket)) return S->error;
    rei_server::Done &d = S->done[ticket];
    char *rb = out->regex;
    size_t rc = out->regex_cap;
    uint8_t *tb = out->tree;
    size_t tc = out->tree_cap;
    *out = d.r;
    out->regex = rb;
    out->regex_cap = rc;
    out->tree = tb;
    out->tree_cap = tc;
    out->regex_len = d.regex.size();
    out->tree_len = d.tree.size();
    rei_status s = REI_OK;
    if (rb) {
        if (rc >= d.regex.size() + 1) {
            memcpy(rb, d.regex.data(), d.regex.size());
            rb[d.regex.size()] = 0;
        } else {
            s = REI_EBUFSZ;
        }
    }
    if (tb) {
        if (tc >= d.tree.size()) memcpy(tb, d.tree.data(), d.tree.size());
        else s = REI_EBUFSZ;
    }
    if (s == REI_OK) {
        S->done.erase(ticket);
        S->open.erase(ticket);
    }
    return s;
}

void rei_server_destroy(rei_server *S) {
    if (!S) return;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
    }
    S->cv.notify_all();
    if (S->worker.joinable()) S->worker.join();
    if (S->kstream) {
        cudaStreamSynchronize(S->kstream);
        cudaStreamDestroy(S->kstream);
    }
    if (S->kdone) cudaEventDestroy(S->kdone);
    if (getenv("REI_DEBUG") && S->args.head) {
        unsigned long long h[3] = {0, 0, 0};
        if (cudaMemcpyAsync(h, S->args.head, sizeof h, cudaMemcpyDeviceToHost, S->ctx->stream) == cudaSuccess &&
            cudaStreamSynchronize(S->ctx->stream) == cudaSuccess)
            fprintf(stderr, "rei server: %llu jobs claimed, %llu ring entries incomplete when first read, "
                    "%llu given up\n", h[0], h[1], h[2]);
    }
    for (DevBuf &b : S->bufs) dev_free(S->ctx, b);
    if (S->ring_h) cudaFreeHost(S->ring_h);
    if (S->outs_h) cudaFreeHost(S->outs_h);
    if (S->ctl_h) cudaFreeHost(S->ctl_h);
    delete S;
}

}  // extern "C"
