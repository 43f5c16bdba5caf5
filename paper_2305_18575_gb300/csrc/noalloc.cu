// noalloc.cu -- rei_solve_noalloc: a solve that allocates nothing.
//
// Some callers cannot allocate device memory while they solve: code that runs
// inside another framework's fixed memory arena, a real-time or signal-safe
// host thread that must not enter the CUDA allocator (which can block on
// device-wide synchronisation), or a process whose allocator is owned by
// someone else.  For them this entry point runs the same staging and search
// kernels as rei_solve_problem, but every piece of device scratch (the
// uploaded strings, the staged problem, the language cache, the uniqueness
// table, the chunk workspace and the search state) is carved out of one
// file-scope device array of fixed size, reserved when the library is
// loaded and held by every GPU that loads it until the process exits.
//
// Host code cannot use the array's name as a device address (on the host it
// names a host-side stand-in), so the first call on each device looks its
// device address up with cudaGetSymbolAddress, with that device current, and
// caches it.  Every call waits for its stream partway through (to read the
// staged sizes back), so no call can run while its stream is being captured
// into a graph.  All calls share the one array and it keeps the previous call's contents: the
// regions that must start cleared are cleared on the caller's stream at the
// start of every call, and calls that overlap on the GPU (two streams, two
// host threads) race on the array and must not be issued.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstring>
#include <mutex>

#include "rei_dev.cuh"
#include "args.h"

namespace rei {
cudaError_t launch_stage(const StageJob *jobs_dev, uint32_t n_jobs, cudaStream_t stream);
cudaError_t launch_solve(const SolveJob *job, uint32_t grid, uint32_t threads, size_t smem,
                         cudaStream_t stream);
cudaError_t solve_occupancy(uint32_t threads, size_t smem, int *blocks_per_sm);
cudaError_t solve_smem_max(size_t *bytes);
size_t solve_smem_bytes(uint32_t W, uint32_t n, uint32_t G, uint32_t max_len, uint32_t seg_cap,
                        bool gt_in_smem, uint32_t warps, uint32_t small_rows = 0);
}  // namespace rei

using namespace rei;

namespace {

constexpr size_t kAlign = 256;
constexpr size_t kInputBytes = 1u << 20;      // example bytes
constexpr uint32_t kMaxStrings = 1u << 16;    // examples (offsets table)
constexpr uint32_t kPairCap = 1u << 18;       // guide-table pairs
constexpr uint32_t kMaxGrid = 4096;           // search CTAs
constexpr uint64_t kChunkMax = 1u << 16;      // candidates per dedup chunk

// the scratch array: REI_NOALLOC_SCRATCH_BYTES bytes on every device
static __device__ __align__(256) unsigned char g_scratch[REI_NOALLOC_SCRATCH_BYTES];

std::mutex g_setup_mu;
unsigned char *g_scratch_dev[256] = {};  // device address of g_scratch per device ordinal

// set-up, once per device: the device address of the scratch array
cudaError_t scratch_address(int device, unsigned char **out) {
    std::lock_guard<std::mutex> g(g_setup_mu);
    if (device < 0 || device >= 256) return cudaErrorInvalidDevice;
    if (!g_scratch_dev[device]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_dev[device] = (unsigned char *)p;
    }
    *out = g_scratch_dev[device];
    return cudaSuccess;
}

// bump carving of the scratch array
struct Carve {
    unsigned char *base;
    size_t used, cap;
    void *take(size_t bytes) {
        const size_t at = (used + kAlign - 1) & ~(kAlign - 1);
        if (at + bytes > cap) return nullptr;
        used = at + bytes;
        return base + at;
    }
};

uint64_t pow2_at_least(uint64_t x) {
    uint64_t p = 1;
    while (p < x) p <<= 1;
    return p;
}

// postfix tokens -> pretty string, with fixed-size stack storage only
size_t format_noalloc(const uint8_t *tok, uint32_t ntok, const uint8_t *alpha, char *out, size_t cap) {
    struct N {
        uint8_t k, a;
        int l, r;
    };
    N nodes[REI_MAX_COST + 2];
    int st[REI_MAX_COST + 2];
    int sp = 0;
    if (ntok > REI_MAX_COST + 1) return 0;
    for (uint32_t i = 0; i < ntok; i++) {
        const uint8_t k = tok[2 * i], a = tok[2 * i + 1];
        N n{k, a, -1, -1};
        if (k == '?' || k == '*') {
            if (sp < 1) return 0;
            n.l = st[--sp];
        } else if (k == '.' || k == '+') {
            if (sp < 2) return 0;
            n.r = st[--sp];
            n.l = st[--sp];
        }
        nodes[i] = n;
        st[sp++] = (int)i;
    }
    if (sp != 1) return 0;
    // iterative printer: frames of (node, need, stage)
    struct F {
        int x, need, stage;
    };
    F fr[2 * (REI_MAX_COST + 2)];
    int fp = 0;
    size_t len = 0;
    auto put = [&](const char *s, size_t n) {
        for (size_t i = 0; i < n; i++) {
            if (len + 1 < cap) out[len] = s[i];
            len++;
        }
    };
    auto prec = [](uint8_t k) { return k == '+' ? 0 : k == '.' ? 1 : 2; };
    fr[fp++] = {st[0], 0, 0};
    while (fp > 0) {
        F &f = fr[fp - 1];
        const N &n = nodes[f.x];
        const bool par = prec(n.k) < f.need;
        if (f.stage == 0) {
            if (par) put("(", 1);
            f.stage = 1;
            if (n.k == 'a') {
                const char c = (char)alpha[n.a];
                put(&c, 1);
            } else if (n.k == 'e') {
                put("\xce\xb5", 2);
            } else if (n.k == '0') {
                put("\xe2\x88\x85", 3);
            } else {
                const int need = (n.k == '?' || n.k == '*') ? 2 : prec(n.k);
                fr[fp++] = {n.l, need, 0};
            }
            continue;
        }
        if (f.stage == 1 && (n.k == '.' || n.k == '+')) {
            f.stage = 2;
            if (n.k == '+') put("+", 1);
            fr[fp++] = {n.r, prec(n.k), 0};
            continue;
        }
        if (n.k == '?' || n.k == '*') {
            const char c = (char)n.k;
            put(&c, 1);
        }
        if (par) put(")", 1);
        fp--;
    }
    // always terminated when there is room for one byte (a string that does
    // not fit is cut at cap - 1 bytes; the caller gets REI_EBUFSZ and the length)
    if (cap) out[len < cap ? len : cap - 1] = 0;
    return len;
}

// a failed CUDA call ends the call with REI_ECUDA, in the return value and
// in out->status alike
#define NA_CK(x)                          \
    do {                                  \
        if ((x) != cudaSuccess) {         \
            out->status = REI_ECUDA;      \
            return REI_ECUDA;             \
        }                                 \
    } while (0)

// every early return: the same status in the return value and out->status
#define NA_RET(st)            \
    do {                      \
        out->status = (st);   \
        return (st);          \
    } while (0)

}  // namespace

extern "C" rei_status rei_solve_noalloc(const rei_problem *p, void *stream_v, rei_result *out) {
    if (!p || !out) return REI_EINVAL;
    const cudaStream_t stream = (cudaStream_t)stream_v;
    memset(&out->stats, 0, sizeof(out->stats));
    out->status = REI_EINVAL;
    out->cost = 0;
    out->regex_len = 0;
    out->tree_len = 0;

    // argument checks: the rules of every other entry point (args.h)
    if (check_problem(p) != REI_OK) NA_RET(REI_EINVAL);
    const uint32_t n_str = p->n_pos + p->n_neg;  // (at most 2^24: checked)
    const bool dev_in = (p->flags & REI_F_DEVICE_INPUT) != 0;
    const uint64_t total = dev_in ? p->total_bytes : (n_str ? p->offsets[n_str] : 0);
    // sizes beyond what the scratch array holds are refused, not truncated
    if (total > kInputBytes || n_str + 1 > kMaxStrings) NA_RET(REI_ESCRATCH);

    int device = 0;
    NA_CK(cudaGetDevice(&device));
    unsigned char *scratch = nullptr;
    NA_CK(scratch_address(device, &scratch));
    cudaDeviceProp prop;
    NA_CK(cudaGetDeviceProperties(&prop, device));

    Carve cv{scratch, 0, (size_t)REI_NOALLOC_SCRATCH_BYTES};
    uint8_t *d_bytes = (uint8_t *)cv.take(kInputBytes);
    uint32_t *d_offs = (uint32_t *)cv.take(4ull * kMaxStrings);
    StageJob *d_sj = (StageJob *)cv.take(sizeof(StageJob));
    StageInfo *d_si = (StageInfo *)cv.take(sizeof(StageInfo));
    uint32_t *d_ws = (uint32_t *)cv.take(4ull * kMaxIC);
    uint32_t *d_wl = (uint32_t *)cv.take(4ull * kMaxIC);
    uint32_t *d_ls = (uint32_t *)cv.take(4ull * (REI_MAX_STRLEN + 2));
    uint32_t *d_go = (uint32_t *)cv.take(4ull * (kMaxIC + 1));
    uint32_t *d_gp = (uint32_t *)cv.take(4ull * kPairCap);
    uint32_t *d_pos = (uint32_t *)cv.take(4ull * kMaxWords);
    uint32_t *d_neg = (uint32_t *)cv.take(4ull * kMaxWords);
    uint32_t *d_leaf = (uint32_t *)cv.take(4ull * kMaxWords * 256);
    const size_t tree_bytes = 2ull * (REI_MAX_COST + 1);
    SolveState *d_st = (SolveState *)cv.take(sizeof(SolveState) + tree_bytes);
    int64_t *d_lvs = (int64_t *)cv.take(8ull * (REI_MAX_COST + 2));
    int64_t *d_lvc = (int64_t *)cv.take(8ull * (REI_MAX_COST + 2));
    uint32_t *d_tstack = (uint32_t *)cv.take(16ull * (REI_MAX_COST + 2));
    uint32_t *d_trace = (uint32_t *)cv.take(4ull * kMaxGrid);
    uint32_t *d_blk = (uint32_t *)cv.take(4ull * kMaxGrid);
    if (!d_blk) NA_RET(REI_ESCRATCH);

    // inputs: device inputs are read in place; host inputs are copied in
    const uint8_t *in_bytes = d_bytes;
    const uint32_t *in_offs = d_offs;
    if (dev_in && n_str) {
        in_bytes = p->bytes;
        in_offs = p->offsets;
    } else {
        if (total) NA_CK(cudaMemcpyAsync(d_bytes, p->bytes, total, cudaMemcpyHostToDevice, stream));
        if (n_str) NA_CK(cudaMemcpyAsync(d_offs, p->offsets, 4ull * (n_str + 1), cudaMemcpyHostToDevice, stream));
        else NA_CK(cudaMemsetAsync(d_offs, 0, 4, stream));
        out->stats.bytes_h2d += total + 4ull * (n_str + 1);
    }

    // staging
    StageJob sj;
    memset(&sj, 0, sizeof sj);
    sj.bytes = in_bytes;
    sj.offs = in_offs;
    sj.n_pos = p->n_pos;
    sj.n_neg = p->n_neg;
    memcpy(sj.alphabet, p->alphabet, p->n_sym);
    sj.n_sym = p->n_sym;
    sj.total_bytes = (uint32_t)total;
    sj.info = d_si;
    sj.word_start = d_ws;
    sj.word_len = d_wl;
    sj.len_start = d_ls;
    sj.gt_off = d_go;
    sj.gt_pair = d_gp;
    sj.pair_cap = kPairCap;
    sj.pos_mask = d_pos;
    sj.neg_mask = d_neg;
    sj.leaf = d_leaf;
    NA_CK(cudaMemcpyAsync(d_sj, &sj, sizeof sj, cudaMemcpyHostToDevice, stream));
    NA_CK(cudaMemsetAsync(d_si, 0, sizeof(StageInfo), stream));
    NA_CK(launch_stage(d_sj, 1, stream));
    StageInfo I;
    NA_CK(cudaMemcpyAsync(&I, d_si, sizeof I, cudaMemcpyDeviceToHost, stream));
    NA_CK(cudaStreamSynchronize(stream));
    out->stats.launches = 1;
    out->stats.n_ic = I.n;
    out->stats.words = I.W;
    out->stats.max_len = I.max_len;
    out->stats.guide_pairs = I.G;
    if (I.status == SE_PAIRS) NA_RET(REI_ESCRATCH);
    if (I.status != SE_OK) NA_RET(REI_EINVAL);

    const uint32_t n = I.n, W = I.W, G = I.G, max_len = I.max_len, max_cost = p->max_cost;
    const uint64_t per = 4ull * W + 28;
    const uint64_t cap = std::min<uint64_t>(p->mem_budget / per, 0x7FFF0000ull);

    // the search region: chunk workspace, then the whole cache and its table
    const uint64_t chunk = std::max<uint64_t>(1024, std::min<uint64_t>(kChunkMax, (4ull << 20) / (4ull * W)));
    const uint64_t tslots = pow2_at_least(std::max<uint64_t>(2 * (cap + chunk), 1024));
    uint32_t *d_tmp = (uint32_t *)cv.take(4ull * W * chunk);
    uint32_t *d_pend = (uint32_t *)cv.take(4ull * chunk);
    uint32_t *d_slot = (uint32_t *)cv.take(4ull * chunk);
    uint32_t *d_bitmap = (uint32_t *)cv.take(4ull * ((chunk + 31) / 32));
    unsigned long long *d_table = (unsigned long long *)cv.take(8ull * tslots);
    uint32_t *d_cs = (uint32_t *)cv.take(4ull * W * std::max<uint64_t>(cap, 1));
    uint8_t *d_op = (uint8_t *)cv.take(std::max<uint64_t>(cap, 1));
    uint32_t *d_l = (uint32_t *)cv.take(4ull * std::max<uint64_t>(cap, 1));
    uint32_t *d_r = (uint32_t *)cv.take(4ull * std::max<uint64_t>(cap, 1));
    uint32_t *d_used = (uint32_t *)cv.take(4ull * std::max<uint64_t>(cap, 1));
    if (!d_used) NA_RET(REI_ESCRATCH);  // the budget's cache does not fit the array

    // launch shape (as the allocating path chooses it), within the dynamic
    // shared memory the search kernel can take
    size_t smem_max = 0;
    NA_CK(solve_smem_max(&smem_max));
    const uint32_t seg_cap = 2 * max_cost + 4;
    bool gt_smem = 4ull * (n + 1 + G + max_len + 2) <= 96 * 1024;
    uint32_t warps = 8;
    size_t smem = solve_smem_bytes(W, n, G, max_len, seg_cap, gt_smem, warps);
    while (smem > smem_max && warps > 1) {
        warps /= 2;
        smem = solve_smem_bytes(W, n, G, max_len, seg_cap, gt_smem, warps);
    }
    if (smem > smem_max && gt_smem) {
        gt_smem = false;
        warps = 8;
        smem = solve_smem_bytes(W, n, G, max_len, seg_cap, gt_smem, warps);
        while (smem > smem_max && warps > 1) {
            warps /= 2;
            smem = solve_smem_bytes(W, n, G, max_len, seg_cap, gt_smem, warps);
        }
    }
    if (smem > smem_max) NA_RET(REI_EINVAL);
    int bps = 0;
    NA_CK(solve_occupancy(32 * warps, smem, &bps));
    if (bps < 1) NA_RET(REI_ECUDA);
    const uint32_t grid = std::min<uint32_t>(kMaxTeam, (uint32_t)(prop.multiProcessorCount * bps));

    // what must start cleared: table, survivor bitmap, level sizes
    NA_CK(cudaMemsetAsync(d_table, 0xFF, 8ull * tslots, stream));
    NA_CK(cudaMemsetAsync(d_bitmap, 0, 4ull * ((chunk + 31) / 32), stream));
    NA_CK(cudaMemsetAsync(d_lvs, 0, 8ull * (REI_MAX_COST + 2), stream));
    NA_CK(cudaMemsetAsync(d_lvc, 0, 8ull * (REI_MAX_COST + 2), stream));
    SolveState hs;
    memset(&hs, 0, sizeof hs);
    hs.status = ST_RUNNING;
    {
        uint16_t lc[256];
        uint8_t ls[256];
        fill_leaves(p, &hs.level, lc, ls);
    }
    hs.found = kNone;
    hs.partial_level = max_cost + 1;
    NA_CK(cudaMemcpyAsync(d_st, &hs, sizeof hs, cudaMemcpyHostToDevice, stream));

    SolveJob j;
    memset(&j, 0, sizeof j);
    j.n = n;
    j.W = W;
    j.G = G;
    j.n_sym = p->n_sym;
    j.max_len = max_len;
    j.gt_off = d_go;
    j.gt_pair = d_gp;
    j.len_start = d_ls;
    j.pos_mask = d_pos;
    j.neg_mask = d_neg;
    j.leaf = d_leaf;
    j.leaf_stride = kMaxWords;
    j.n_pos_set = I.n_pos_set;
    j.pos_eps = I.pos_eps;
    j.neg_eps = I.neg_eps;
    j.c[0] = p->costs.c_sym;
    j.c[1] = p->costs.c_opt;
    j.c[2] = p->costs.c_star;
    j.c[3] = p->costs.c_cat;
    j.c[4] = p->costs.c_alt;
    fill_leaves(p, &j.cmin, j.leaf_cost, j.leaf_sym);
    j.max_cost = max_cost;
    j.max_errors = p->max_errors;
    j.flags = p->flags;
    j.cap = cap;
    j.cs = d_cs;
    j.bp_op = d_op;
    j.bp_l = d_l;
    j.bp_r = d_r;
    j.used = d_used;
    j.cache_alloc = cap;  // the whole budget is resident: the search never asks to grow
    j.table = d_table;
    j.table_mask = tslots - 1;
    j.tmp = d_tmp;
    j.pending = d_pend;
    j.slotpos = d_slot;
    j.bitmap = d_bitmap;
    j.blk = d_blk;
    j.chunk_max = chunk;
    j.lvl_start = d_lvs;
    j.lvl_count = d_lvc;
    j.seg_cap = seg_cap;
    j.st = d_st;
    j.tree = (uint8_t *)(d_st + 1);
    j.tstack = d_tstack;
    j.trace = d_trace;
    j.gt_in_smem = gt_smem ? 1 : 0;
    j.solo_tiles = 8 * warps;
    NA_CK(launch_solve(&j, grid, 32 * warps, smem, stream));
    struct {
        SolveState s;
        uint8_t tree[2 * (REI_MAX_COST + 1)];
    } hr;
    NA_CK(cudaMemcpyAsync(&hr, d_st, sizeof(SolveState) + tree_bytes, cudaMemcpyDeviceToHost, stream));
    NA_CK(cudaStreamSynchronize(stream));
    out->stats.launches = 2;
    out->stats.search_launches = 1;
    out->stats.grid = grid;
    out->stats.candidates = hr.s.candidates;
    out->stats.unique = hr.s.unique_done;
    out->stats.levels = hr.s.level;
    out->stats.star_pairs = (uint64_t)G - n;
    for (int k = 0; k < 5; k++) out->stats.cand_op[k] = hr.s.cand_op[k];
    out->stats.bytes_d2h = sizeof I + sizeof(SolveState) + tree_bytes;

    rei_status result;
    switch (hr.s.status) {
    case ST_FOUND: result = REI_OK; break;
    case ST_NOT_FOUND: result = REI_NOT_FOUND; break;
    case ST_OOM: result = REI_OOM; break;
    case ST_TIMEOUT: result = REI_ETIMEOUT; break;
    default: result = REI_ECUDA; break;
    }
    out->status = result;
    if (result != REI_OK) return result;
    // the outcome stays in out->status; a buffer too small for the answer is
    // reported by the return value (needed sizes written back), as in
    // rei_solve_problem
    out->cost = hr.s.ans_cost;
    const uint32_t ntok = hr.s.tree_len;
    out->tree_len = 2ull * ntok;
    rei_status ws = REI_OK;
    if (out->tree) {
        if (out->tree_cap >= out->tree_len) memcpy(out->tree, hr.tree, out->tree_len);
        else ws = REI_EBUFSZ;
    }
    out->regex_len = format_noalloc(hr.tree, ntok, p->alphabet, out->regex, out->regex ? out->regex_cap : 0);
    if (out->regex && out->regex_cap < out->regex_len + 1) ws = REI_EBUFSZ;
    else if (!out->regex && out->regex_cap) ws = REI_EINVAL;
    return ws;
}
