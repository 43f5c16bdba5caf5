// args.h -- argument checks of a packed problem (host side, internal).
//
// The one set of rules every entry point applies before it touches a device:
// rei_solve / rei_solve_problem / rei_stage / rei_solve_batch /
// rei_server_submit (host.cu) and rei_solve_noalloc (noalloc.cu).  A problem
// that fails them is answered REI_EINVAL without any launch, so a bad argument
// never reaches a kernel as a bad pointer or size.
#pragma once
#include <cstdint>

#include "leaves.h"

namespace rei {

// REI_OK, or REI_EINVAL when: the alphabet is missing, empty, longer than 256
// or repeats a symbol; a cost is 0 or above REI_MAX_COST; max_cost is above
// REI_MAX_COST; a per-symbol cost is 0; there are more than 2^24 strings; the
// strings have no offsets, or bytes are missing while some string is not
// empty; host offsets do not start at 0, decrease, or give a string longer
// than REI_MAX_STRLEN.  (Symbols, overlaps and |ic| are checked by the
// staging kernel, which reads the bytes.)
inline rei_status check_problem(const rei_problem *p) {
    if (!p || !p->alphabet || p->n_sym == 0 || p->n_sym > 256) return REI_EINVAL;
    const uint32_t c[5] = {p->costs.c_sym, p->costs.c_opt, p->costs.c_star, p->costs.c_cat, p->costs.c_alt};
    for (uint32_t v : c)
        if (v < 1 || v > REI_MAX_COST) return REI_EINVAL;
    if (p->max_cost > REI_MAX_COST) return REI_EINVAL;
    if (check_sym_costs(p)) return REI_EINVAL;
    bool seen[256] = {};
    for (uint32_t i = 0; i < p->n_sym; i++) {
        if (seen[p->alphabet[i]]) return REI_EINVAL;
        seen[p->alphabet[i]] = true;
    }
    const uint64_t n_str = (uint64_t)p->n_pos + p->n_neg;
    if (n_str > (1u << 24)) return REI_EINVAL;
    if (!n_str) return REI_OK;
    if (!p->offsets) return REI_EINVAL;
    if (p->flags & REI_F_DEVICE_INPUT) {
        // device offsets are checked by the staging kernel (start at 0, never
        // decrease, end at total_bytes)
        if (!p->bytes && p->total_bytes) return REI_EINVAL;
        if (p->total_bytes > 0xFFFFFFF0ull) return REI_EINVAL;
        return REI_OK;
    }
    if (p->offsets[0] != 0) return REI_EINVAL;
    for (uint64_t k = 0; k < n_str; k++) {
        if (p->offsets[k + 1] < p->offsets[k]) return REI_EINVAL;
        if (p->offsets[k + 1] - p->offsets[k] > REI_MAX_STRLEN) return REI_EINVAL;
    }
    if (!p->bytes && p->offsets[n_str]) return REI_EINVAL;
    return REI_OK;
}

}  // namespace rei
