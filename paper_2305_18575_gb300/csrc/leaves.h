// leaves.h -- the search's leaves from a problem's costs (host side, internal).
//
// Every alphabet symbol is a leaf of the search at the level of its cost
// (Alg. 1 seeds the symbols; Sec. 3 allows different costs for different
// symbols).  The job lists the symbols ordered by (cost, alphabet order) with
// their costs, so that a level's leaves are one contiguous range, and the
// cheapest cost, below which no expression exists.
#pragma once
#include <cstdint>
#include <cstring>

#include "rei_dev.cuh"

namespace rei {

// 0 when every given per-symbol cost is >= 1 (or none are given)
inline int check_sym_costs(const rei_problem *p) {
    if (!p->sym_costs) return 0;
    for (uint32_t a = 0; a < p->n_sym; a++)
        if (p->sym_costs[a] < 1) return 1;
    return 0;
}

// fill cmin, leaf_sym[], leaf_cost[] of a job (n_sym <= 256)
inline void fill_leaves(const rei_problem *p, uint32_t *cmin, uint16_t *leaf_cost, uint8_t *leaf_sym) {
    const uint32_t n = p->n_sym;
    uint32_t cost[256];
    for (uint32_t a = 0; a < n; a++) {
        const uint32_t c = p->sym_costs ? p->sym_costs[a] : p->costs.c_sym;
        cost[a] = c > REI_MAX_COST ? REI_MAX_COST + 1 : c;
    }
    // stable insertion by cost: equal costs keep alphabet order
    uint32_t m = 0;
    for (uint32_t a = 0; a < n; a++) {
        uint32_t i = m++;
        while (i > 0 && leaf_cost[i - 1] > cost[a]) {
            leaf_cost[i] = leaf_cost[i - 1];
            leaf_sym[i] = leaf_sym[i - 1];
            i--;
        }
        leaf_cost[i] = (uint16_t)cost[a];
        leaf_sym[i] = (uint8_t)a;
    }
    *cmin = n ? leaf_cost[0] : p->costs.c_sym;
}

}  // namespace rei
