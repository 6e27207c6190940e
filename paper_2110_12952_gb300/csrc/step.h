// step.h -- shared definitions of the compact step kernel and its
// multi-instance (batched) launch (internal; not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "handle.h"

namespace fr {

// A life-like rule: bit c of birth/survive decides a dead/live cell with c
// live neighbours; lut holds the same rule as byte tables for 4-cell look-ups
// (see rule4 in step.cu).
struct Rule {
    uint32_t birth, survive;
    uint32_t lut[4];
    uint32_t lut_sparse[2];   // for cells with at most 6 member neighbours (rule4_sparse)
};

void make_rule(uint32_t birth, uint32_t survive, Rule *r);

// One instance of a multi-instance launch.  Generation j (1-based) writes
// `odd_dst` when j is odd and `even_dst` when j is even; it reads `first` when
// j = 1 and otherwise the buffer generation j - 1 wrote.
struct InstDesc {
    const uint8_t *first;
    uint8_t *odd_dst;
    uint8_t *even_dst;
    const int32_t *nbr;   // the instance's neighbour-tile table
    int64_t cells;        // k^r
    int64_t tile0;        // first tile of the instance in the launch's tile list
    Rule rule;
};

// Launch one generation (`gen`, 1-based within the tick) of the first
// `ninst` instances of `descs`, all of which share the plan of `cls` (same
// fractal and tile depth).  `tile_inst[t]` is the instance of launch tile t;
// `total` is the tile count of those ninst instances.
int launch_step_multi(const fractal *cls, const InstDesc *descs, const int32_t *tile_inst,
                      int ninst, int64_t total, int gen, cudaStream_t st);

}  // namespace fr
