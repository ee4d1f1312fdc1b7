// Two-level blocking (Sec. III-B: the block is sized by the last-level
// cache; here GB300's L2).  Consecutive register-stage tile passes whose tile
// qubits together lie inside a block of 2^l amplitudes run as one launch,
// block by block: pass p of block b only reads amplitudes of block b, all of
// which pass p-1 of block b wrote moments earlier, so between the group's
// first read and last write the block moves through L2, not HBM.
#pragma once

#include <cstddef>
#include <cstdint>
#include <string>
#include <vector>

#include "plan.h"

namespace sv {

constexpr int kMaxGroupPasses = 4;

struct L2Group {
    int first = 0, count = 0;    // passes [first, first + count) of the plan
    int l = 0;                   // block qubits: a block holds 2^l amplitudes
    uint64_t bmask = 0;          // physical qubits inside a block (l bits)
    int lag = 1;                 // steps between pass p and pass p + 1 of one block
    int chunk_log = 0;           // a claim takes 2^chunk_log consecutive tiles of a segment
    // the launch's work in claim order, one entry per (block, pass), each
    // covering the 2^(l - k) tiles of that pass inside that block:
    // (block << 3) | pass.  Steps s = 0, 1, ...: pass p of block s - p * lag.
    std::vector<uint32_t> segs;
};

// Default block qubits for an L2 of `l2_bytes` and amplitudes of
// `amp_bytes`: the largest l with 2^l * amp_bytes <= l2_bytes / 8 (room for
// the blocks in flight between a block's passes, see lag_for).
int l2_default_qubits(size_t l2_bytes, size_t amp_bytes);

// Steps between consecutive passes of one block, so that when a CTA claims
// pass p of block b, the (resident, persistent) grid of `grid` CTAs, each
// holding up to two claims of `chunk` tiles, has almost surely finished pass
// p - 1 of block b: about 2.5 grids of claims lie between them in claim order.
int lag_for(int npass, int tiles_per_block, int grid, int chunk);

// Groups of at least two consecutive passes with eligible[i] (the pass runs
// on the register-stage kernel with tiles of 2^k amplitudes), no remap or
// general-set step before any pass but the first, and at most l_cap qubits in
// the union of their tile qubits.  The block is that union padded with the
// lowest other physical qubits up to min(l_cap, n) qubits.  A claim takes
// `chunk` tiles (at most a segment's).  Returns "" or why no group can be
// formed at all (an argument outside its range).
std::string form_l2_groups(const Plan &plan, const std::vector<char> &eligible, int n, int k,
                           int l_cap, int grid, int chunk, std::vector<L2Group> *out);

}  // namespace sv
