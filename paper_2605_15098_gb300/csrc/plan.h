// Tile-pass programme: the plan the partitioned path executes.
//
// Sec. III-B of arxiv 2605.15098 splits the qubits into local ones (their
// amplitudes lie inside one block) and global ones, defers gates on local
// qubits and applies all deferred gates to one block before moving to the
// next, brings a global target qubit local before it is used, and decides a
// gate whose global qubit is only a control per block from the block index.
// Here a "block" is a shared-memory tile of 2^k amplitudes: the k local
// qubits of a pass are the c lowest physical bits (one contiguous chunk of
// 2^c amplitudes, the unit of a bulk copy) plus k - c further physical bits
// chosen per pass, so a global target is brought local by gathering its
// chunks into the tile instead of moving amplitudes in a separate SWAP sweep.
//
// The paper's own scheme is kept as an option (PlanOptions::paper): the
// local qubits are always the k lowest physical bits (one contiguous block),
// and a gate whose target is global is preceded by a remap pass that
// exchanges it with the least recently used local qubit.
#pragma once

#include <cstdint>
#include <string>
#include <utility>
#include <vector>

#include "sv.h"

namespace sv {

constexpr int kMaxTileQubits = 14;

enum TileOpType : int32_t {
    TOP_GATE = 0,   // 2x2 on local slot `slot`
    TOP_GATE_CL,    // ... when local slot `cslot` is 1
    TOP_GATE_CG,    // ... when global physical bit `cbit` of the tile is 1
    TOP_DIAG,       // merged diagonal run: terms [tb, te)
    TOP_SWAP,       // exchange local slots `slot` and `cslot`
    TOP_H,          // Hadamard on `slot` (real matrix)
    TOP_X           // X on `slot` (pure exchange)
};

// One step of a tile programme (96 bytes, read by the kernel).
struct TileOp {
    int32_t type;
    int32_t slot;
    int32_t cslot;
    int32_t cbit;
    int32_t tb, te;
    int32_t pad[2];
    double m[8];  // U11 re, im, U12 re, im, U21 re, im, U22 re, im
};

enum TermKind : int32_t {
    TERM_L = 0,    // x_a                  (a local slot)
    TERM_LL = 1,   // x_a x_b              (a, b local slots)
    TERM_G = 2,    // x_g                  (g global physical bit)
    TERM_LG = 3,   // x_a x_g
    TERM_GG = 4    // x_g x_h
};

// One term of a diagonal run's phase polynomial: the amplitude picks up
// theta (a fraction of a turn in units of 2^-64) when the named bits are 1.
struct PhaseTerm {
    int32_t kind;
    int32_t a, b;
    int32_t pad;
    uint64_t theta;
};

struct TilePass {
    int k = 0, c = 0;
    int slot_phys[kMaxTileQubits];  // physical bit of local slot s
    uint64_t gmask = 0;             // physical bits outside the tile
    int ngates = 0;                 // circuit gates the pass applies
    // Physical bit pairs (local, global) exchanged by a remap pass before
    // this pass runs: amplitude x moves to x with each pair's bits swapped.
    // The pairs are disjoint.
    std::vector<std::pair<int, int>> remap_before;
    std::vector<TileOp> ops;
    std::vector<PhaseTerm> terms;
    // A gate of the general set (MCU, U2Q with its rows, MEASURE), physical
    // qubits: the step runs it on the per-gate path; ops and terms are empty.
    std::vector<sv_gate> general;
};

struct PlanOptions {
    int n = 0;
    int k = 0, c = 0;
    bool merge_diag = true;
    bool relabel = true;
    bool paper = false;  // explicit LRU remaps, tile = the k lowest physical bits
    bool split_u3 = false;  // U3 as P(phi) RY(theta) P(lambda): phases join the diagonal runs
    bool late_diag = true;  // diagonal gates move to the pass of their first successor
    bool search = true;     // refine each pass's local qubits by local search (the greedy
                            // plan is kept when it has fewer passes)
    int first_c = 0;        // chunk qubits of the list's first pass (0: c); SV_FLAG_NARROW_FIRST
};

// Planner options of a configuration (library defaults filled in).
PlanOptions plan_options(int n, sv_dtype dt, const sv_config &cfg);

struct Plan {
    std::vector<TilePass> passes;
    int relabels = 0;
    int remaps = 0;  // remap passes (pairs exchanged in one sweep count once)
};

// Kernel of one tile pass.
enum PassKernel : int8_t { PK_GENERIC = 0, PK_T2 = 1, PK_T3 = 2 };

// A plan fixed by the learned planner: planner options and, per pass of the
// resulting plan, the kernel to run it on.
struct PlanOverride {
    PlanOptions opt;
    std::vector<int8_t> kernel;
};

// Build the programme; phys (logical -> physical, n entries) is updated by
// SWAP relabelling.  Gates must be valid.  A gate of the general set splits
// the list: the gates before it are planned, the gate becomes a step of its
// own (TilePass::general), and the rest is planned from the qubit map then.
// Returns an empty string on success.
std::string build_plan(const std::vector<sv_gate> &gates, const PlanOptions &opt, int *phys,
                       Plan *out);

}  // namespace sv
