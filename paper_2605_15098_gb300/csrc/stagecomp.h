// Compiled register-stage programme of one tile pass (complex64).
#pragma once

#include <cuda_runtime.h>

#include <memory>
#include <string>
#include <vector>

#include "l2group.h"
#include "plan.h"
#include "tileprog.h"

namespace sv {

struct T2Pass {
    int format = 1;  // 1: fused kernel (k_tile3); 2: CUDA-core kernels (tileprog.h, format 2)
    int k = 0, c = 0;
    int rb = kT2RegBits, threads = kT2Threads;  // geometry (see tileprog.h)
    int slot_phys[kMaxTileQubits] = {};
    uint64_t gmask = 0;
    int ngates = 0;
    int nruns = 0;
    int n_h = 0;                    // unnormalised Hadamards (2^(-n_h/2) at the end)
    int sign_flips = 0;             // rotations run as -1 times a shear product (sign at the end)
    uint32_t gen_hmask = 0;         // tile bits of the leading Hadamards (T2_HG)
    int last_stage = -1;            // index in `ins` of the last T2_STAGE
    std::vector<T2Ins> ins;
    std::vector<T2Stage> stages;
    std::vector<T2LayoutX> layx;    // per stage, the kernel-side layout
    T2Epilogue epi{};               // write-back offsets of the final layout
    std::vector<T2Mat> mats;
    std::vector<T2Factor> factors;  // format 1
    std::vector<uint32_t> stat;     // format 1: per-thread static phases, row r = stat[r*256 ..]
    std::vector<T2Fac> fac2;        // format 2 factor applications
    std::vector<float> statc;       // format 2: static complex rows, (re, im) per thread
    std::vector<T2Slot> slots;      // format 2: tile-uniform slots
    std::vector<int32_t> soff;      // format 2: slot s's terms are sterms[soff[s] .. soff[s + 1])
    std::vector<T2SlotTerm> sterms;
    // complex128 (compile_t2v2_c128): 64-bit phases and FP64 values in place
    // of sterms, mats and statc (same record indexing: a matrix record is 8
    // doubles, a table's entry x is (re, im) at doubles 2x, 2x + 1)
    int wide = 0;
    std::vector<T2SlotTerm64> sterms64;
    std::vector<double> mats64;
    std::vector<double> statc64;
    // format 2, first pass of a plan: the variant run when the pass starts
    // from a recorded basis state (generated in registers, leading Hadamards
    // included); null when not compiled
    std::shared_ptr<T2Pass> genv;
    // the gen variant: the pass's closing scale (2^(-n_h/2), sign flips),
    // multiplied into the generated state instead of applied at the end
    double gen_scale = 1.0;
    std::vector<T2TileTerm> tterms;
    int nblocks = 0;
    std::vector<double> blocks64;   // fused: per block 2 x 32 x 32 (re, im), row = output index
    std::vector<float> blocks_dev;  // fused: per block kBlockFloats in the device layout
};

// Device copies of a compiled pass (inside the handle's programme buffer).
struct T2Device {
    const T2Ins *ins;
    const T2Stage *stages;
    const T2Mat *mats;
    const void *fac;         // T2Factor (format 1) or T2Fac (format 2) records
    const uint32_t *stat;    // format 1
    const float *statc;      // format 2
    const T2Slot *slots;     // format 2
    const int32_t *soff;     // format 2
    const T2SlotTerm *sterms;  // format 2
    const T2TileTerm *tterms;
    const float *blocks;
    const T2LayoutX *layx;
    const T2Epilogue *epi;
};

// Launch parameters of one register-stage pass in format 2 (device pointers).
struct T2Args {
    uint64_t gmask, ntiles;
    int c, nins;
    int nfac, nrows, nslots, nmats, nstages;  // factor records, static rows, slots, matrix records, stages
    int last_stage;  // index of the last T2_STAGE instruction
    int slot_phys[kMaxTileQubits];
    // the tile's physical base index: tile index bits [gs[r], gs[r] + gl[r])
    // go to physical bits gd[r].. (runs of the global bits)
    int ngr;
    int8_t gs[32], gd[32], gl[32];
    const int4 *ins;       // T2Ins records
    const int4 *stages;    // T2Stage records
    const float4 *mats;    // T2Mat records (two float4 each)
    const int4 *fac;       // T2Fac records
    const float2 *statc;   // static complex rows (threads entries each)
    const int32_t *soff;   // slot term ranges
    const T2SlotTerm *sterms;
    const float2 *tables;
    int *err;
    const T2LayoutX *layx;  // per stage
    const T2Epilogue *epi;  // write-back offsets
    // gen != 0: the state is H on the physical qubits gen_ghmask (global
    // qubits of the pass) and the tile bits gen_hmask applied to the basis
    // state |gen_basis> (physical index), generated in registers instead of
    // read; gen_local is the basis index's tile-local part; gen_val the
    // magnitude of a nonzero amplitude before the pass's closing scale (the
    // tile-bit Hadamards of the programme's own prefix are unnormalised and
    // the scale holds their 2^(-1/2); the recorded ones are in gen_val)
    int gen, gen_local;
    uint64_t gen_basis, gen_ghmask;
    uint32_t gen_hmask;
    float gen_val;
    // write-back: 0 streams the tile out (evict-first stores, the pass's
    // result goes to HBM); 1 keeps it in L2 (plain stores: the next pass of
    // an L2 block reads it)
    int keep;
    double gen_val64;  // gen_val in FP64 (complex128 kernel)
    // the tile-uniform slot values computed for every tile before the launch
    // (k_slotv: nsp values per tile, nslots rounded up to even, so that one
    // tile's values are one 16-byte-multiple bulk copy); NULL: each tile
    // computes its own
    const float2 *slotv;
    int nsp;
};

// Bytes of the per-tile slot values of a complex64 register-stage pass
// (T2Args::slotv), 0 when the pass computes them per tile: no slots, or more
// than kSlotvMaxBytes.
constexpr size_t kSlotvMaxBytes = (size_t)256 << 20;
size_t t2_slotv_bytes(const T2Pass &p, int n);

// Fill the counts, pointers and geometry of a format-2 pass (not gen,
// tables or err).
void t2_fill_args(const T2Pass &p, const T2Device &d, int n, T2Args *a);

// Re-order a pass's tile index for an L2 block of the physical qubits
// `bmask`: the low bits of the tile index run over the pass's global qubits
// inside the block, the high bits (the block index) over the qubits outside
// it.  Returns false if the runs do not fit the argument record.
bool t2_block_runs(T2Args *a, uint64_t gmask, uint64_t bmask, int n);

// One launch of an L2 block group: its passes' arguments and the claim order.
struct GroupArgs {
    T2Args pass[kMaxGroupPasses];
    const uint32_t *segs;       // (block << 3) | pass, in claim order
    uint64_t nitems;            // segments x tiles per block
    int npass, tpb_log;         // passes; log2 of a pass's tiles inside a block
    int chunk_log;              // a claim takes 2^chunk_log consecutive items
    unsigned *done;             // per (block, pass): tiles finished (zero at launch)
    unsigned long long *queue;  // next item to claim (zero at launch)
    int *err;
};

// One instance of a batch: its state, passes and read-out qubits.
struct BatchInst {
    uint64_t state_off;  // in amplitudes
    int npass, pass0;    // passes [pass0, pass0 + npass) of the batch's pass table
    int nphys;           // qubits of the stored state (>= 13)
    int m;               // read-out qubits
    int out;             // result slot
    int pos[34];         // physical bit of read-out bit j
};

// Work items of a batched launch, in claim order: x = instance, y = kind |
// (pass << 4), z = first tile, w = tiles.
enum { kBatchWhole = 0, kBatchTiles = 1, kBatchReadout = 2 };
constexpr int kBatchClaimTiles = 8;  // tiles of one claim of a split instance

struct BatchArgs {
    const BatchInst *inst;
    const T2Args *passes;
    const int4 *work;  // work items in claim order
    int nwork;
    unsigned *done;    // per pass (index into passes): tiles finished (zero at launch)
    int *queue;
    uint64_t *out_idx;
    double *out_p;
    int *err;
    const float2 *tables;
    int need;  // gate kinds the programmes use (host side: picks the kernel instantiation)
};

// Compile a tile pass; returns "" on success or the reason the pass cannot
// use the register-stage kernel (it then runs on the generic tile kernel).
// Without fused blocks the programme is in format 2 (compile_t2v2).
std::string compile_t2(const TilePass &tp, T2Pass *out, bool fused = false);

// Format 2; `gen`: the variant for a pass that starts from a recorded basis
// state, which it generates in registers (no shared-memory read of its first
// stage; the leading Hadamards are part of the generated state).
std::string compile_t2v2(const TilePass &tp, T2Pass *out, bool gen);

// The same programme for the complex128 register-stage kernel (k_tile2d):
// 64-bit phases, FP64 matrices, tables and rows; 2^13-amplitude tiles.
std::string compile_t2v2_c128(const TilePass &tp, T2Pass *out, bool gen);

}  // namespace sv
