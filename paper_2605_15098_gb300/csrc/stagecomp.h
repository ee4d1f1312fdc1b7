// Compiled register-stage programme of one tile pass (complex64).
#pragma once

#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "plan.h"
#include "tileprog.h"

namespace sv {

struct T2Pass {
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
    std::vector<T2Factor> factors;
    std::vector<uint32_t> stat;     // per-thread static phases: row r is stat[r*256 .. r*256+255]
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
    const T2Factor *fac;
    const uint32_t *stat;
    const T2TileTerm *tterms;
    const float *blocks;
    const T2LayoutX *layx;
    const T2Epilogue *epi;
};

// Launch parameters of one register-stage pass (device pointers).
struct T2Args {
    uint64_t gmask, ntiles;
    int c, nins, nruns, ntterms;
    int nfac, nstat;  // factor records, static phase words
    int last_stage;  // index of the last T2_STAGE instruction
    int slot_phys[kMaxTileQubits];
    const int4 *ins;       // T2Ins records
    const int4 *stages;    // T2Stage records
    const float4 *mats;    // T2Mat records (two float4 each)
    const int4 *fac;       // T2Factor records
    const uint32_t *stat;  // per-thread static phases
    const T2TileTerm *tterms;
    const float2 *tables;
    int *err;
    const T2LayoutX *layx;  // per stage (register-stage kernel)
    const T2Epilogue *epi;  // write-back offsets (register-stage kernel)
    // gen != 0: the state is the basis state |gen_basis> (physical index) and
    // is generated in registers instead of read; gen_local is its index inside
    // the tile that holds it; gen_hmask: tile bits whose leading Hadamards
    // (T2_HG) the generation includes
    int gen, gen_local;
    uint64_t gen_basis;
    uint32_t gen_hmask;
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

struct BatchArgs {
    const BatchInst *inst;
    const T2Args *passes;
    const int *order;  // processing order (largest first)
    int count;
    int *queue;
    uint64_t *out_idx;
    double *out_p;
    int *err;
    const float2 *tables;
    int need;  // gate kinds the programmes use (host side: picks the kernel instantiation)
};

// Compile a tile pass; returns "" on success or the reason the pass cannot
// use the register-stage kernel (it then runs on the generic tile kernel).
std::string compile_t2(const TilePass &tp, T2Pass *out, bool fused = false);

}  // namespace sv
