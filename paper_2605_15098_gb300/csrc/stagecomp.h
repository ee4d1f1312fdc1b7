// Compiled register-stage programme of one tile pass (complex64).
#pragma once

#include <string>
#include <vector>

#include "plan.h"
#include "tileprog.h"

namespace sv {

struct T2Pass {
    int k = 0, c = 0;
    int slot_phys[kMaxTileQubits] = {};
    uint64_t gmask = 0;
    int ngates = 0;
    int nruns = 0;
    int n_h = 0;                    // unnormalised Hadamards (2^(-n_h/2) at the end)
    std::vector<T2Ins> ins;
    std::vector<T2Stage> stages;
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
};

// Compile a tile pass; returns "" on success or the reason the pass cannot
// use the register-stage kernel (it then runs on the generic tile kernel).
std::string compile_t2(const TilePass &tp, T2Pass *out, bool fused = false);

}  // namespace sv
