// Register-stage tile programme (complex64 tile kernel).
//
// A tile pass (see plan.h) is compiled into stages.  In a stage every thread
// of the CTA holds 2^RB amplitudes of the 2^13-amplitude tile in registers:
// register bit 0 is always tile bit 0 (two neighbouring amplitudes form one
// 16-byte shared-memory vector), register bits 1..RB-1 are tile bits chosen
// per stage, lane bits 0..2 are tile bits 1..3 (so that the eight lanes of a
// quarter-warp read one 128-byte row: conflict-free), lane bits 3..4 and the
// warp bits are the remaining tile bits.  A gate on a register bit is
// thread-local arithmetic; a gate on a lane bit exchanges amplitudes with
// warp shuffles; a stage change stores the tile to shared memory and reloads
// it in the next stage's layout.
//
// A merged diagonal run multiplies amplitude x by e^{2 pi i phi(x) / 2^32}
// with phi a quadratic polynomial over the bits of x (Sec. III-B's rule that
// global qubits are constants of a block, applied to every diagonal gate).
// It is compiled into factor applications: each application multiplies the
// amplitudes whose register bits include `mask` by one complex factor, which
// is either a constant (generated in FP64 on the host) or e^{2 pi i u / 2^32}
// for a per-thread integer phase u, read from FP64-generated tables.  The
// part of u that does not depend on the tile is tabulated per thread on the
// host; the kernel adds the tile's global-qubit contributions.
#pragma once

#include <cstdint>

namespace sv {

constexpr int kT2Qubits = 13;   // tile: 2^13 complex64 amplitudes (64 KiB)
constexpr int kT2WideQubits = 14;  // wide tile of the CUDA-core kernel: 2^14 amplitudes,
                                   // 512 threads, one CTA per SM
constexpr int kT2MaxQubits = 14;
// The programme format is written for a geometry: register bits RB, 5 lane
// bits and 13 - RB - 5 warp bits.  The CUDA-core kernels (k_tile2, k_batch)
// and the fused tensor-core kernel (k_tile3) both hold 32 amplitudes per
// thread in 256 threads (5 register bits, the index of a 32x32 block for the
// fused kernel).  A 16-amplitude, 512-thread geometry for the CUDA-core
// kernels was measured slower: the per-thread work of a diagonal factor
// (its record and its table lookups) is then spread over half as many
// amplitudes.
constexpr int kT2Threads = 256;
constexpr int kT2RegBits = 5;
constexpr int kT2WarpBits = 3;
constexpr int kT3Threads = 256;
constexpr int kT3RegBits = 5;
constexpr int kT3WarpBits = 3;
constexpr int kMaxRegBits = 5;
constexpr int kMaxThreadBits = 9;  // 5 lane bits + up to 4 warp bits
constexpr int kT2MaxRuns = 64;  // diagonal runs per pass with per-tile data
// The register-stage kernel keeps a pass's programme in shared memory.
constexpr int kT2SmemIns = 128;      // instructions
constexpr int kT2SmemFactors = 128;  // factor applications
constexpr int kT2SmemStatRows = 16;  // per-thread static phase rows (later rows stay in global memory)

enum T2Op : int32_t {
    T2_STAGE = 0,  // switch layout (stage record `aux`), through shared memory
    T2_GATE = 1,   // general 2x2 (matrix record `aux`) on the target
    T2_H = 2,      // unnormalised Hadamard [[1,1],[1,-1]] on the target
    T2_X = 3,      // X on the target
    T2_DIAG = 4,   // factor applications [e0, e1)
    T2_SCALE = 5,  // multiply every amplitude by hi + lo (matrix record `aux`: m[0], m[1])
    T2_BLOCK = 6,  // fused kernel: 32x32 block `aux` on the register bits (tensor cores)
    T2_RGATE = 7,  // real 2x2 (matrix record `aux`, imaginary parts zero): half the arithmetic
    T2_ROT = 8,    // uncontrolled register-bit rotation as three shears (record: t, s)
    T2_HPH = 9,    // diagonal run [e0, e1) then H on register bit idx, in one sweep:
                   // the run is the identity where bit idx is 0, and holds at
                   // most one phase table and one per-thread factor on bit idx
                   // (no dynamic thread bits); with ccls == kT2HphDirect the
                   // step also names them: aux = (row + 1) << 16 | (table + 1)
                   // (0 = none), cidx = the factor's slot (-1 = none)
    T2_HG = 10     // H of the programme's leading Hadamards (distinct tile bits, before
                   // any other step): a pass that generates a basis state generates
                   // the state after them and skips them; otherwise an H
};

// Fused blocks: a 32x32 complex matrix U on the register index (bit j of the
// index = register bit j) multiplies each thread's 32 amplitudes.  On the
// device a block is 4 x 32 x 32 floats: Re U and Im U rounded to TF32 (hi),
// then the remainders (lo), each in the K-major, no-swizzle operand layout of
// the tensor-core B operand: element (n, k) at byte
//   (n / 8) * 1024 + (k / 4) * 128 + (n % 8) * 16 + (k % 4) * 4.
constexpr int kBlockFloats = 4 * 32 * 32;
constexpr int kMaxBlocks = 4;  // shared-memory block slots; more blocks stream through them

// Handler of a gate instruction, set by the stage compiler so that the
// register-stage kernel dispatches a gate with one switch:
// kT2Handler + 8 * kind + slot, kind 0..5 = H, X, real 2x2, shear rotation,
// general 2x2, phased H (T2_HPH); slot 0..4 = register bit (uncontrolled),
// 5 = lane bit (uncontrolled), 6 = lane bit with a thread control, 7 = any
// other control.
// Codes stay below 256: the kernel takes the field's high byte, zero, as the
// opaque all-ones mask of its gate code.
constexpr int kT2Handler = 16;

enum T2Class : int32_t { T2C_NONE = 0, T2C_REG = 1, T2C_LANE = 2, T2C_THREAD = 3, T2C_GLOBAL = 4 };
// control-class field of a T2_HPH step whose table, row and slot are in the step
constexpr int8_t kT2HphDirect = 0x40;
// The same, for a step on register bit j whose table depends only on
// register bits 0..j-1 (j = 1..3 in complex64 programmes, where bit 0 is the
// element of a packed pair; j = 0..3 in complex128 ones).  The inverse QFT's
// phases on a qubit come from the qubits it transformed before, often
// register bits of the same stage.  The distinct products of the thread
// factor and the table (2^(j-1) packed, 2^j in FP64) are formed once, and
// each pair takes one of them.  A kernel that does not know the code reads
// the run from its factor records.
constexpr int8_t kT2HphShared = 0x41;

// One programme step, 16 bytes (one vector load in the kernel).
struct T2Ins {
    int8_t op;
    int8_t cls;    // target class: T2C_REG (idx = register bit) or T2C_LANE (idx = lane bit)
    int8_t idx;
    int8_t ccls;   // control class: NONE, REG (register bit), THREAD (bit of threadIdx.x), GLOBAL
    int16_t cidx;  // control: register bit, thread bit, or physical bit
    int16_t hd;    // gates: handler code (kT2Handler), 0 otherwise
    int16_t e0, e1;  // T2_DIAG: factor applications
    int32_t aux;     // T2_STAGE: stage record; T2_GATE / T2_SCALE: matrix record
};

// Layout of a stage: tile bit of register bits 0..4, lane bits 0..4 (thread
// bits 0..4) and warp bits 0..2 (thread bits 5..7).
struct T2Stage {
    int8_t tb[16];
};

// Kernel-side form of a stage layout, computed on the host: the tile offset
// (in amplitudes) of the lane bits (lo, indexed by tid & 31) and the warp bits
// (hi, indexed by tid >> 5), and of register bits 1..  A thread's packed pair q
// sits at tile offset lo + hi + sum over the set bits j of q of s[j].
// The p* fields give the same positions in the swizzled shared-memory order
// of a stage change (format 2, below): the float4 slot of packed pair q is
// plo ^ phi ^ (xor over the set bits j of q of ps[j]).
struct T2LayoutX {
    uint16_t lo[32];  // lane bits (tid & 31)
    uint16_t hi[16];  // warp bits (tid >> 5)
    int32_t s[4];     // register bits 1.. (unused ones 0)
    uint16_t plo[32];
    uint16_t phi[16];
    int32_t ps[4];
};

// ---------------------------------------------------------------- format 2
// The complex64 register-stage kernel (k_tile2, k_batch) runs programmes in
// format 2, compiled by compile_t2 without fused blocks:
//  * every gate target is a register bit of its stage (no shuffle gates): a
//    target outside the register bits starts a new stage;
//  * a stage change stores the tile to shared memory and loads it back in the
//    new layout, both in a swizzled order: the 16-byte vector of float4 index
//    f (tile index >> 1) lives at slot swz(f) = f ^ fold(f), where fold(f)
//    XORs f's bits 3.., three at a time, onto bits 0..2.  A quarter-warp's
//    eight lanes then hit eight distinct bank groups whenever lane bits 0..2
//    are tile bits whose float4 bits (tile bit - 1) differ mod 3, which the
//    stage compiler arranges;
//  * the first stage of a pass that reads its tile takes it from the bulk
//    copies' linear order, so its lane bits 0..2 are tile bits 1..3; a pass
//    that generates a recorded basis state has a variant of its own, without
//    that rule and without the leading Hadamards (they are part of the
//    generated state);
//  * diagonal runs compile to T2Fac records: a per-thread factor is a static
//    complex row (one FP32 e^{i phi} per thread, formed in FP64 on the host)
//    times tile-uniform slot values (e^{i phi} of the tile's global-qubit
//    terms, formed once per tile from FP64-generated tables), times one slot
//    per dynamic thread bit; constants become 32-entry tables as before.
inline int swz_fold(int f) { return ((f >> 3) ^ (f >> 6) ^ (f >> 9) ^ (f >> 12)) & 7; }
inline int swz(int f) { return f ^ swz_fold(f); }

// One factor application of format 2, 16 bytes.
//   w0: as T2Factor (bits 0..7 register mask, bit 8 per-thread, bits 10..13
//       thread predicate of a table, bits 19..27 dynamic thread bits, bit 28
//       table); the other bits 0
//   slot: tile-uniform slot multiplied into a per-thread factor, -1 = none
//   dslot: slot of the lowest dynamic thread bit; the k-th lowest set bit of
//       the dynamic mask uses dslot + k
//   row: per-thread factor: static complex row (-1 = none); table: first
//       matrix record of the 32-entry table
struct T2Fac {
    uint32_t w0;
    int16_t slot, dslot;
    int32_t row;
    int32_t pad;
};

// A tile-uniform slot: e^{2 pi i (lin[i0] + lin[i1]) / 2^32} for the per-tile
// phase words lin[run * 16 + tb] (tb = tile bit; 15 = the run's constant);
// i1 = -1: lin[i0] alone.
struct T2Slot {
    int16_t i0, i1;
};
constexpr int kT2MaxSlots = 256;
constexpr int kT2SmemMats = 384;     // matrix records kept in shared memory
constexpr int kT2SmemRows = 8;       // static complex rows kept in shared memory
constexpr int kT2SmemStages = 16;    // stage layouts kept in shared memory

// One global-qubit term of a slot, for the kernel: theta (turns / 2^32) when
// physical bits g0 (and g1, if >= 0) of the tile are set.  The terms of slot
// s are sterms[soff[s] .. soff[s + 1]): those of its phase words i0 and i1.
struct T2SlotTerm {
    int16_t g0, g1;
    uint32_t theta;
};
// The same with a 64-bit phase (complex128 kernel).
struct T2SlotTerm64 {
    int16_t g0, g1;
    int32_t pad;
    uint64_t theta;
};

// Handler codes of the non-gate steps (format 2), in the same field as the
// gate handlers: the kernel dispatches every step with one switch.
constexpr int kT2HdStage = 1, kT2HdScale = 2, kT2HdDiag = 3;

// Write-back offsets of the final layout in the global state (amplitudes),
// relative to the tile's base: lane bits, warp bits and register bits 1..
struct T2Epilogue {
    uint64_t glo[32];
    uint64_t ghi[16];
    uint64_t g[4];
};

struct T2Mat {
    float m[8];  // U11 re, im, U12 re, im, U21 re, im, U22 re, im
};

// One factor application, 16 bytes.
//   w0 bits 0..7:   register-bit mask the amplitude must have set (popcount <= 2)
//   w0 bit 8:       1 = per-thread phase, 0 = constant (c0, c1)
//   w0 bit 9:       phase += cst[run] (the tile's global-only part)
//   w0 bits 10..13: constant factors only: 1 + thread bit t; only threads with
//                   bit t set apply the factor (0 = every thread)
//   w0 bits 14..18: 1 + tile bit whose per-tile coefficient lin[run][tb] is added, 0 = none
//   w0 bits 19..27: thread bits t whose per-tile coefficient lin[run][tile bit of t] is added
//                   when thread bit t is set
//   w0 bit 28:      phase table: the amplitude with register index x (bits of
//                   the register bits) is multiplied by entry x of the 32-entry
//                   constant table starting at matrix record c0 (as an int), which
//                   holds, per packed pair q, (re[2q], re[2q+1], im[2q], im[2q+1]);
//                   bits 10..13 as for a constant, mask bits 0
// A per-thread phase starts from row c0 of the host table of per-thread
// static phases (one entry per thread of the geometry).
constexpr int kFacLinShift = 14;
constexpr int kFacDynShift = 19;
constexpr uint32_t kFacTable = 1u << 28;
struct T2Factor {
    int32_t w0;
    int32_t run;
    float c0, c1;
};

// Global-dependent term, applied once per tile: adds theta to lin[run][tb]
// (tb >= 0) or to cst[run] (tb < 0) when physical bits g0 (and g1, if >= 0)
// of the tile are set.
struct T2TileTerm {
    int32_t run, tb, g0, g1;
    uint32_t theta;
    int32_t pad;
};

}  // namespace sv
