// Register-stage tile kernel (complex64, tiles of 2^13 amplitudes), running
// programmes in format 2 (tileprog.h).
//
// Per tile (persistent grid, two CTAs per SM, 256 threads each, 32 amplitudes per thread):
//   1. one warp issues 2^(13-c) bulk copies (TMA, cp.async.bulk) of the
//      tile's contiguous 2^c-amplitude chunks into shared memory, completing
//      on an mbarrier;
//   2. the pass's per-tile diagonal data (global-qubit contributions, which
//      are constants of the tile: Sec. III-B of arxiv 2605.15098) is summed
//      as integer phases while the copies are in flight, then turned into the
//      tile's complex slot values;
//   3. the stage programme runs: each thread holds 32 amplitudes as 16
//      packed pairs (re and im of two neighbouring amplitudes); every gate
//      targets a register bit (packed f32x2 arithmetic); a stage change goes
//      through shared memory in the swizzled order; once the last stage
//      change has read shared memory, the next tile's copies start;
//   4. each thread writes its amplitudes straight from registers to the
//      global state (16-byte streaming stores).
// Hadamards are applied unnormalised ([[1,1],[1,-1]]) and the pass ends with
// one multiplication by 2^(-h/2), exact for even h, so the norm carries no
// bias from a rounded 1/sqrt(2).
#include <algorithm>

#include "common.h"
#include "plan.h"
#include "stagecomp.h"
#include "tiledev.cuh"
#include "tileprog.h"

namespace sv {
namespace {

using namespace tiledev;

constexpr int kTabN = 256;               // four levels of 2^8 entries
constexpr int kNP2 = 1 << (kT2RegBits - 1);  // packed pairs per thread (32 amplitudes)
constexpr int kTabEntries = 4 * kTabN;

// Shared-memory layout of a CTA for tiles of 2^K amplitudes (K = 13: 256
// threads, two CTAs per SM; K = 14: 512 threads, one CTA per SM).  The CTA
// copies the pass's programme into shared memory once.
template <int K>
struct Geo {
    static constexpr int kThreads = 1 << (K - kT2RegBits);
    static constexpr int kWarps = kThreads / 32;
    static constexpr uint32_t kTileBytes = 8u << K;
    static constexpr size_t kOffTab = kTileBytes;
    static constexpr size_t kOffRows = kOffTab + (size_t)kTabEntries * 8;
    static constexpr size_t kOffMats = kOffRows + (size_t)kT2SmemRows * kThreads * 8;
    static constexpr size_t kOffFac = kOffMats + (size_t)kT2SmemMats * sizeof(T2Mat);
    static constexpr size_t kOffIns = kOffFac + (size_t)kT2SmemFactors * 16;
    static constexpr size_t kOffSlotc = kOffIns + (size_t)kT2SmemIns * 16;  // two buffers
    static constexpr size_t kOffLay = kOffSlotc + 2 * (size_t)kT2MaxSlots * 8;
    static constexpr size_t kOffEpi = kOffLay + (size_t)kT2SmemStages * sizeof(T2LayoutX);
    static constexpr size_t kOffOnes = kOffEpi + sizeof(T2Epilogue);  // the identity phase table
    static constexpr size_t kOffBar = kOffOnes + 16 * 16;
    // a claimed work item (L2 block and batched kernels).  No kernel here
    // declares static shared memory: it would sit before the 1024-byte
    // aligned dynamic area and push two CTAs past the SM's shared memory.
    static constexpr size_t kOffClaim = kOffBar + 16;
    // the current pass's arguments (L2 block kernel)
    static constexpr size_t kOffArgs = kOffClaim + 16;
    static constexpr size_t kSmemBytes = kOffArgs + ((sizeof(T2Args) + 15) / 16) * 16;
};
using G13 = Geo<13>;
constexpr size_t kSmemBytes = G13::kSmemBytes;
static_assert(2 * (G13::kSmemBytes + 1024) <= 228 * 1024, "two CTAs per SM");
static_assert(Geo<14>::kSmemBytes <= 227 * 1024, "one CTA per SM");
static_assert(sizeof(T2LayoutX) % 16 == 0 && sizeof(T2Epilogue) % 16 == 0, "16-byte records");

// ---------------------------------------------------------------- the kernel
// Run a pass's programme (in shared memory) on the tile.  The first stage
// reads the tile from shared memory (interleaved complex64, linear tile
// order), or generates the recorded basis state.  After the last stage change
// has read shared memory, `hook()` runs (the callers start the next tile's
// bulk copies there).  The result goes straight from registers to the global
// state, at the offsets of the final layout's write-back record.

extern __shared__ __align__(1024) unsigned char t2_dyn_smem[];

// Float4 index (amplitude pair) of packed pair q in a stage layout, linear
// tile order, for thread tid, from the host-computed layout record.
struct Layout2 {
    int bt, s1, s2, s3, s4;
    __device__ Layout2(const T2LayoutX *x, int tid) {
        bt = (int)x->lo[tid & 31] + (int)x->hi[tid >> 5];
        const int4 sv = *reinterpret_cast<const int4 *>(x->s);
        s1 = sv.x;
        s2 = sv.y;
        s3 = sv.z;
        s4 = sv.w;
    }
    __device__ int idx(int q) const {
        return (bt + ((q & 1) ? s1 : 0) + ((q & 2) ? s2 : 0) + ((q & 4) ? s3 : 0) +
                ((q & 8) ? s4 : 0)) >> 1;
    }
};

// The same positions in the swizzled order of a stage change (tileprog.h).
struct LayoutS {
    int b, p1, p2, p3, p4;
    __device__ LayoutS(const T2LayoutX *x, int tid) {
        b = (int)x->plo[tid & 31] ^ (int)x->phi[tid >> 5];
        const int4 pv = *reinterpret_cast<const int4 *>(x->ps);
        p1 = pv.x;
        p2 = pv.y;
        p3 = pv.z;
        p4 = pv.w;
    }
    __device__ int idx(int q) const {
        return b ^ ((q & 1) ? p1 : 0) ^ ((q & 2) ? p2 : 0) ^ ((q & 4) ? p3 : 0) ^ ((q & 8) ? p4 : 0);
    }
};

// Gate kinds an instantiation carries besides H and the diagonal runs (the
// host launches the smallest one that covers a pass's programme: every gate
// path in the loop costs registers and instructions in all the others).
constexpr int kFeatX = 1, kFeatR = 2, kFeatU = 4, kFeatAll = 7;

// Gate KIND (0..4: H, X, real 2x2, shear rotation, general 2x2) on register
// bit SLOT (0..4).  Kinds outside the instantiation's set F compile to
// nothing: the host never launches them there.
template <int F, int KIND, int SLOT, int NP>
__device__ __forceinline__ void run_gate(RegsN<NP> &r, const float4 *mrec, uint32_t qm) {
    constexpr int need = KIND == 0 ? 0 : KIND == 1 ? kFeatX : KIND == 4 ? kFeatU : kFeatR;
    if constexpr ((need & F) != need) {
        return;
    } else {
        float m[8] = {};
        if constexpr (KIND >= 2) {
            const float4 m0 = mrec[0], m1 = mrec[1];
            m[0] = m0.x; m[1] = m0.y; m[2] = m0.z; m[3] = m0.w;
            m[4] = m1.x; m[5] = m1.y; m[6] = m1.z; m[7] = m1.w;
        }
        if constexpr (KIND == 0) reg_h2<SLOT>(r, qm);
        else if constexpr (KIND == 1) reg_x2<SLOT>(r, qm);
        else if constexpr (KIND == 2) reg_r2<SLOT>(r, qm, m);
        else if constexpr (KIND == 3) reg_rot<SLOT>(r, qm, m);
        else reg_u2<SLOT>(r, qm, m);
    }
}

// General 2x2 on register bit J, applied to the packed pairs in `pm` only (a
// control on register bit J' >= 1); `odd`: to the odd element of each pair
// only (a control on register bit 0).  Controlled gates are rare in the
// workloads: this path favours code size over speed.
template <int J, int NP>
__device__ __forceinline__ void reg_u2_ctrl(RegsN<NP> &r, uint32_t pm, bool odd, const float4 *mrec) {
    const float4 m0 = mrec[0], m1 = mrec[1];
    const float u0r = m0.x, u0i = m0.y, u1r = m0.z, u1i = m0.w;
    const float u2r = m1.x, u2i = m1.y, u3r = m1.z, u3i = m1.w;
#pragma unroll
    for (int q = 0; q < NP; q++) {
        if (!((pm >> q) & 1)) continue;
        if constexpr (J >= 1) {
            constexpr int S = 1 << (J - 1);
            if (q & S) continue;
            const int q1 = q | S;
            if (odd) {
                const float ar = r.re[q].y, ai = r.im[q].y, br = r.re[q1].y, bi = r.im[q1].y;
                r.re[q].y = u0r * ar - u0i * ai + u1r * br - u1i * bi;
                r.im[q].y = u0r * ai + u0i * ar + u1r * bi + u1i * br;
                r.re[q1].y = u2r * ar - u2i * ai + u3r * br - u3i * bi;
                r.im[q1].y = u2r * ai + u2i * ar + u3r * bi + u3i * br;
            } else {
                const float2 ar = r.re[q], ai = r.im[q], br = r.re[q1], bi = r.im[q1];
                r.re[q] = fma2(bi, f2(-u1i), fma2(br, f2(u1r), fma2(ai, f2(-u0i), mul2(ar, f2(u0r)))));
                r.im[q] = fma2(br, f2(u1i), fma2(bi, f2(u1r), fma2(ar, f2(u0i), mul2(ai, f2(u0r)))));
                r.re[q1] = fma2(bi, f2(-u3i), fma2(br, f2(u3r), fma2(ai, f2(-u2i), mul2(ar, f2(u2r)))));
                r.im[q1] = fma2(br, f2(u3i), fma2(bi, f2(u3r), fma2(ar, f2(u2i), mul2(ai, f2(u2r)))));
            }
        } else {
            const float ar = r.re[q].x, ai = r.im[q].x, br = r.re[q].y, bi = r.im[q].y;
            r.re[q].x = u0r * ar - u0i * ai + u1r * br - u1i * bi;
            r.im[q].x = u0r * ai + u0i * ar + u1r * bi + u1i * br;
            r.re[q].y = u2r * ar - u2i * ai + u3r * br - u3i * bi;
            r.im[q].y = u2r * ai + u2i * ar + u3r * bi + u3i * br;
        }
    }
}

// Multiply amplitude x of the register index by entry x of a 32-entry
// constant phase table in shared memory: T[q] = (re[2q], re[2q+1], im[2q],
// im[2q+1]).  `qm` as in reg_h2 (all ones at run time; bounds the loads kept
// in flight).
template <int NP>
__device__ __forceinline__ void apply_table_s(RegsN<NP> &r, const float4 *T, uint32_t qm) {
#pragma unroll
    for (int g4 = 0; g4 < NP / 4; g4++) {
        if (!((qm >> g4) & 1)) continue;
#pragma unroll
        for (int i = 0; i < 4; i++) {
            const int q = 4 * g4 + i;
            const float4 t = T[q];
            const float2 tr = make_float2(t.x, t.y), ti = make_float2(t.z, t.w);
            const float2 nr = fma2(r.im[q], make_float2(-t.z, -t.w), mul2(r.re[q], tr));
            const float2 ni = fma2(r.im[q], tr, mul2(r.re[q], ti));
            r.re[q] = nr;
            r.im[q] = ni;
        }
    }
}

// Phased Hadamard on register bit J: the amplitude b of each pair (bit J = 1)
// is multiplied by T[x] (a 32-entry phase table in shared memory laid out as
// for apply_table_s), then by the per-thread factor (fr + i fi), and the pair
// becomes (a + p, a - p) with p that product.  Butterflies without a table are
// grouped four at a time as in reg_h2, those with one all eight together.
// Without a table (`tab` false: the run's phase is the
// per-thread factor alone, as for the first Hadamard of a stage in an inverse
// QFT) the table product is skipped.
template <int J, int NP>
__device__ __forceinline__ void reg_hph_s(RegsN<NP> &r, uint32_t qm, const float4 *T, bool tab, float fr,
                                          float fi, bool shared) {
    const float2 Fr = f2(fr), Fi = f2(fi), Fni = f2(-fi);
    if constexpr (J >= 1) {
        if constexpr (J <= 3) {
            if (tab && shared) {
                // the table depends only on register bits below J
                // (kT2HphShared): the 2^(J-1) products u = F T, once, then
                // b <- u b per pair
                constexpr int NV = 1 << (J - 1);
                float2 ur[NV], ui[NV], nui[NV];
#pragma unroll
                for (int v = 0; v < NV; v++) {
                    const float4 t = T[v | NV];
                    const float2 tr = make_float2(t.x, t.y), ti = make_float2(t.z, t.w);
                    ur[v] = fma2(ti, Fni, mul2(tr, Fr));
                    ui[v] = fma2(tr, Fi, mul2(ti, Fr));
                    nui[v] = make_float2(-ui[v].x, -ui[v].y);
                }
#pragma unroll
                for (int g = 0; g < NP / 16; g++) {
                    if (!((qm >> g) & 1)) continue;
#pragma unroll
                    for (int i = 0; i < 8; i++) {
                        const int q = bfly_q<J>(8 * g + i), q1 = q | (1 << (J - 1));
                        const int v = q1 & (NV - 1);
                        const float2 br = r.re[q1], bi = r.im[q1];
                        const float2 pr = fma2(bi, nui[v], mul2(br, ur[v]));
                        const float2 pi = fma2(bi, ur[v], mul2(br, ui[v]));
                        r.re[q1] = sub2(r.re[q], pr);
                        r.im[q1] = sub2(r.im[q], pi);
                        r.re[q] = add2(r.re[q], pr);
                        r.im[q] = add2(r.im[q], pi);
                    }
                }
                return;
            }
        }
        if (!tab) {
#pragma unroll
            for (int g = 0; g < NP / 8; g++) {
                if (!((qm >> g) & 1)) continue;
#pragma unroll
                for (int i = 0; i < 4; i++) {
                    const int q = bfly_q<J>(4 * g + i), q1 = q | (1 << (J - 1));
                    const float2 br = r.re[q1], bi = r.im[q1];
                    const float2 pr = fma2(bi, Fni, mul2(br, Fr));
                    const float2 pi = fma2(bi, Fr, mul2(br, Fi));
                    r.re[q1] = sub2(r.re[q], pr);
                    r.im[q1] = sub2(r.im[q], pi);
                    r.re[q] = add2(r.re[q], pr);
                    r.im[q] = add2(r.im[q], pi);
                }
            }
            return;
        }
#pragma unroll
        for (int g = 0; g < NP / 16; g++) {  // all eight butterflies in one group (measured faster)
            if (!((qm >> g) & 1)) continue;
#pragma unroll
            for (int i = 0; i < 8; i++) {
                const int q = bfly_q<J>(8 * g + i), q1 = q | (1 << (J - 1));
                const float4 t = T[q1];
                const float2 tr = make_float2(t.x, t.y), ti = make_float2(t.z, t.w);
                const float2 nti = make_float2(-t.z, -t.w);
                const float2 b0r = r.re[q1], b0i = r.im[q1];
                const float2 br = fma2(b0i, nti, mul2(b0r, tr));  // T b
                const float2 bi = fma2(b0i, tr, mul2(b0r, ti));
                const float2 pr = fma2(bi, Fni, mul2(br, Fr));    // F (T b)
                const float2 pi = fma2(bi, Fr, mul2(br, Fi));
                r.re[q1] = sub2(r.re[q], pr);
                r.im[q1] = sub2(r.im[q], pi);
                r.re[q] = add2(r.re[q], pr);
                r.im[q] = add2(r.im[q], pi);
            }
        }
    } else {
#pragma unroll
        for (int g4 = 0; g4 < NP / 4; g4++) {
            if (!((qm >> g4) & 1)) continue;
#pragma unroll
            for (int i = 0; i < 4; i++) {
                const int q = 4 * g4 + i;
                float mr = fr, mi = fi;
                if (tab) {
                    const float4 t = T[q];  // odd entries (bit 0 set): y and w
                    mr = t.y * fr - t.w * fi;
                    mi = t.y * fi + t.w * fr;
                }
                float2 &x = r.re[q], &y = r.im[q];
                const float pr = x.y * mr - y.y * mi, pi = x.y * mi + y.y * mr;
                x.y = x.x - pr;
                y.y = y.x - pi;
                x.x = x.x + pr;
                y.x = y.x + pi;
            }
        }
    }
}

// `rbar`: mbarrier that every warp arrives at once it has read a stage's
// layout from shared memory (count: the CTA's warps); `rd` counts this
// thread's arrivals.  A stage change waits for the phase of the previous read
// before it overwrites the tile, so no warp overwrites data another warp has
// not read yet, without a CTA barrier.  `base`: the tile's physical base
// index; `slotc`: the tile's slot values.  After the last stage change has
// read shared memory, `hook()` runs (the callers start the next tile's bulk
// copies there, once rbar shows every warp's reads done).
template <int K, int F, typename Hook>
__device__ __forceinline__ void t2_run(const T2Args &a, float4 *gstate, uint64_t *rbar, uint32_t &rd,
                                       uint64_t base, const float2 *slotc, Hook hook) {
    using G = Geo<K>;
    // the programme: copied to shared memory by k_tile2 (once per CTA) and
    // k_batch (once per pass); static rows and layouts beyond the copy stay
    // in global memory
    const int4 *ins = reinterpret_cast<const int4 *>(t2_dyn_smem + G::kOffIns);
    const int4 *fac = reinterpret_cast<const int4 *>(t2_dyn_smem + G::kOffFac);
    const float2 *rows = reinterpret_cast<const float2 *>(t2_dyn_smem + G::kOffRows);
    const float4 *M = reinterpret_cast<const float4 *>(t2_dyn_smem + G::kOffMats);
    const T2LayoutX *lays = reinterpret_cast<const T2LayoutX *>(t2_dyn_smem + G::kOffLay);
    const float4 *ones = reinterpret_cast<const float4 *>(t2_dyn_smem + G::kOffOnes);
    float4 *tile4 = reinterpret_cast<float4 *>(t2_dyn_smem);
    const int tid = threadIdx.x;
    auto layout = [&](int st) -> const T2LayoutX * { return st < kT2SmemStages ? lays + st : a.layx + st; };
    RegsN<kNP2> r;
    int stage = 0;
    bool live = false;
    // a per-thread factor: static row x tile slot x one slot per dynamic thread bit set
    auto thread_factor = [&](const int4 fd) -> float2 {
        const uint32_t w0 = (uint32_t)fd.x;
        const int sl = (int16_t)(fd.y & 0xffff), dsl = (int16_t)((uint32_t)fd.y >> 16);
        float2 f = make_float2(1.f, 0.f);
        if (fd.z >= 0)
            f = fd.z < kT2SmemRows ? rows[fd.z * G::kThreads + tid]
                                   : __ldg(a.statc + (size_t)fd.z * G::kThreads + tid);
        if (sl >= 0) f = cx(f, slotc[sl]);
        const uint32_t dmask = (w0 >> kFacDynShift) & 0x1ffu;
        uint32_t dm = dmask & (uint32_t)tid;
        while (dm) {
            const int t = __ffs(dm) - 1;
            dm &= dm - 1;
            f = cx(f, slotc[dsl + __popc(dmask & ((1u << t) - 1u))]);
        }
        return f;
    };
    // the run of a phased butterfly: its table (or the identity) and its factor
    auto hph_run = [&](const int4 w, const float4 *&T, float2 &ph) {
        const int e0 = (int16_t)(w.z & 0xffff), e1 = (int16_t)(w.z >> 16);
        T = ones;
        ph = make_float2(1.f, 0.f);
        for (int e = e0; e < e1; e++) {
            const int4 fd = fac[e];
            if ((uint32_t)fd.x & kFacTable)
                T = M + 2 * fd.z;
            else
                ph = thread_factor(fd);
        }
    };
    // the same from the step itself: its table, static row and slot are
    // independent loads (no factor record first)
    auto hph_direct = [&](const int4 w, const float4 *&T, float2 &ph) {
        const int trec = (int)((uint32_t)w.w & 0xffffu) - 1, row = (int)((uint32_t)w.w >> 16) - 1;
        const int sl = (int16_t)(w.y & 0xffff);
        T = trec >= 0 ? M + 2 * trec : ones;
        ph = make_float2(1.f, 0.f);
        if (row >= 0)
            ph = row < kT2SmemRows ? rows[row * G::kThreads + tid]
                                   : __ldg(a.statc + (size_t)row * G::kThreads + tid);
        if (sl >= 0) ph = cx(ph, slotc[sl]);
    };
    // loop bounds in registers: `a` may live in memory the compiler cannot
    // prove unchanged by the tile's shared-memory stores (the L2 block kernel
    // indexes its passes' arguments)
    const int nins = a.nins, last_stage = a.last_stage;
    for (int pc = 0; pc < nins; pc++) {
        const int4 w = ins[pc];
        // all ones at run time (the handler code is below 256), opaque to the
        // compiler (see reg_h2)
        const uint32_t qm = ~((uint32_t)w.y >> 24);
        const float4 *mrec = M + 2 * w.w;
        // one switch on the handler code the stage compiler set (tileprog.h)
        switch (((uint32_t)w.y >> 16) & 0xffu) {
            case kT2HdStage: {
                if (live) {
                    // every warp has read the previous layout before any overwrites it
                    if (!mbar_wait(rbar, (rd - 1u) & 1u)) atomicExch(a.err, 1);
                    const LayoutS L(layout(stage), tid);
#pragma unroll
                    for (int q = 0; q < kNP2; q++)
                        tile4[L.idx(q)] = make_float4(r.re[q].x, r.re[q].y, r.im[q].x, r.im[q].y);
                    __syncthreads();
                    stage = w.w;
                    const LayoutS L2(layout(stage), tid);
#pragma unroll
                    for (int q = 0; q < kNP2; q++) {
                        const float4 v = tile4[L2.idx(q)];
                        r.re[q] = make_float2(v.x, v.y);
                        r.im[q] = make_float2(v.z, v.w);
                    }
                } else {
                    stage = w.w;
                    const Layout2 L(layout(stage), tid);
                    if (a.gen) {
                        // the product state H^{hq}|b>, generated instead of
                        // read: +-v where the index agrees with b off the
                        // Hadamard qubits (global ones decide the whole tile),
                        // with the sign of the parity of b on them, 0 elsewhere.
                        // Element x of the register index (bit 0: the element
                        // of a packed pair, bits 1..4: register bits 1..4) sits
                        // at tile index bt + sum of the s_k of its set bits, so
                        // both conditions split into a per-thread part and one
                        // bit mask over the 32 elements each.
                        const uint32_t gl = (uint32_t)a.gen_local, hm = a.gen_hmask;
                        const uint32_t pos[5] = {1u, (uint32_t)L.s1, (uint32_t)L.s2, (uint32_t)L.s3,
                                                 (uint32_t)L.s4};
                        const uint32_t R = pos[0] | pos[1] | pos[2] | pos[3] | pos[4];
                        const uint32_t bt = (uint32_t)L.bt;
                        bool has = ((a.gen_basis ^ base) & a.gmask & ~a.gen_ghmask) == 0;
                        has = has && ((bt ^ gl) & ~hm & ~R) == 0;
                        uint32_t neg = (((uint32_t)__popcll(base & a.gen_basis & a.gen_ghmask) ^
                                         (uint32_t)__popc(bt & gl & hm)) & 1u) ? ~0u : 0u;
                        uint32_t nz = has ? ~0u : 0u;
                        // x's bit k set: the elements of the k-th alternating bit mask
                        const uint32_t Mk[5] = {0xAAAAAAAAu, 0xCCCCCCCCu, 0xF0F0F0F0u, 0xFF00FF00u,
                                                0xFFFF0000u};
#pragma unroll
                        for (int k = 0; k < 5; k++) {
                            if (pos[k] & ~hm) nz &= (gl & pos[k]) ? Mk[k] : ~Mk[k];
                            if (pos[k] & gl & hm) neg ^= Mk[k];
                        }
                        const uint32_t vb = __float_as_uint(a.gen_val);
                        auto amp = [&](int x) -> float {
                            return __uint_as_float((((neg >> x) & 1u) << 31 ^ vb) & (0u - ((nz >> x) & 1u)));
                        };
#pragma unroll
                        for (int q = 0; q < kNP2; q++) {
                            r.re[q] = make_float2(amp(2 * q), amp(2 * q + 1));
                            r.im[q] = make_float2(0.f, 0.f);
                        }
                    } else {  // the bulk copies' linear order: lane bits 0..2 are tile bits 1..3
#pragma unroll
                        for (int q = 0; q < kNP2; q++) {
                            const float4 v = tile4[L.idx(q)];
                            r.re[q] = make_float2(v.x, v.z);
                            r.im[q] = make_float2(v.y, v.w);
                        }
                    }
                }
                live = true;
                __syncwarp();
                if ((tid & 31) == 0) mbar_arrive(rbar);
                rd++;
                if (pc == last_stage) hook();
                continue;
            }
            case kT2HdScale: {
                const float4 mm = mrec[0];
                const float hi = mm.x, lo = mm.y;
                if (lo == 0.f) {  // an even number of Hadamards: an exact power of two
#pragma unroll
                    for (int q = 0; q < kNP2; q++) {
                        r.re[q] = mul2(r.re[q], f2(hi));
                        r.im[q] = mul2(r.im[q], f2(hi));
                    }
                    continue;
                }
#pragma unroll
                for (int q = 0; q < kNP2; q++) {
                    r.re[q] = fma2(r.re[q], f2(hi), mul2(r.re[q], f2(lo)));
                    r.im[q] = fma2(r.im[q], f2(hi), mul2(r.im[q], f2(lo)));
                }
                continue;
            }
            case kT2HdDiag: {
                const int e0 = (int16_t)(w.z & 0xffff), e1 = (int16_t)(w.z >> 16);
                for (int e = e0; e < e1; e++) {
                    const int4 fd = fac[e];
                    const uint32_t w0 = (uint32_t)fd.x;
                    if (w0 & kFacTable) {
                        const int pb = (int)((w0 >> 10) & 0xfu);  // thread-bit predicate
                        if (pb && !((tid >> (pb - 1)) & 1)) continue;
                        apply_table_s(r, M + 2 * fd.z, qm);
                        continue;
                    }
                    const float2 ff = thread_factor(fd);
                    apply_factor_bit(r, (int)(w0 & 0xffu), ff.x, ff.y);
                }
                continue;
            }
#define SV_HPH_CASE(J)                                              \
    case kT2Handler + 8 * 5 + J: {                                  \
        const float4 *T;                                            \
        float2 ph;                                                  \
        const int8_t hc = (int8_t)(w.x >> 24);                      \
        if (hc == kT2HphDirect || hc == kT2HphShared)               \
            hph_direct(w, T, ph);                                   \
        else                                                        \
            hph_run(w, T, ph);                                      \
        reg_hph_s<J>(r, qm, T, T != ones, ph.x, ph.y, hc == kT2HphShared); \
        continue;                                                   \
    }
            SV_HPH_CASE(0)
            SV_HPH_CASE(1)
            SV_HPH_CASE(2)
            SV_HPH_CASE(3)
            SV_HPH_CASE(4)
#undef SV_HPH_CASE
#define SV_GATE_CASES(K)                                                         \
    case kT2Handler + 8 * K + 0: run_gate<F, K, 0>(r, mrec, qm); continue;       \
    case kT2Handler + 8 * K + 1: run_gate<F, K, 1>(r, mrec, qm); continue;       \
    case kT2Handler + 8 * K + 2: run_gate<F, K, 2>(r, mrec, qm); continue;       \
    case kT2Handler + 8 * K + 3: run_gate<F, K, 3>(r, mrec, qm); continue;       \
    case kT2Handler + 8 * K + 4: run_gate<F, K, 4>(r, mrec, qm); continue;
            SV_GATE_CASES(0)
            SV_GATE_CASES(1)
            SV_GATE_CASES(2)
            SV_GATE_CASES(3)
            SV_GATE_CASES(4)
#undef SV_GATE_CASES
            default: break;
        }
        {  // slot 7: a register-bit gate with a register, thread or tile control
            const int j = (int8_t)((w.x >> 16) & 0xff);
            const int ccls = (w.x >> 24) & 0xff;
            const int cidx = (int16_t)(w.y & 0xffff);
            if (ccls == T2C_GLOBAL) {
                if (!((base >> cidx) & 1)) continue;  // tile-uniform
            } else if (ccls == T2C_THREAD) {
                if (!((tid >> cidx) & 1)) continue;
            }
            const int kind = ((((uint32_t)w.y >> 16) & 0xffu) - kT2Handler) >> 3;
            if (ccls == T2C_REG) {  // general 2x2 on the pairs that hold the control
                if constexpr ((F & (kFeatR | kFeatU)) != 0) {
                    const uint32_t pm = (uint32_t)w.z & 0xffffu;
                    const bool odd = ((uint32_t)w.z >> 16) != 0;
                    switch (j) {
                        case 0: reg_u2_ctrl<0>(r, pm, odd, mrec); break;
                        case 1: reg_u2_ctrl<1>(r, pm, odd, mrec); break;
                        case 2: reg_u2_ctrl<2>(r, pm, odd, mrec); break;
                        case 3: reg_u2_ctrl<3>(r, pm, odd, mrec); break;
                        default: reg_u2_ctrl<4>(r, pm, odd, mrec); break;
                    }
                }
                continue;
            }
#define SV_CTRL_CASE(K)                                                   \
    if (kind == K) {                                                      \
        switch (j) {                                                      \
            case 0: run_gate<F, K, 0>(r, mrec, qm); break;                \
            case 1: run_gate<F, K, 1>(r, mrec, qm); break;                \
            case 2: run_gate<F, K, 2>(r, mrec, qm); break;                \
            case 3: run_gate<F, K, 3>(r, mrec, qm); break;                \
            default: run_gate<F, K, 4>(r, mrec, qm); break;               \
        }                                                                 \
        continue;                                                         \
    }
            SV_CTRL_CASE(2)
            SV_CTRL_CASE(4)
#undef SV_CTRL_CASE
        }
    }
    if (!live) return;
    const T2Epilogue *E = reinterpret_cast<const T2Epilogue *>(t2_dyn_smem + G::kOffEpi);
    // offsets inside the state, in 16-byte vectors from the tile's base (bit 0
    // of every amplitude offset is a tile bit, so they are even); 32 bits wide
    // while the state holds at most 2^33 amplitudes
    float4 *gt = gstate + (base >> 1);
    if (a.ntiles <= (UINT64_C(1) << (33 - K))) {
        const uint32_t o0 = (uint32_t)((E->glo[tid & 31] + E->ghi[tid >> 5]) >> 1);
        const uint32_t o1 = (uint32_t)(E->g[0] >> 1), o2 = (uint32_t)(E->g[1] >> 1);
        const uint32_t o3 = (uint32_t)(E->g[2] >> 1), o4 = (uint32_t)(E->g[3] >> 1);
        auto off = [&](int q) {
            return o0 + ((q & 1) ? o1 : 0u) + ((q & 2) ? o2 : 0u) + ((q & 4) ? o3 : 0u) + ((q & 8) ? o4 : 0u);
        };
        if (a.keep) {  // the next pass of an L2 block reads it: plain stores
#pragma unroll
            for (int q = 0; q < kNP2; q++) gt[off(q)] = make_float4(r.re[q].x, r.im[q].x, r.re[q].y, r.im[q].y);
            return;
        }
#pragma unroll
        for (int q = 0; q < kNP2; q++) __stcs(gt + off(q), make_float4(r.re[q].x, r.im[q].x, r.re[q].y, r.im[q].y));
        return;
    }
    const uint64_t g0 = E->glo[tid & 31] + E->ghi[tid >> 5];
    const uint64_t g1 = E->g[0], g2 = E->g[1], g3 = E->g[2], g4 = E->g[3];
    auto off64 = [&](int q) {
        return (g0 + ((q & 1) ? g1 : 0) + ((q & 2) ? g2 : 0) + ((q & 4) ? g3 : 0) + ((q & 8) ? g4 : 0)) >> 1;
    };
    if (a.keep) {
#pragma unroll
        for (int q = 0; q < kNP2; q++) gt[off64(q)] = make_float4(r.re[q].x, r.im[q].x, r.re[q].y, r.im[q].y);
        return;
    }
#pragma unroll
    for (int q = 0; q < kNP2; q++) __stcs(gt + off64(q), make_float4(r.re[q].x, r.im[q].x, r.re[q].y, r.im[q].y));
}

// Physical base index of tile `tile`: its index bits spread over the runs of
// the global qubits.
__device__ __forceinline__ uint64_t tile_base(const T2Args &a, uint64_t tile) {
    uint64_t b = 0;
    for (int i = 0; i < a.ngr; i++)
        b |= ((tile >> a.gs[i]) & ((UINT64_C(1) << a.gl[i]) - 1)) << a.gd[i];
    return b;
}

// The tile's bulk copies (warp 0); with `slots` the tile's precomputed slot
// values come on the same barrier.
template <int K>
__device__ __forceinline__ void issue_tile_load(const T2Args &a, unsigned char *sm, const float *state,
                                                uint64_t tile, uint64_t *bar, int tid,
                                                float2 *slots = nullptr) {
    const int nchunks = 1 << (K - a.c);
    const uint32_t chunk_bytes = 8u << a.c;
    const uint64_t base = tile_base(a, tile);
    if (tid == 0) {
        fence_async_smem();
        const uint32_t sb = slots ? (uint32_t)a.nsp * 8u : 0u;
        mbar_expect_tx(bar, Geo<K>::kTileBytes + sb);
        if (slots) bulk_g2s(slots, a.slotv + tile * (uint64_t)a.nsp, sb, bar);
    }
    __syncwarp();
    for (int j = tid; j < nchunks; j += 32) {
        uint64_t off = 0;
        for (int b = 0; b < K - a.c; b++)
            if ((j >> b) & 1) off |= UINT64_C(1) << a.slot_phys[a.c + b];
        bulk_g2s(sm + (size_t)j * chunk_bytes, state + 2 * (base + off), chunk_bytes, bar);
    }
}

// The pass's programme into shared memory (sizes bounded by the stage compiler).
template <int K>
__device__ __forceinline__ void load_programme(const T2Args &a, unsigned char *sm, int tid, int nthreads) {
    using G = Geo<K>;
    int4 *si = reinterpret_cast<int4 *>(sm + G::kOffIns);
    int4 *sf = reinterpret_cast<int4 *>(sm + G::kOffFac);
    float2 *sr = reinterpret_cast<float2 *>(sm + G::kOffRows);
    float4 *smat = reinterpret_cast<float4 *>(sm + G::kOffMats);
    int4 *slay = reinterpret_cast<int4 *>(sm + G::kOffLay);
    int4 *sepi = reinterpret_cast<int4 *>(sm + G::kOffEpi);
    for (int i = tid; i < a.nins; i += nthreads) si[i] = __ldg(a.ins + i);
    for (int i = tid; i < a.nfac; i += nthreads) sf[i] = __ldg(a.fac + i);
    for (int i = tid; i < 2 * a.nmats; i += nthreads) smat[i] = __ldg(a.mats + i);
    const int nl = min(a.nstages, kT2SmemStages) * (int)(sizeof(T2LayoutX) / 16);
    for (int i = tid; i < nl; i += nthreads) slay[i] = __ldg(reinterpret_cast<const int4 *>(a.layx) + i);
    for (int i = tid; i < (int)(sizeof(T2Epilogue) / 16); i += nthreads)
        sepi[i] = __ldg(reinterpret_cast<const int4 *>(a.epi) + i);
    const int nr = min(a.nrows, kT2SmemRows) * G::kThreads;
    for (int i = tid; i < nr; i += nthreads) sr[i] = __ldg(a.statc + i);
    float4 *ones = reinterpret_cast<float4 *>(sm + G::kOffOnes);  // the identity phase table
    for (int i = tid; i < 16; i += nthreads) ones[i] = make_float4(1.f, 1.f, 0.f, 0.f);
}

// The tile's slot values (Sec. III-B: global qubits are constants of the
// tile): each warp sums the terms of its slots over its lanes (exact 32-bit
// phase arithmetic), and one lane forms e^{2 pi i u / 2^32} from the four
// FP64-generated tables.
template <int K>
__device__ __forceinline__ void tile_slots(const T2Args &a, const float2 *tab, float2 *slotc, uint64_t base,
                                           int tid) {
    const int warp = tid >> 5, lane = tid & 31;
    for (int sl = warp; sl < a.nslots; sl += Geo<K>::kWarps) {
        const int t0 = __ldg(a.soff + sl), t1 = __ldg(a.soff + sl + 1);
        uint32_t u = 0;
        for (int t = t0 + lane; t < t1; t += 32) {
            const T2SlotTerm st = a.sterms[t];
            bool on = (base >> st.g0) & 1;
            if (st.g1 >= 0) on = on && ((base >> st.g1) & 1);
            if (on) u += st.theta;
        }
#pragma unroll
        for (int o = 16; o; o >>= 1) u += __shfl_xor_sync(0xffffffffu, u, o);
        if (lane == 0)
            slotc[sl] = cx(cx(tab[u >> 24], tab[kTabN + ((u >> 16) & 255u)]),
                           cx(tab[2 * kTabN + ((u >> 8) & 255u)], tab[3 * kTabN + (u & 255u)]));
    }
}

// The slot values of every tile of a pass (the same sums and table products
// as tile_slots, one thread per tile and slot), computed before the pass so
// that its tiles receive them with their bulk copies.
__global__ void k_slotv(const T2Args a, float2 *__restrict__ out) {
    const uint64_t total = a.ntiles * (uint64_t)a.nsp;
    const float2 *tab = a.tables;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t tile = i / (uint64_t)a.nsp;
        const int sl = (int)(i - tile * (uint64_t)a.nsp);
        float2 v = make_float2(1.f, 0.f);
        if (sl < a.nslots) {
            const uint64_t base = tile_base(a, tile);
            uint32_t u = 0;
            const int t1 = __ldg(a.soff + sl + 1);
            for (int t = __ldg(a.soff + sl); t < t1; t++) {
                const T2SlotTerm st = a.sterms[t];
                bool on = (base >> st.g0) & 1;
                if (st.g1 >= 0) on = on && ((base >> st.g1) & 1);
                if (on) u += st.theta;
            }
            v = cx(cx(__ldg(tab + (u >> 24)), __ldg(tab + kTabN + ((u >> 16) & 255u))),
                   cx(__ldg(tab + 2 * kTabN + ((u >> 8) & 255u)), __ldg(tab + 3 * kTabN + (u & 255u))));
        }
        out[i] = v;
    }
}

// Persistent CTA over the pass's tiles.  Tile i+1's bulk copies start as
// soon as tile i's last stage change has read shared memory, so they overlap
// the rest of tile i's programme and its write-back, which goes from
// registers straight to the global state (16-byte stores; lanes 0..7 cover
// tile bits 1..3, so a quarter-warp writes 128 contiguous bytes).
template <int K, int F>
__global__ void __launch_bounds__(Geo<K>::kThreads, K == kT2Qubits ? 2 : 1)
    k_tile2(float *__restrict__ state, const T2Args a) {
    using G = Geo<K>;
    extern __shared__ __align__(1024) unsigned char sm[];
    float2 *tab = reinterpret_cast<float2 *>(sm + G::kOffTab);
    float2 *slotc = reinterpret_cast<float2 *>(sm + G::kOffSlotc);
    uint64_t *bar = reinterpret_cast<uint64_t *>(sm + G::kOffBar);
    uint64_t *rbar = bar + 1;
    const int tid = threadIdx.x;

    for (int i = tid; i < kTabEntries; i += blockDim.x) tab[i] = a.tables[i];
    load_programme<K>(a, sm, tid, blockDim.x);
    if (tid == 0) {
        mbar_init(bar, 1);
        mbar_init(rbar, G::kWarps);
        fence_mbar_init();
    }
    __syncthreads();
    // precomputed slot values: tile t's arrive with its copies (a pass that
    // generates its state copies only them), into the slot buffer the previous
    // tile did not use
    const bool pre = a.slotv != nullptr;
    auto issue_slots_only = [&](uint64_t t, float2 *dst) {
        fence_async_smem();
        mbar_expect_tx(bar, (uint32_t)a.nsp * 8u);
        bulk_g2s(dst, a.slotv + t * (uint64_t)a.nsp, (uint32_t)a.nsp * 8u, bar);
    };
    if ((uint64_t)blockIdx.x < a.ntiles) {
        if (!a.gen && tid < 32)
            issue_tile_load<K>(a, sm, state, blockIdx.x, bar, tid, pre ? slotc : nullptr);
        else if (a.gen && pre && tid == 0)
            issue_slots_only(blockIdx.x, slotc);
    }

    uint32_t parity = 0, rd = 0, buf = 0;
    for (uint64_t tile = blockIdx.x; tile < a.ntiles; tile += gridDim.x) {
        const uint64_t next = tile + gridDim.x;
        const uint64_t base = tile_base(a, tile);
        // the tile's slot values while its copies are in flight, into the
        // buffer the previous tile did not use (every warp passed that tile's
        // barrier below, so none still reads the one before)
        float2 *sc = slotc + buf * kT2MaxSlots;
        if (!pre) tile_slots<K>(a, tab, sc, base, tid);
        const bool timed_out = (a.gen && !pre) ? false : !mbar_wait(bar, parity);
        if (__syncthreads_or(timed_out)) {
            if (tid == 0) atomicExch(a.err, 1);
            mbar_wait(bar, parity);  // give copies still in flight a second bounded wait
            return;
        }
        // the next tile's copies, once every warp has read the last layout
        auto hook = [&]() {
            float2 *nsc = slotc + (buf ^ 1u) * kT2MaxSlots;
            if (!a.gen && tid < 32 && next < a.ntiles) {
                if (!mbar_wait(rbar, (rd - 1u) & 1u)) atomicExch(a.err, 1);
                issue_tile_load<K>(a, sm, state, next, bar, tid, pre ? nsc : nullptr);
            } else if (a.gen && pre && tid == 0 && next < a.ntiles) {
                issue_slots_only(next, nsc);
            }
        };
        t2_run<K, F>(a, reinterpret_cast<float4 *>(state), rbar, rd, base, sc, hook);
        parity ^= 1u;
        buf ^= 1u;
    }
}

// ---------------------------------------------------------------- L2 blocks
// Two-level blocking (Sec. III-B, the block sized by the last-level cache):
// the passes of a group run in one launch over blocks of 2^l amplitudes.
// Persistent CTAs claim tiles from one queue in the order of G.segs, where
// pass p of block b comes G.lag steps after pass p-1 of block b: by the time
// it is claimed the block's previous pass has almost always finished, and
// its result is still in L2 (written with plain stores; the group's last
// pass streams its result out).  A tile of pass p >= 1 starts its bulk copies
// once the (block, p-1) counter shows all of that pass's tiles done:
//   - at the hook of the tile before it if the counter is already full
//     there (the usual case: the copies overlap that tile's end);
//   - otherwise at the top of its own iteration, after the CTA has finished
//     and counted its previous tile, with a bounded wait on the counter.
// Claim order is a topological order of the dependencies and only running
// CTAs claim, so the wait at the top always ends; a CTA never waits for a
// tile it holds itself.
template <int F>
__global__ void __launch_bounds__(kT2Threads, 2)
    k_group(float *__restrict__ state, const __grid_constant__ GroupArgs G) {
    extern __shared__ __align__(1024) unsigned char sm[];
    float2 *tab = reinterpret_cast<float2 *>(sm + G13::kOffTab);
    float2 *slotc = reinterpret_cast<float2 *>(sm + G13::kOffSlotc);
    uint64_t *bar = reinterpret_cast<uint64_t *>(sm + G13::kOffBar);
    uint64_t *rbar = bar + 1;
    unsigned long long &s_next = *reinterpret_cast<unsigned long long *>(sm + G13::kOffClaim);
    const int tid = threadIdx.x;
    const unsigned tpb = 1u << G.tpb_log;
    for (int i = tid; i < kTabEntries; i += blockDim.x) tab[i] = G.pass[0].tables[i];
    if (tid == 0) {
        mbar_init(bar, 1);
        mbar_init(rbar, G13::kWarps);
        fence_mbar_init();
        s_next = atomicAdd(G.queue, 1ull) << G.chunk_log;
    }
    __syncthreads();
    // item q: tile (q mod tpb) of the (block, pass) segment q / tpb; a claim
    // takes the 2^chunk_log consecutive items of one chunk
    const unsigned long long cmask = (1ull << G.chunk_log) - 1ull;
    auto decode = [&](unsigned long long q, int &p, uint32_t &b, uint32_t &t) -> bool {
        if (q >= G.nitems) return false;
        const uint32_t s = __ldg(G.segs + (q >> G.tpb_log));
        p = (int)(s & 7u);
        b = s >> 3;
        t = (uint32_t)q & (tpb - 1u);
        return true;
    };
    auto tile_of = [&](uint32_t b, uint32_t t) { return (uint64_t)t | ((uint64_t)b << G.tpb_log); };
    int p = 0;
    uint32_t b = 0, t = 0;
    unsigned long long q = s_next;
    bool have = decode(q, p, b, t);
    bool issued = false;    // warp 0: this item's copies were started at the previous hook
    bool inflight = false;  // warp 0: this item's copies are in flight
    int loaded = -1;        // the pass whose programme is in shared memory
    long long sig = -1;     // the counter the previous item raises (-1: none)
    uint32_t parity = 0, rd = 0, buf = 0;
    for (;;) {
        // a previous item that a later pass reads is counted once its
        // write-back is complete in every thread; a pass change needs every
        // thread past the previous item's use of the programme area
        if (sig >= 0 || (have && p != loaded)) {
            if (sig >= 0) fence_async_global();
            __syncthreads();
            if (tid == 0 && sig >= 0) {
                __threadfence();
                atomicAdd(G.done + sig, 1u);
            }
        }
        if (!have) break;
        // the pass's arguments, copied next to its programme: shared-memory
        // loads instead of loads from the parameter block at a run-time index
        T2Args &a = *reinterpret_cast<T2Args *>(sm + G13::kOffArgs);
        if (p != loaded) {
            for (int i = tid; i < (int)(sizeof(T2Args) / 4); i += blockDim.x)
                reinterpret_cast<int *>(&a)[i] = reinterpret_cast<const int *>(&G.pass[p])[i];
            load_programme<kT2Qubits>(G.pass[p], sm, tid, blockDim.x);
            loaded = p;
            __syncthreads();
        }
        if (tid < 32) {
            inflight = issued;
            if (!issued && !a.gen) {
                bool ok = true;
                if (tid == 0 && p > 0)
                    ok = wait_count(G.done + (size_t)b * G.npass + (p - 1), tpb, G.err);
                ok = __shfl_sync(0xffffffffu, ok, 0);
                // every warp has read the previous item's last layout
                if (ok && rd && !mbar_wait(rbar, (rd - 1u) & 1u)) ok = false;
                if (ok) {
                    fence_async_global();
                    issue_tile_load<kT2Qubits>(a, sm, state, tile_of(b, t), bar, tid);
                    inflight = true;
                } else if (tid == 0) {
                    atomicExch(G.err, 1);
                }
            }
            if (tid == 0) s_next = ((q + 1) & cmask) ? q + 1 : (atomicAdd(G.queue, 1ull) << G.chunk_log);
        }
        const uint64_t base = tile_base(a, tile_of(b, t));
        float2 *sc = slotc + buf * kT2MaxSlots;
        tile_slots<kT2Qubits>(a, tab, sc, base, tid);
        const bool timed_out = a.gen ? false : !mbar_wait(bar, parity);
        if (__syncthreads_or(timed_out)) {
            if (tid == 0) atomicExch(G.err, 1);
            if (tid < 32 && inflight) mbar_wait(bar, parity);  // a second bounded wait for copies in flight
            return;
        }
        int np = 0;
        uint32_t nb = 0, nt = 0;
        const unsigned long long nq = s_next;
        const bool nhave = decode(nq, np, nb, nt);
        bool nissued = false;
        auto hook = [&]() {
            if (tid < 32 && nhave && !G.pass[np].gen) {
                bool ok = true;
                if (tid == 0 && np > 0) ok = ld_acquire(G.done + (size_t)nb * G.npass + (np - 1)) >= tpb;
                ok = __shfl_sync(0xffffffffu, ok, 0);
                if (ok) {
                    if (!mbar_wait(rbar, (rd - 1u) & 1u)) atomicExch(G.err, 1);
                    fence_async_global();
                    issue_tile_load<kT2Qubits>(G.pass[np], sm, state, tile_of(nb, nt), bar, tid);
                    nissued = true;
                }
            }
        };
        t2_run<kT2Qubits, F>(a, reinterpret_cast<float4 *>(state), rbar, rd, base, sc, hook);
        sig = p + 1 < G.npass ? (long long)b * G.npass + p : -1;
        if (!a.gen) parity ^= 1u;
        buf ^= 1u;
        q = nq;
        p = np;
        b = nb;
        t = nt;
        have = nhave;
        issued = nissued;
    }
}

// ---------------------------------------------------------------- batched instances
// CTAs take work items from a shared queue, in the claim order the host
// built:
//   - a small instance whole: all of its passes (the first generates its
//     starting product state in registers instead of reading the state),
//     then the FP64 argmax of the marginal over its read-out qubits;
//   - kBatchClaimTiles tiles of one pass of a large instance (pass p waits,
//     bounded, for a per-pass counter to show all tiles of pass p-1 done);
//   - the read-out of a large instance, after its last pass.
// Large instances come first, their passes lagged so that a pass's tiles are
// claimed well after the previous pass's; claim order is a topological order
// of those waits and a CTA counts its previous item before it waits, so
// every wait ends.  States of up to 2^20 amplitudes stay in L2.
template <int F>
__global__ void __launch_bounds__(kT2Threads, 2) k_batch(float *__restrict__ states, const BatchArgs B) {
    extern __shared__ __align__(1024) unsigned char sm[];
    float2 *tab = reinterpret_cast<float2 *>(sm + G13::kOffTab);
    float2 *slotc = reinterpret_cast<float2 *>(sm + G13::kOffSlotc);
    uint64_t *bar = reinterpret_cast<uint64_t *>(sm + G13::kOffBar);
    uint64_t *rbar = bar + 1;
    int &s_item = *reinterpret_cast<int *>(sm + G13::kOffClaim);
    // read-out reduction scratch lives in the tile buffer (free after the last pass)
    double *s_val = reinterpret_cast<double *>(sm);
    uint64_t *s_idx = reinterpret_cast<uint64_t *>(sm + 8 * kT2Threads);
    double *s_tot = reinterpret_cast<double *>(sm + 16 * kT2Threads);
    const int tid = threadIdx.x;
    for (int i = tid; i < kTabEntries; i += blockDim.x) tab[i] = B.tables[i];
    if (tid == 0) {
        mbar_init(bar, 1);
        mbar_init(rbar, kT2Threads / 32);
        fence_mbar_init();
    }
    __syncthreads();
    uint32_t parity = 0, rd = 0, buf = 0;
    // tiles [t0, t0 + nt) of one pass; false: a bounded wait ran out
    auto run_tiles = [&](const T2Args &ga, float *state, uint64_t t0, uint64_t nt) -> bool {
        // the pass's arguments, copied next to its programme (shared memory
        // instead of global loads inside the programme loop)
        T2Args &a = *reinterpret_cast<T2Args *>(sm + G13::kOffArgs);
        for (int i = tid; i < (int)(sizeof(T2Args) / 4); i += blockDim.x)
            reinterpret_cast<int *>(&a)[i] = reinterpret_cast<const int *>(&ga)[i];
        // a generated first pass reads nothing; later passes read the state
        // with bulk copies, the next tile's issued as soon as the current
        // one's last stage change has read shared memory, and write it
        // straight from registers
        if (!ga.gen && tid < 32) {
            fence_async_global();
            issue_tile_load<kT2Qubits>(ga, sm, state, t0, bar, tid);
        }
        load_programme<kT2Qubits>(ga, sm, tid, blockDim.x);
        __syncthreads();
        for (uint64_t tile = t0; tile < t0 + nt; tile++) {
            const uint64_t base = tile_base(a, tile);
            // slot values into the buffer the previous tile did not use
            float2 *sc = slotc + buf * kT2MaxSlots;
            tile_slots<kT2Qubits>(a, tab, sc, base, tid);
            bool timed_out = false;
            if (!a.gen) {
                timed_out = !mbar_wait(bar, parity);
                parity ^= 1u;
            }
            if (__syncthreads_or(timed_out)) {
                if (tid == 0) atomicExch(B.err, 1);
                mbar_wait(bar, parity ^ 1u);  // a second bounded wait for copies in flight
                return false;
            }
            auto hook = [&]() {
                if (!a.gen && tid < 32 && tile + 1 < t0 + nt) {
                    if (!mbar_wait(rbar, (rd - 1u) & 1u)) atomicExch(B.err, 1);
                    issue_tile_load<kT2Qubits>(a, sm, state, tile + 1, bar, tid);
                }
            };
            t2_run<kT2Qubits, F>(a, reinterpret_cast<float4 *>(state), rbar, rd, base, sc, hook);
            buf ^= 1u;
        }
        // the next pass's bulk copies (and the read-out) see this pass's stores
        fence_async_global();
        __syncthreads();
        return true;
    };
    // argmax (lowest index among ties) of the FP64 marginal over I.pos
    auto readout = [&](const BatchInst &I, const float *state) {
        // Outcomes are visited in the order of their physical index (bit i of
        // the visit index v is the i-th lowest physical read-out qubit), so
        // that a warp's loads are contiguous whatever qubit map the passes
        // left (QPE's inverse QFT ends bit-reversed).  Tables, in the tile
        // buffer after the reduction scratch: per byte of v, its physical
        // offset (T) and its outcome bits (Y).
        uint64_t *T = reinterpret_cast<uint64_t *>(sm + 24 * kT2Threads);
        uint32_t *Y = reinterpret_cast<uint32_t *>(T + 3 * 256);
        uint64_t mask = 0;
        for (int j = 0; j < I.m; j++) mask |= UINT64_C(1) << I.pos[j];
        for (int e = tid; e < 3 * 256; e += blockDim.x) {
            const int lvl = e >> 8, v = e & 255;
            uint64_t x = 0;
            uint32_t yb = 0;
            for (int b = 0; b < 8; b++) {
                const int i = lvl * 8 + b;  // rank among the read-out qubits' physical bits
                if (i >= I.m || !((v >> b) & 1)) continue;
                uint64_t mm = mask;
                for (int k = 0; k < i; k++) mm &= mm - 1;
                const int ph = __ffsll((long long)mm) - 1;
                x |= UINT64_C(1) << ph;
                for (int j = 0; j < I.m; j++)
                    if (I.pos[j] == ph) yb |= 1u << j;
            }
            T[e] = x;
            Y[e] = yb;
        }
        __syncthreads();
        const uint64_t all = (UINT64_C(1) << I.nphys) - 1;
        const uint64_t rest = all & ~mask;
        const uint64_t nrest = UINT64_C(1) << (I.nphys - I.m);
        const uint64_t outcomes = UINT64_C(1) << I.m;
        const float2 *st2 = reinterpret_cast<const float2 *>(state);
        double best = -1.0, tot = 0.0;
        uint64_t bidx = ~UINT64_C(0);
        for (uint64_t v = tid; v < outcomes; v += blockDim.x) {
            const uint64_t xy = T[v & 255] | T[256 + ((v >> 8) & 255)] | T[512 + ((v >> 16) & 255)];
            const uint64_t y = Y[v & 255] | Y[256 + ((v >> 8) & 255)] | Y[512 + ((v >> 16) & 255)];
            // exact FP32 squares (product + fmaf remainder) summed as a
            // double-float pair: FP64-accurate without FP64 arithmetic
            float hi = 0.f, lo = 0.f;
            auto two_sum = [&](float b) {
                const float t = hi + b;
                const float bb = t - hi;
                lo += (hi - (t - bb)) + (b - bb);
                hi = t;
            };
            // the amplitudes of outcome y in increasing index order, four
            // independent loads in flight at a time
            uint64_t xr = 0;
            for (uint64_t r = 0; r < nrest; r += 4) {
                uint64_t xs[4];
#pragma unroll
                for (int u = 0; u < 4; u++) {
                    xs[u] = xr;
                    xr = ((xr | ~rest) + 1) & rest;
                }
                float2 v[4];
#pragma unroll
                for (int u = 0; u < 4; u++)
                    v[u] = r + u < nrest ? st2[xy | xs[u]] : make_float2(0.f, 0.f);
#pragma unroll
                for (int u = 0; u < 4; u++) {
                    if (r + u >= nrest) break;
                    const float2 amp = v[u];
                    const float pr = amp.x * amp.x, pi = amp.y * amp.y;
                    lo += fmaf(amp.x, amp.x, -pr) + fmaf(amp.y, amp.y, -pi);
                    two_sum(pr);
                    two_sum(pi);
                }
            }
            const double acc = (double)hi + (double)lo;
            tot += acc;
            if (acc > best || (acc == best && y < bidx)) {
                best = acc;
                bidx = y;
            }
        }
        s_val[tid] = best;
        s_idx[tid] = bidx;
        s_tot[tid] = tot;
        __syncthreads();
        for (int w = kT2Threads / 2; w; w >>= 1) {
            if (tid < w) {
                const double v2 = s_val[tid + w];
                const uint64_t i2 = s_idx[tid + w];
                if (v2 > s_val[tid] || (v2 == s_val[tid] && i2 < s_idx[tid])) {
                    s_val[tid] = v2;
                    s_idx[tid] = i2;
                }
                s_tot[tid] += s_tot[tid + w];
            }
            __syncthreads();
        }
        if (tid == 0) {
            B.out_idx[I.out] = s_idx[0];
            B.out_p[I.out] = s_tot[0] > 0.0 ? s_val[0] / s_tot[0] : 0.0;
        }
        __syncthreads();
    };
    for (;;) {
        if (tid == 0) s_item = atomicAdd(B.queue, 1);
        __syncthreads();
        const int item = s_item;
        __syncthreads();
        if (item >= B.nwork) break;
        const int4 wk = __ldg(B.work + item);
        const BatchInst &I = B.inst[wk.x];
        float *state = states + 2 * I.state_off;
        const int kind = wk.y & 15, p = wk.y >> 4;
        const bool whole = kind == kBatchWhole;
        if (whole && I.npass == 0) {  // empty circuit: |0...0>
            float4 *sv4 = reinterpret_cast<float4 *>(state);
            for (uint64_t v = tid; v < (UINT64_C(1) << I.nphys) / 2; v += blockDim.x)
                sv4[v] = make_float4(v == 0 ? 1.f : 0.f, 0.f, 0.f, 0.f);
            __syncthreads();
        }
        if (!whole) {  // a large instance: wait for the pass this item reads (all of its tiles)
            const int dep = kind == kBatchTiles ? (p > 0 ? I.pass0 + p - 1 : -1) : I.pass0 + I.npass - 1;
            bool ok = true;
            if (tid == 0 && dep >= 0)
                ok = wait_count(B.done + dep, (unsigned)B.passes[I.pass0].ntiles, B.err);
            if (__syncthreads_or(!ok)) {
                if (tid == 0) atomicExch(B.err, 1);
                return;
            }
        }
        // passes [q0, q1): every pass of a whole instance, one pass's tile
        // range of a large one (one call site keeps the programme loop
        // inlined once)
        const int q0 = whole ? 0 : p, q1 = whole ? I.npass : kind == kBatchTiles ? p + 1 : p;
        for (int q = q0; q < q1; q++) {
            const T2Args &ga = B.passes[I.pass0 + q];
            if (!run_tiles(ga, state, whole ? 0 : (uint64_t)wk.z, whole ? ga.ntiles : (uint64_t)wk.w)) return;
        }
        if (kind == kBatchTiles) {
            if (tid == 0) {  // every thread's stores precede the barrier that ended run_tiles
                __threadfence();
                atomicAdd(B.done + I.pass0 + p, (unsigned)wk.w);
            }
            continue;
        }
        readout(I, state);
    }
}

// e^{2 pi i x} for x = j/2^8, j/2^16, j/2^24, j/2^32 (j < 256): FP64 sincospi, then rounded.
__global__ void k_phase_tables(float2 *t) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= kTabEntries) return;
    const int l = i / kTabN, j = i % kTabN;
    const double x = (double)j * ldexp(1.0, -8 * (l + 1));
    double s, c;
    sincospi(2.0 * x, &s, &c);
    t[i] = make_float2((float)c, (float)s);
}

}  // namespace

size_t t2_smem_bytes() { return kSmemBytes; }

size_t t2_slotv_bytes(const T2Pass &p, int n) {
    if (p.slots.empty() || p.wide) return 0;
    const size_t nsp = (p.slots.size() + 1) & ~(size_t)1;
    const size_t bytes = ((size_t)1 << (n - p.k)) * nsp * sizeof(float2);
    return bytes <= kSlotvMaxBytes ? bytes : 0;
}

int t2_gate_kinds(const T2Pass &p) {
    int need = 0;
    for (const T2Ins &in : p.ins)
        need |= in.op == T2_X                             ? kFeatX
                : (in.op == T2_RGATE || in.op == T2_ROT) ? kFeatR
                : in.op == T2_GATE                        ? kFeatU
                                                          : 0;
    return need;
}

sv_status t2_prepare(sv_state *h) {
    if (h->t2_tables) return SV_OK;
    void *p = nullptr;
    if (dev_malloc(&p, kTabEntries * sizeof(float2) + 64) != cudaSuccess) {
        cudaGetLastError();
        return fail(SV_ERR_OOM, "cannot allocate phase tables");
    }
    h->t2_tables = p;
    h->t2_err = reinterpret_cast<int *>(reinterpret_cast<char *>(p) + kTabEntries * sizeof(float2));
    if (cudaMallocHost(&h->flag_host, sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        h->flag_host = nullptr;
        return fail(SV_ERR_OOM, "cannot allocate the pinned error word");
    }
    *h->flag_host = 0;
    SV_CUDA(cudaMemsetAsync(h->t2_err, 0, sizeof(int), h->stream));
    k_phase_tables<<<(kTabEntries + 255) / 256, 256, 0, h->stream>>>(reinterpret_cast<float2 *>(p));
    SV_CUDA(cudaGetLastError());
    note_launch();
    static bool configured = false;
    if (!configured) {
        for (auto kern : {k_tile2<13, 0>, k_tile2<13, kFeatX>, k_tile2<13, kFeatR>, k_tile2<13, kFeatAll>})
            SV_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)Geo<13>::kSmemBytes));
        for (auto kern : {k_tile2<14, 0>, k_tile2<14, kFeatX>, k_tile2<14, kFeatR>, k_tile2<14, kFeatAll>})
            SV_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)Geo<14>::kSmemBytes));
        for (auto kern : {k_group<0>, k_group<kFeatX>, k_group<kFeatR>, k_group<kFeatAll>})
            SV_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)Geo<13>::kSmemBytes));
        configured = true;
    }
    return SV_OK;
}

void t2_fill_args(const T2Pass &p, const T2Device &d, int n, T2Args *a) {
    a->gmask = p.gmask;
    a->ntiles = UINT64_C(1) << (n - p.k);
    a->c = p.c;
    a->nins = (int)p.ins.size();
    a->nfac = (int)p.fac2.size();
    a->nrows = (int)((p.wide ? p.statc64.size() : p.statc.size()) / (2 * (size_t)p.threads));
    a->nslots = (int)p.slots.size();
    a->nmats = (int)(p.wide ? p.mats64.size() / 8 : p.mats.size());
    a->nstages = (int)p.stages.size();
    a->last_stage = p.last_stage;
    for (int s = 0; s < p.k; s++) a->slot_phys[s] = p.slot_phys[s];
    // runs of the global bits: tile index bit i is the i-th lowest set bit of gmask
    a->ngr = 0;
    int ti = 0;
    const uint64_t gm = p.gmask & ((n >= 64) ? ~UINT64_C(0) : ((UINT64_C(1) << n) - 1));
    for (int b = 0; b < n;) {
        if (!((gm >> b) & 1)) {
            b++;
            continue;
        }
        int e = b;
        while (e < n && ((gm >> e) & 1)) e++;
        a->gs[a->ngr] = (int8_t)ti;
        a->gd[a->ngr] = (int8_t)b;
        a->gl[a->ngr] = (int8_t)(e - b);
        a->ngr++;
        ti += e - b;
        b = e;
    }
    a->ins = reinterpret_cast<const int4 *>(d.ins);
    a->stages = reinterpret_cast<const int4 *>(d.stages);
    a->mats = reinterpret_cast<const float4 *>(d.mats);
    a->fac = reinterpret_cast<const int4 *>(d.fac);
    a->statc = reinterpret_cast<const float2 *>(d.statc);
    a->soff = d.soff;
    a->sterms = d.sterms;
    a->layx = d.layx;
    a->epi = d.epi;
}

bool t2_block_runs(T2Args *a, uint64_t gmask, uint64_t bmask, int n) {
    const uint64_t all = n >= 64 ? ~UINT64_C(0) : ((UINT64_C(1) << n) - 1);
    int pos[64], np = 0;
    for (int q = 0; q < n; q++)
        if (((gmask & bmask & all) >> q) & 1) pos[np++] = q;
    for (int q = 0; q < n; q++)
        if (((gmask & ~bmask & all) >> q) & 1) pos[np++] = q;
    a->ngr = 0;
    for (int i = 0; i < np;) {
        int e = i + 1;
        while (e < np && pos[e] == pos[e - 1] + 1) e++;
        if (a->ngr == 32) return false;
        a->gs[a->ngr] = (int8_t)i;
        a->gd[a->ngr] = (int8_t)pos[i];
        a->gl[a->ngr] = (int8_t)(e - i);
        a->ngr++;
        i = e;
    }
    return true;
}

void t2_set_gen(const T2Pass &p, int64_t gen_basis, uint64_t basis_h, T2Args *a) {
    // the programme's leading Hadamards P (unnormalised, tile bits) applied
    // to the recorded product state H^{hq}|basis> (normalised Hadamards on
    // the physical qubits of hq): on a qubit in both they give sqrt(2) I, so
    // the generated state has Hadamards on P xor hq (its global ones decide
    // presence and sign per tile) and magnitude 2^{(|P and hq| - |hq without P|) / 2}
    a->gen = 1;
    a->gen_basis = (uint64_t)gen_basis;
    a->gen_local = 0;
    uint32_t hq_local = 0;
    for (int s = 0; s < p.k; s++) {
        a->gen_local |= (int)((a->gen_basis >> p.slot_phys[s]) & 1) << s;
        if ((basis_h >> p.slot_phys[s]) & 1) hq_local |= 1u << s;
    }
    a->gen_hmask = p.gen_hmask ^ hq_local;
    a->gen_ghmask = basis_h & p.gmask;
    const int both = __builtin_popcount(p.gen_hmask & hq_local);
    const int hq_only = __builtin_popcountll(basis_h) - both;
    a->gen_val64 = std::pow(2.0, 0.5 * (both - hq_only)) * p.gen_scale;
    a->gen_val = (float)a->gen_val64;
}

sv_status t2_launch(sv_state *h, const T2Pass &p, const T2Device &d, const sv_launch_record &meta,
                    int64_t gen_basis) {
    if (p.format != 2) return fail(SV_ERR_ARG, "internal: register-stage pass not in format 2");
    SV_TRY(launch_check());
    T2Args a{};
    t2_fill_args(p, d, h->n, &a);
    if (gen_basis >= 0) t2_set_gen(p, gen_basis, h->basis_h, &a);
    a.tables = reinterpret_cast<const float2 *>(h->t2_tables);
    a.err = h->t2_err;
    if (p.k != 13 && p.k != 14) return fail(SV_ERR_ARG, "internal: register-stage tile of 2^%d", p.k);
    // the tiles' slot values, computed ahead into the handle's buffer (sized
    // by t2_slotv_bytes before the first launch of the call)
    const size_t sbytes = t2_slotv_bytes(p, h->n);
    if (sbytes && sbytes <= h->slotv_cap) {
        a.nsp = (int)((p.slots.size() + 1) & ~(size_t)1);
        a.slotv = reinterpret_cast<const float2 *>(h->slotv);
        const uint64_t total = a.ntiles * (uint64_t)a.nsp;
        const unsigned blocks = (unsigned)std::min<uint64_t>((total + 255) / 256, (uint64_t)h->sm_count * 8);
        k_slotv<<<blocks, 256, 0, h->stream>>>(a, reinterpret_cast<float2 *>(h->slotv));
        SV_CUDA(cudaGetLastError());
        note_launch();
    }
    // the smallest instantiation whose gate kinds cover the programme
    const int need = t2_gate_kinds(p);
    auto kern = need == 0 ? k_tile2<13, 0>
              : need == kFeatX ? k_tile2<13, kFeatX>
              : need == kFeatR ? k_tile2<13, kFeatR>
                               : k_tile2<13, kFeatAll>;
    if (p.k == 14)
        kern = need == 0 ? k_tile2<14, 0>
             : need == kFeatX ? k_tile2<14, kFeatX>
             : need == kFeatR ? k_tile2<14, kFeatR>
                              : k_tile2<14, kFeatAll>;
    const int threads = p.k == 13 ? Geo<13>::kThreads : Geo<14>::kThreads;
    const size_t smem = p.k == 13 ? Geo<13>::kSmemBytes : Geo<14>::kSmemBytes;
    int per_sm = 0;
    SV_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem));
    if (per_sm < 1) return fail(SV_ERR_UNSUPPORTED, "register-stage tile kernel does not fit");
    h->stats.ctas_per_sm = h->stats.ctas_per_sm ? std::min(h->stats.ctas_per_sm, per_sm) : per_sm;
    const uint64_t grid = std::min<uint64_t>(a.ntiles, (uint64_t)per_sm * h->sm_count);
    const int slot = prof_begin(h);
    kern<<<(unsigned)grid, threads, smem, h->stream>>>(reinterpret_cast<float *>(h->amps), a);
    SV_CUDA(cudaGetLastError());
    note_launch();
    prof_end(h, slot, meta);
    h->stats.kernels++;
    return SV_OK;
}

sv_status t2_group_launch(sv_state *h, const GroupArgs &g, int need, const sv_launch_record &meta) {
    SV_TRY(launch_check());
    auto kern = need == 0 ? k_group<0>
              : need == kFeatX ? k_group<kFeatX>
              : need == kFeatR ? k_group<kFeatR>
                               : k_group<kFeatAll>;
    int per_sm = 0;
    SV_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kT2Threads, kSmemBytes));
    if (per_sm < 1) return fail(SV_ERR_UNSUPPORTED, "L2 block kernel does not fit on an SM");
    h->stats.ctas_per_sm = h->stats.ctas_per_sm ? std::min(h->stats.ctas_per_sm, per_sm) : per_sm;
    const uint64_t grid = std::min<uint64_t>(g.nitems, (uint64_t)per_sm * h->sm_count);
    const int slot = prof_begin(h);
    kern<<<(unsigned)grid, kT2Threads, kSmemBytes, h->stream>>>(reinterpret_cast<float *>(h->amps), g);
    SV_CUDA(cudaGetLastError());
    note_launch();
    prof_end(h, slot, meta);
    h->stats.kernels++;
    return SV_OK;
}

sv_status t2_build_tables(void **tables, int **err, cudaStream_t stream) {
    void *p = nullptr;
    if (dev_malloc(&p, kTabEntries * sizeof(float2) + 64) != cudaSuccess) {
        cudaGetLastError();
        return fail(SV_ERR_OOM, "cannot allocate phase tables");
    }
    *tables = p;
    *err = reinterpret_cast<int *>(reinterpret_cast<char *>(p) + kTabEntries * sizeof(float2));
    SV_CUDA(cudaMemsetAsync(*err, 0, sizeof(int), stream));
    k_phase_tables<<<(kTabEntries + 255) / 256, 256, 0, stream>>>(reinterpret_cast<float2 *>(p));
    SV_CUDA(cudaGetLastError());
    note_launch();
    return SV_OK;
}

sv_status t2_batch_launch(float *states, const BatchArgs &b, int sm_count, cudaStream_t stream) {
    static bool configured = false;
    if (!configured) {
        for (auto kern : {k_batch<0>, k_batch<kFeatX>, k_batch<kFeatR>, k_batch<kFeatAll>})
            SV_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemBytes));
        configured = true;
    }
    // the smallest instantiation whose gate kinds cover every programme
    auto kern = b.need == 0 ? k_batch<0>
              : b.need == kFeatX ? k_batch<kFeatX>
              : b.need == kFeatR ? k_batch<kFeatR>
                                 : k_batch<kFeatAll>;
    int per_sm = 0;
    SV_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kT2Threads, kSmemBytes));
    if (per_sm < 1) return fail(SV_ERR_UNSUPPORTED, "batched kernel does not fit on an SM");
    const int grid = std::max(1, std::min(b.nwork, per_sm * sm_count));
    kern<<<grid, kT2Threads, kSmemBytes, stream>>>(states, b);
    SV_CUDA(cudaGetLastError());
    note_launch();
    return SV_OK;
}

}  // namespace sv
