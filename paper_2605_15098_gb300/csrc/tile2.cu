// Register-stage tile kernel (complex64, tiles of 2^13 amplitudes).
//
// Per tile (persistent grid, two CTAs per SM, 256 threads each, 32 amplitudes per thread):
//   1. one warp issues 2^(13-c) bulk copies (TMA, cp.async.bulk) of the
//      tile's contiguous 2^c-amplitude chunks into shared memory, completing
//      on an mbarrier;
//   2. the pass's per-tile diagonal data (global-qubit contributions, which
//      are constants of the tile: Sec. III-B of arxiv 2605.15098) is formed
//      while the copies are in flight;
//   3. the stage programme runs: each thread holds 32 amplitudes as 16
//      packed pairs (re and im of two neighbouring amplitudes), gates on
//      register bits are packed f32x2 arithmetic, gates on lane bits use
//      warp shuffles, a stage change goes through shared memory; once the
//      last stage change has read shared memory, the next tile's copies start;
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
    static constexpr uint32_t kTileBytes = 8u << K;
    static constexpr int kStatRows = kT2SmemStatRows;
    static constexpr size_t kOffTab = kTileBytes;
    static constexpr size_t kOffStat = kOffTab + (size_t)kTabEntries * 8;
    static constexpr size_t kOffFac = kOffStat + (size_t)kStatRows * kThreads * 4;
    static constexpr size_t kOffIns = kOffFac + (size_t)kT2SmemFactors * 16;
    static constexpr size_t kOffLin = kOffIns + (size_t)kT2SmemIns * 16;
    static constexpr size_t kOffCst = kOffLin + (size_t)kT2MaxRuns * 16 * 4;
    static constexpr size_t kOffBar = kOffCst + (size_t)kT2MaxRuns * 4;
    static constexpr size_t kSmemBytes = kOffBar + 16;
};
using G13 = Geo<13>;
constexpr uint32_t kTileBytes = G13::kTileBytes;
constexpr size_t kOffTab = G13::kOffTab;
constexpr size_t kOffLin = G13::kOffLin;
constexpr size_t kOffCst = G13::kOffCst;
constexpr size_t kOffBar = G13::kOffBar;
constexpr size_t kSmemBytes = G13::kSmemBytes;


// ---------------------------------------------------------------- the kernel
// Run a pass's programme (in shared memory) on the tile.  The first stage
// reads the tile from shared memory (interleaved complex64, local index
// order), or generates the recorded basis state.  After the last stage change
// has read shared memory, `hook()` runs (the callers start the next tile's
// bulk copies there).  The result goes straight from registers to the global
// state, at the offsets of the final layout's write-back record.

extern __shared__ __align__(1024) unsigned char t2_dyn_smem[];
__shared__ uint64_t t2_tile_base;  // physical index of the current tile's amplitude 0

// Float4 index (amplitude pair) of packed pair q in a stage layout, for
// thread tid, from the host-computed layout record.
struct Layout2 {
    int bt, s1, s2, s3, s4;
    __device__ Layout2(const T2LayoutX *x, int tid) {
        bt = (int)__ldg(&x->lo[tid & 31]) + (int)__ldg(&x->hi[tid >> 5]);
        const int4 sv = __ldg(reinterpret_cast<const int4 *>(x->s));
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

// Gate kinds an instantiation carries besides H and the diagonal runs (the
// host launches the smallest one that covers a pass's programme: every gate
// path in the loop costs registers and instructions in all the others).
constexpr int kFeatX = 1, kFeatR = 2, kFeatU = 4, kFeatAll = 7;

// Gate KIND (0..4: H, X, real 2x2, shear rotation, general 2x2) on register
// bit SLOT (0..4), or on lane bit l (SLOT 5; SLOT 6 with the thread
// predicate `pred`).  Kinds outside the instantiation's set F compile to
// nothing: the host never launches them there.
template <int F, int KIND, int SLOT, int NP>
__device__ __forceinline__ void run_gate(RegsN<NP> &r, const float4 *mrec, uint32_t qm, int l, bool pred) {
    constexpr int need = KIND == 0 ? 0 : KIND == 1 ? kFeatX : KIND == 4 ? kFeatU : kFeatR;
    if constexpr ((need & F) != need) {
        return;
    } else {
        float m[8] = {};
        if constexpr (KIND >= 2) {
            const float4 m0 = __ldg(mrec), m1 = __ldg(mrec + 1);
            m[0] = m0.x; m[1] = m0.y; m[2] = m0.z; m[3] = m0.w;
            m[4] = m1.x; m[5] = m1.y; m[6] = m1.z; m[7] = m1.w;
        }
        if constexpr (SLOT <= 4) {
            if constexpr (KIND == 0) reg_h2<SLOT>(r, qm);
            else if constexpr (KIND == 1) reg_x2<SLOT>(r, qm);
            else if constexpr (KIND == 2) reg_r2<SLOT>(r, qm, m);
            else if constexpr (KIND == 3) reg_rot<SLOT>(r, qm, m);
            else reg_u2<SLOT>(r, qm, m);
        } else if constexpr (KIND != 3) {
            constexpr int OP = KIND == 0 ? T2_H : KIND == 1 ? T2_X : KIND == 2 ? T2_RGATE : T2_GATE;
            lane_op3<OP, SLOT == 6>(r, l, pred, qm, m);
        }
    }
}

template <int K, int F, typename Hook>
__device__ __forceinline__ void t2_run(const T2Args &a, float4 *gstate, Hook hook) {
    using G = Geo<K>;
    // the programme: copied to shared memory by k_tile2 (once per CTA) and
    // k_batch (once per pass); static phase rows beyond the copy stay in global memory
    const int4 *ins = reinterpret_cast<const int4 *>(t2_dyn_smem + G::kOffIns);
    const int4 *fac = reinterpret_cast<const int4 *>(t2_dyn_smem + G::kOffFac);
    const uint32_t *stat = reinterpret_cast<const uint32_t *>(t2_dyn_smem + G::kOffStat);
    float4 *tile4 = reinterpret_cast<float4 *>(t2_dyn_smem);
    const float2 *tab = reinterpret_cast<const float2 *>(t2_dyn_smem + G::kOffTab);
    const uint32_t *lin = reinterpret_cast<const uint32_t *>(t2_dyn_smem + G::kOffLin);
    const uint32_t *cst = reinterpret_cast<const uint32_t *>(t2_dyn_smem + G::kOffCst);
    const int tid = threadIdx.x;
    RegsN<kNP2> r;
    int stage = 0;
    bool live = false;
    bool hooked = false;
    for (int pc = 0; pc < a.nins; pc++) {
        const int4 w = ins[pc];
        const int op = w.x & 0xff;
        // all ones at run time (the handler code is below 256), opaque to the
        // compiler (see reg_h2)
        const uint32_t qm = ~((uint32_t)w.y >> 24);
        if (op == T2_STAGE) {
            if (live) {
                const Layout2 L(a.layx + stage, tid);
#pragma unroll
                for (int q = 0; q < kNP2; q++)
                    tile4[L.idx(q)] = make_float4(r.re[q].x, r.re[q].y, r.im[q].x, r.im[q].y);
                __syncthreads();
            }
            stage = w.w;
            {
                const Layout2 L(a.layx + stage, tid);
                if (!live && a.gen) {
                    // the basis state |b>, after the leading Hadamards on the
                    // tile bits in gen_hmask (unnormalised: the closing scale
                    // holds their 2^(-1/2)), generated instead of read:
                    // +-1 where the index agrees with b off those bits, with
                    // the sign of the parity of b on them, 0 elsewhere
                    const bool has = (a.gen_basis & a.gmask) == t2_tile_base;
                    const uint32_t gl = (uint32_t)a.gen_local, hm = a.gen_hmask;
                    auto amp = [&](uint32_t i) -> float {
                        if (!has || ((i ^ gl) & ~hm)) return 0.f;
                        return (__popc(i & gl & hm) & 1) ? -1.f : 1.f;
                    };
#pragma unroll
                    for (int q = 0; q < kNP2; q++) {
                        const uint32_t i0 = 2u * (uint32_t)L.idx(q);
                        r.re[q] = make_float2(amp(i0), amp(i0 + 1));
                        r.im[q] = make_float2(0.f, 0.f);
                    }
                } else {
#pragma unroll
                    for (int q = 0; q < kNP2; q++) {
                        const float4 v = tile4[L.idx(q)];
                        if (live) {
                            r.re[q] = make_float2(v.x, v.y);
                            r.im[q] = make_float2(v.z, v.w);
                        } else {
                            r.re[q] = make_float2(v.x, v.z);
                            r.im[q] = make_float2(v.y, v.w);
                        }
                    }
                }
            }
            live = true;
            if (pc == a.last_stage) {
                __syncthreads();  // every thread has read shared memory
                hook();
                hooked = true;
            }
            continue;
        }
        if (op == T2_SCALE) {
            const float4 mm = __ldg(a.mats + 2 * w.w);
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
        // e^{2 pi i u / 2^32} for this thread's phase u of a per-thread factor
        auto thread_phase = [&](const int4 fd) -> float2 {
            const uint32_t w0 = (uint32_t)fd.x;
            const int run = fd.y;
            uint32_t u = fd.z >= G::kStatRows ? __ldg(a.stat + fd.z * G::kThreads + tid)
                                              : stat[fd.z * G::kThreads + tid];
            if (w0 & 0x200u) u += cst[run];
            const int lr = (int)((w0 >> kFacLinShift) & 0x1fu) - 1;
            if (lr >= 0) u += lin[run * 16 + lr];
            uint32_t dm = (w0 >> kFacDynShift) & 0x1ffu & (uint32_t)tid;
            while (dm) {
                const int t = __ffs(dm) - 1;
                dm &= dm - 1;
                const int8_t *tbp = reinterpret_cast<const int8_t *>(a.stages + stage);
                u += lin[run * 16 + tbp[5 + t]];
            }
            return cx(cx(tab[u >> 24], tab[kTabN + ((u >> 16) & 255u)]),
                      cx(tab[2 * kTabN + ((u >> 8) & 255u)], tab[3 * kTabN + (u & 255u)]));
        };
        if (op == T2_HPH) {  // diagonal run + H on register bit j in one sweep (stage compiler)
            const int e0 = (int16_t)(w.z & 0xffff), e1 = (int16_t)(w.z >> 16);
            const float4 *T = nullptr;
            float2 ph = make_float2(1.f, 0.f);
            for (int e = e0; e < e1; e++) {
                const int4 fd = fac[e];
                if ((uint32_t)fd.x & kFacTable)
                    T = a.mats + 2 * fd.z;
                else
                    ph = thread_phase(fd);
            }
            switch ((w.x >> 16) & 0xff) {
                case 0: reg_hph<0>(r, qm, T, ph.x, ph.y); break;
                case 1: reg_hph<1>(r, qm, T, ph.x, ph.y); break;
                case 2: reg_hph<2>(r, qm, T, ph.x, ph.y); break;
                case 3: reg_hph<3>(r, qm, T, ph.x, ph.y); break;
                default: reg_hph<4>(r, qm, T, ph.x, ph.y); break;
            }
            continue;
        }
        if (op == T2_DIAG) {
            const int e0 = (int16_t)(w.z & 0xffff), e1 = (int16_t)(w.z >> 16);
            if (e0 >= e1) continue;
            for (int e = e0; e < e1; e++) {
                const int4 fd = fac[e];
                const uint32_t w0 = (uint32_t)fd.x;
                const int run = fd.y;
                const int pb = (int)((w0 >> 10) & 0xfu);  // thread-bit predicate of a constant
                if (pb && !((tid >> (pb - 1)) & 1)) continue;  // not this thread's factor
                if (w0 & kFacTable) {
                    apply_table(r, a.mats + 2 * fd.z, qm);
                    continue;
                }
                // per-thread phase (constants are tables, see the stage compiler)
                const float2 ff = thread_phase(fd);
                apply_factor_bit(r, (int)(w0 & 0xffu), ff.x, ff.y);
            }
            continue;
        }
        if (op == T2_HG && a.gen) continue;  // included in the generated state
        // gates (no register-bit controls: the stage compiler never emits them);
        // one switch on the handler code the stage compiler set (tileprog.h)
        const int j = (int8_t)((w.x >> 16) & 0xff);
        const float4 *mrec = a.mats + 2 * w.w;
        switch (((uint32_t)w.y >> 16) & 0xffu) {
#define SV_GATE_CASES(K)                                                                 \
    case kT2Handler + 8 * K + 0: run_gate<F, K, 0>(r, mrec, qm, j, true); continue;     \
    case kT2Handler + 8 * K + 1: run_gate<F, K, 1>(r, mrec, qm, j, true); continue;     \
    case kT2Handler + 8 * K + 2: run_gate<F, K, 2>(r, mrec, qm, j, true); continue;     \
    case kT2Handler + 8 * K + 3: run_gate<F, K, 3>(r, mrec, qm, j, true); continue;     \
    case kT2Handler + 8 * K + 4: run_gate<F, K, 4>(r, mrec, qm, j, true); continue;     \
    case kT2Handler + 8 * K + 5: run_gate<F, K, 5>(r, mrec, qm, j, true); continue;     \
    case kT2Handler + 8 * K + 6:                                                         \
        run_gate<F, K, 6>(r, mrec, qm, j, (tid >> (int16_t)(w.y & 0xffff)) & 1); continue;
            SV_GATE_CASES(0)
            SV_GATE_CASES(1)
            SV_GATE_CASES(2)
            SV_GATE_CASES(3)
            SV_GATE_CASES(4)
#undef SV_GATE_CASES
            default: break;
        }
        {  // slot 7: a register-bit gate with a thread or tile control
            const int ccls = (w.x >> 24) & 0xff;
            const int cidx = (int16_t)(w.y & 0xffff);
            if (ccls == T2C_GLOBAL) {
                if (!((t2_tile_base >> cidx) & 1)) continue;  // tile-uniform
            } else if (ccls == T2C_THREAD) {
                if (!((tid >> cidx) & 1)) continue;
            }
            const int kind = ((((uint32_t)w.y >> 16) & 0xffu) - kT2Handler) >> 3;
            const bool lane = ((w.x >> 8) & 0xff) == T2C_LANE;
#define SV_CTRL_CASE(K)                                                                  \
    if (kind == K) {                                                                     \
        if (lane) {                                                                      \
            run_gate<F, K, 5>(r, mrec, qm, j, true);                                     \
        } else {                                                                         \
            switch (j) {                                                                 \
                case 0: run_gate<F, K, 0>(r, mrec, qm, j, true); break;                  \
                case 1: run_gate<F, K, 1>(r, mrec, qm, j, true); break;                  \
                case 2: run_gate<F, K, 2>(r, mrec, qm, j, true); break;                  \
                case 3: run_gate<F, K, 3>(r, mrec, qm, j, true); break;                  \
                default: run_gate<F, K, 4>(r, mrec, qm, j, true); break;                 \
            }                                                                            \
        }                                                                                \
        continue;                                                                        \
    }
            SV_CTRL_CASE(0)
            SV_CTRL_CASE(1)
            SV_CTRL_CASE(2)
            SV_CTRL_CASE(4)
#undef SV_CTRL_CASE
        }
    }
    if (!hooked) {  // a programme without a stage change still releases the buffer
        __syncthreads();
        hook();
    }
    if (!live) return;
    const T2Epilogue *E = a.epi;
    const uint64_t g0 = t2_tile_base + __ldg(&E->glo[tid & 31]) + __ldg(&E->ghi[tid >> 5]);
    const uint64_t g1 = __ldg(&E->g[0]), g2 = __ldg(&E->g[1]), g3 = __ldg(&E->g[2]), g4 = __ldg(&E->g[3]);
#pragma unroll
    for (int q = 0; q < kNP2; q++) {
        const uint64_t g = g0 + ((q & 1) ? g1 : 0) + ((q & 2) ? g2 : 0) + ((q & 4) ? g3 : 0) +
                           ((q & 8) ? g4 : 0);
        __stcs(gstate + (g >> 1), make_float4(r.re[q].x, r.im[q].x, r.re[q].y, r.im[q].y));
    }
}

template <int K>
__device__ __forceinline__ void issue_tile_load(const T2Args &a, unsigned char *sm, const float *state,
                                                uint64_t tile, uint64_t *bar, int tid) {
    const int nchunks = 1 << (K - a.c);
    const uint32_t chunk_bytes = 8u << a.c;
    const uint64_t base = pdep(tile, a.gmask);
    if (tid == 0) {
        fence_async_smem();
        mbar_expect_tx(bar, Geo<K>::kTileBytes);
    }
    __syncwarp();
    for (int j = tid; j < nchunks; j += 32) {
        uint64_t off = 0;
        for (int b = 0; b < K - a.c; b++)
            if ((j >> b) & 1) off |= UINT64_C(1) << a.slot_phys[a.c + b];
        bulk_g2s(sm + (size_t)j * chunk_bytes, state + 2 * (base + off), chunk_bytes, bar);
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
    float4 *tile4 = reinterpret_cast<float4 *>(sm);
    float2 *tab = reinterpret_cast<float2 *>(sm + G::kOffTab);
    uint32_t *lin = reinterpret_cast<uint32_t *>(sm + G::kOffLin);
    uint32_t *cst = reinterpret_cast<uint32_t *>(sm + G::kOffCst);
    uint64_t *bar = reinterpret_cast<uint64_t *>(sm + G::kOffBar);
    const int tid = threadIdx.x;

    for (int i = tid; i < kTabEntries; i += blockDim.x) tab[i] = a.tables[i];
    {  // the programme, once per CTA (sizes bounded by the stage compiler)
        int4 *si = reinterpret_cast<int4 *>(sm + G::kOffIns);
        int4 *sf = reinterpret_cast<int4 *>(sm + G::kOffFac);
        uint32_t *ss = reinterpret_cast<uint32_t *>(sm + G::kOffStat);
        for (int i = tid; i < a.nins; i += blockDim.x) si[i] = __ldg(a.ins + i);
        for (int i = tid; i < a.nfac; i += blockDim.x) sf[i] = __ldg(a.fac + i);
        const int nst = min(a.nstat, G::kStatRows * G::kThreads);
        for (int i = tid; i < nst; i += blockDim.x) ss[i] = __ldg(a.stat + i);
    }
    if (tid == 0) {
        mbar_init(bar, 1);
        fence_mbar_init();
    }
    __syncthreads();
    if (!a.gen && tid < 32 && (uint64_t)blockIdx.x < a.ntiles)
        issue_tile_load<K>(a, sm, state, blockIdx.x, bar, tid);

    uint32_t parity = 0;
    for (uint64_t tile = blockIdx.x; tile < a.ntiles; tile += gridDim.x) {
        const uint64_t next = tile + gridDim.x;
        // per-tile diagonal data while the copies are in flight (the barrier
        // first: the previous tile's programme may still read lin / cst);
        // one thread forms the tile's base index, the others read it back
        __syncthreads();
        for (int i = tid; i < a.nruns * 16; i += blockDim.x) lin[i] = 0u;
        for (int i = tid; i < a.nruns; i += blockDim.x) cst[i] = 0u;
        if (tid == 0) t2_tile_base = pdep(tile, a.gmask);
        __syncthreads();
        const uint64_t base = t2_tile_base;
        for (int i = tid; i < a.ntterms; i += blockDim.x) {
            const T2TileTerm t = a.tterms[i];
            bool on = (base >> t.g0) & 1;
            if (t.g1 >= 0) on = on && ((base >> t.g1) & 1);
            if (on) atomicAdd(t.tb >= 0 ? &lin[t.run * 16 + t.tb] : &cst[t.run], t.theta);
        }
        const bool timed_out = a.gen ? false : !mbar_wait(bar, parity);
        if (__syncthreads_or(timed_out)) {
            if (tid == 0) atomicExch(a.err, 1);
            mbar_wait(bar, parity);  // give copies still in flight a second bounded wait
            return;
        }
        auto hook = [&]() {
            if (!a.gen && tid < 32 && next < a.ntiles) issue_tile_load<K>(a, sm, state, next, bar, tid);
        };
        t2_run<K, F>(a, reinterpret_cast<float4 *>(state), hook);
        parity ^= 1u;
    }
}

// ---------------------------------------------------------------- batched instances
// One CTA runs whole instances taken from a shared queue (largest first): all
// passes of the instance (the first pass starts from |0...0> in shared memory
// instead of reading the state), then the FP64 argmax of the marginal over
// the instance's read-out qubits.  States of up to 2^20 amplitudes stay in L2.
template <int F>
__global__ void __launch_bounds__(kT2Threads, 2) k_batch(float *__restrict__ states, const BatchArgs B) {
    extern __shared__ __align__(1024) unsigned char sm[];
    float4 *tile4 = reinterpret_cast<float4 *>(sm);
    float2 *tab = reinterpret_cast<float2 *>(sm + kOffTab);
    uint32_t *lin = reinterpret_cast<uint32_t *>(sm + kOffLin);
    uint32_t *cst = reinterpret_cast<uint32_t *>(sm + kOffCst);
    uint64_t *bar = reinterpret_cast<uint64_t *>(sm + kOffBar);
    __shared__ int s_item;
    // read-out reduction scratch lives in the tile buffer (free after the last pass)
    double *s_val = reinterpret_cast<double *>(sm);
    uint64_t *s_idx = reinterpret_cast<uint64_t *>(sm + 8 * kT2Threads);
    double *s_tot = reinterpret_cast<double *>(sm + 16 * kT2Threads);
    const int tid = threadIdx.x;
    for (int i = tid; i < kTabEntries; i += blockDim.x) tab[i] = B.tables[i];
    if (tid == 0) {
        mbar_init(bar, 1);
        fence_mbar_init();
    }
    __syncthreads();
    uint32_t parity = 0;
    for (;;) {
        if (tid == 0) s_item = atomicAdd(B.queue, 1);
        __syncthreads();
        const int item = s_item;
        __syncthreads();
        if (item >= B.count) break;
        const BatchInst &I = B.inst[B.order[item]];
        float *state = states + 2 * I.state_off;
        if (I.npass == 0) {  // empty circuit: |0...0>
            float4 *sv4 = reinterpret_cast<float4 *>(state);
            for (uint64_t v = tid; v < (UINT64_C(1) << I.nphys) / 2; v += blockDim.x)
                sv4[v] = make_float4(v == 0 ? 1.f : 0.f, 0.f, 0.f, 0.f);
            __syncthreads();
        }
        for (int p = 0; p < I.npass; p++) {
            const T2Args &a = B.passes[I.pass0 + p];
            // the first pass generates |0...0> in registers; later passes read
            // the state with bulk copies, the next tile's issued as soon as
            // the current one's last stage change has read shared memory, and
            // write it straight from registers
            if (!a.gen && tid < 32) issue_tile_load<kT2Qubits>(a, sm, state, 0, bar, tid);
            {  // the pass's programme into shared memory (sizes bounded by the stage compiler)
                int4 *si = reinterpret_cast<int4 *>(sm + G13::kOffIns);
                int4 *sf = reinterpret_cast<int4 *>(sm + G13::kOffFac);
                uint32_t *ss = reinterpret_cast<uint32_t *>(sm + G13::kOffStat);
                for (int i = tid; i < a.nins; i += blockDim.x) si[i] = __ldg(a.ins + i);
                for (int i = tid; i < a.nfac; i += blockDim.x) sf[i] = __ldg(a.fac + i);
                const int nst = min(a.nstat, G13::kStatRows * G13::kThreads);
                for (int i = tid; i < nst; i += blockDim.x) ss[i] = __ldg(a.stat + i);
            }
            for (uint64_t tile = 0; tile < a.ntiles; tile++) {
                __syncthreads();  // the previous tile's programme may still read lin / cst
                for (int i = tid; i < a.nruns * 16; i += blockDim.x) lin[i] = 0u;
                for (int i = tid; i < a.nruns; i += blockDim.x) cst[i] = 0u;
                if (tid == 0) t2_tile_base = pdep(tile, a.gmask);
                __syncthreads();
                const uint64_t base = t2_tile_base;
                for (int i = tid; i < a.ntterms; i += blockDim.x) {
                    const T2TileTerm t = a.tterms[i];
                    bool on = (base >> t.g0) & 1;
                    if (t.g1 >= 0) on = on && ((base >> t.g1) & 1);
                    if (on) atomicAdd(t.tb >= 0 ? &lin[t.run * 16 + t.tb] : &cst[t.run], t.theta);
                }
                bool timed_out = false;
                if (!a.gen) {
                    timed_out = !mbar_wait(bar, parity);
                    parity ^= 1u;
                }
                if (__syncthreads_or(timed_out)) {
                    if (tid == 0) atomicExch(B.err, 1);
                    mbar_wait(bar, parity ^ 1u);  // a second bounded wait for copies in flight
                    return;
                }
                auto hook = [&]() {
                    if (!a.gen && tid < 32 && tile + 1 < a.ntiles)
                        issue_tile_load<kT2Qubits>(a, sm, state, tile + 1, bar, tid);
                };
                t2_run<kT2Qubits, F>(a, reinterpret_cast<float4 *>(state), hook);
            }
            // the next pass's bulk copies (and the read-out) see this pass's stores
            asm volatile("fence.proxy.async;" ::: "memory");
            __syncthreads();
        }
        // read-out: argmax (lowest index among ties) of the FP64 marginal over I.pos
        uint64_t mask = 0;
        for (int j = 0; j < I.m; j++) mask |= UINT64_C(1) << I.pos[j];
        const uint64_t all = (UINT64_C(1) << I.nphys) - 1;
        const uint64_t rest = all & ~mask;
        const uint64_t outcomes = UINT64_C(1) << I.m;
        double best = -1.0, tot = 0.0;
        uint64_t bidx = ~UINT64_C(0);
        for (uint64_t y = tid; y < outcomes; y += blockDim.x) {
            uint64_t xy = 0;
            for (int j = 0; j < I.m; j++)
                if ((y >> j) & 1) xy |= UINT64_C(1) << I.pos[j];
            // exact FP32 squares (product + fmaf remainder) summed as a
            // double-float pair: FP64-accurate without FP64 arithmetic
            float hi = 0.f, lo = 0.f;
            auto two_sum = [&](float b) {
                const float t = hi + b;
                const float bb = t - hi;
                lo += (hi - (t - bb)) + (b - bb);
                hi = t;
            };
            uint64_t xr = 0;
            do {
                const float2 amp = reinterpret_cast<const float2 *>(state)[xy | xr];
                const float pr = amp.x * amp.x, pi = amp.y * amp.y;
                lo += fmaf(amp.x, amp.x, -pr) + fmaf(amp.y, amp.y, -pi);
                two_sum(pr);
                two_sum(pi);
                xr = ((xr | ~rest) + 1) & rest;
            } while (xr);
            const double acc = (double)hi + (double)lo;
            tot += acc;
            if (acc > best) {
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
    if (cudaMalloc(&p, kTabEntries * sizeof(float2) + 64) != cudaSuccess) {
        cudaGetLastError();
        return fail(SV_ERR_OOM, "cannot allocate phase tables");
    }
    h->t2_tables = p;
    h->t2_err = reinterpret_cast<int *>(reinterpret_cast<char *>(p) + kTabEntries * sizeof(float2));
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
        configured = true;
    }
    return SV_OK;
}

sv_status t2_launch(sv_state *h, const T2Pass &p, const T2Device &d, const sv_launch_record &meta,
                    int64_t gen_basis) {
    T2Args a{};
    if (gen_basis >= 0) {
        a.gen = 1;
        a.gen_basis = (uint64_t)gen_basis;
        for (int s = 0; s < p.k; s++)
            a.gen_local |= (int)((a.gen_basis >> p.slot_phys[s]) & 1) << s;
        a.gen_hmask = p.gen_hmask;
    }
    a.gmask = p.gmask;
    a.ntiles = UINT64_C(1) << (h->n - p.k);
    a.c = p.c;
    a.nins = (int)p.ins.size();
    a.nfac = (int)p.factors.size();
    a.nstat = (int)p.stat.size();
    a.last_stage = p.last_stage;
    a.nruns = p.nruns;
    a.ntterms = (int)p.tterms.size();
    for (int s = 0; s < p.k; s++) a.slot_phys[s] = p.slot_phys[s];
    a.ins = reinterpret_cast<const int4 *>(d.ins);
    a.stages = reinterpret_cast<const int4 *>(d.stages);
    a.mats = reinterpret_cast<const float4 *>(d.mats);
    a.fac = reinterpret_cast<const int4 *>(d.fac);
    a.stat = d.stat;
    a.tterms = d.tterms;
    a.tables = reinterpret_cast<const float2 *>(h->t2_tables);
    a.err = h->t2_err;
    a.layx = d.layx;
    a.epi = d.epi;
    if (p.k != 13 && p.k != 14) return fail(SV_ERR_ARG, "internal: register-stage tile of 2^%d", p.k);
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
    const uint64_t grid = std::min<uint64_t>(a.ntiles, (uint64_t)per_sm * h->sm_count);
    const int slot = prof_begin(h);
    kern<<<(unsigned)grid, threads, smem, h->stream>>>(reinterpret_cast<float *>(h->amps), a);
    SV_CUDA(cudaGetLastError());
    note_launch();
    prof_end(h, slot, meta);
    h->stats.kernels++;
    return SV_OK;
}

sv_status t2_build_tables(void **tables, int **err, cudaStream_t stream) {
    void *p = nullptr;
    if (cudaMalloc(&p, kTabEntries * sizeof(float2) + 64) != cudaSuccess) {
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
    const int grid = std::max(1, std::min(b.count, per_sm * sm_count));
    kern<<<grid, kT2Threads, kSmemBytes, stream>>>(states, b);
    SV_CUDA(cudaGetLastError());
    note_launch();
    return SV_OK;
}

}  // namespace sv
