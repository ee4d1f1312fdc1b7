// Register-stage tile kernel, complex128 (tiles of 2^13 amplitudes), running
// the same format-2 programmes as the complex64 kernel (tileprog.h), compiled
// with 64-bit phases and FP64 values (compile_t2v2_c128).
//
// Per tile (persistent grid, one CTA per SM, 256 threads, 32 amplitudes per
// thread held as 64 FP64 registers):
//   1. one warp issues 2^(13-c) bulk copies of the tile's 2^c-amplitude chunks
//      into shared memory (128 KiB), completing on an mbarrier;
//   2. the tile's slot values (its global-qubit phase terms, Sec. III-B) are
//      summed as exact 64-bit phases while the copies are in flight and
//      turned into e^{2 pi i u / 2^64} from three FP64-generated tables;
//   3. the stage programme runs: every gate is thread-local FP64 arithmetic
//      on a register bit; a stage change goes through shared memory in the
//      swizzled order of tileprog.h applied to amplitude indices; diagonal
//      runs multiply by per-thread factors (static FP64 rows x tile slots)
//      and 32-entry FP64 tables; once the last stage change has read shared
//      memory, the next tile's copies start;
//   4. each thread writes its amplitudes from registers (16-byte stores).
// Hadamards are unnormalised ([[1,1],[1,-1]]) with one multiplication by
// 2^(-h/2) at the end of the pass; every per-amplitude operation is FP64, so
// the arithmetic per touched amplitude is that of the gates' definitions
// with the diagonal runs' phases merged exactly in integers.
#include <algorithm>

#include "common.h"
#include "plan.h"
#include "stagecomp.h"
#include "tiledev.cuh"
#include "tileprog.h"

namespace sv {
namespace {

using namespace tiledev;

constexpr int kR = 32;           // amplitudes per thread
constexpr int kDThreads = 256;   // 2^13 / 32
constexpr int kDWarps = kDThreads / 32;
constexpr int kTabBits = 18;     // the complex128 phase tables: 3 levels of 2^18
constexpr uint64_t kTabMask = (UINT64_C(1) << kTabBits) - 1;

// Shared-memory layout of a CTA (one per SM).
struct GD {
    static constexpr size_t kTileBytes = (size_t)16 << kT2Qubits;
    static constexpr size_t kOffRows = kTileBytes;
    static constexpr size_t kOffMats = kOffRows + (size_t)kT2SmemRows * kDThreads * 16;
    static constexpr size_t kOffFac = kOffMats + (size_t)kT2SmemMats * 64;
    static constexpr size_t kOffIns = kOffFac + (size_t)kT2SmemFactors * 16;
    static constexpr size_t kOffSlotc = kOffIns + (size_t)kT2SmemIns * 16;  // two buffers
    static constexpr size_t kOffLay = kOffSlotc + 2 * (size_t)kT2MaxSlots * 16;
    static constexpr size_t kOffEpi = kOffLay + (size_t)kT2SmemStages * sizeof(T2LayoutX);
    static constexpr size_t kOffOnes = kOffEpi + sizeof(T2Epilogue);  // the identity table
    static constexpr size_t kOffBar = kOffOnes + 32 * 16;
    static constexpr size_t kSmemBytes = kOffBar + 16;
};
static_assert(GD::kSmemBytes + 1024 <= 228 * 1024, "one CTA per SM");

struct RegsD {
    double re[kR], im[kR];
};

// Swizzled slot of amplitude index t in a stage change (tileprog.h's swz on
// 16-byte vectors): linear over GF(2), so a layout's slot is the XOR of its
// parts' slots.
__device__ __forceinline__ int swz_d(int t) { return t ^ (((t >> 3) ^ (t >> 6) ^ (t >> 9) ^ (t >> 12)) & 7); }

// Amplitude index (linear order) of register r in a stage layout, for thread tid.
struct LayD {
    int b, s1, s2, s3, s4;
    __device__ LayD(const T2LayoutX *x, int tid) {
        b = (int)x->lo[tid & 31] + (int)x->hi[tid >> 5];
        s1 = x->s[0];
        s2 = x->s[1];
        s3 = x->s[2];
        s4 = x->s[3];
    }
    __device__ int idx(int r) const {
        return b + (r & 1) + ((r & 2) ? s1 : 0) + ((r & 4) ? s2 : 0) + ((r & 8) ? s3 : 0) + ((r & 16) ? s4 : 0);
    }
};

// The same positions, swizzled.
struct LaySD {
    int b, p1, p2, p3, p4;
    __device__ LaySD(const T2LayoutX *x, int tid) {
        b = swz_d((int)x->lo[tid & 31] + (int)x->hi[tid >> 5]);
        p1 = swz_d(x->s[0]);
        p2 = swz_d(x->s[1]);
        p3 = swz_d(x->s[2]);
        p4 = swz_d(x->s[3]);
    }
    __device__ int idx(int r) const {  // swz(1) = 1
        return b ^ (r & 1) ^ ((r & 2) ? p1 : 0) ^ ((r & 4) ? p2 : 0) ^ ((r & 8) ? p3 : 0) ^ ((r & 16) ? p4 : 0);
    }
};

__device__ __forceinline__ double2 cxd(double2 a, double2 b) {
    return make_double2(fma(-a.y, b.y, a.x * b.x), fma(a.x, b.y, a.y * b.x));
}

// Register r0 of butterfly g (g = 0..15) on register bit J: g with a 0 inserted at bit J.
template <int J>
__device__ __forceinline__ constexpr int lo_of(int g) {
    return ((g >> J) << (J + 1)) | (g & ((1 << J) - 1));
}

// Uncontrolled gates on register bit J.  The 16 butterflies go in four groups
// of four; `qm` is all ones at run time and testing one of its bits per group
// keeps each group a separate block, which bounds the registers live at once.
template <int J>
__device__ __forceinline__ void d_h(RegsD &r, uint32_t qm) {
#pragma unroll
    for (int g4 = 0; g4 < 4; g4++) {
        if (!((qm >> g4) & 1)) continue;
#pragma unroll
        for (int i = 0; i < 4; i++) {
            const int a = lo_of<J>(4 * g4 + i), b = a | (1 << J);
            const double ar = r.re[a], ai = r.im[a];
            r.re[a] = ar + r.re[b];
            r.im[a] = ai + r.im[b];
            r.re[b] = ar - r.re[b];
            r.im[b] = ai - r.im[b];
        }
    }
}

template <int J>
__device__ __forceinline__ void d_x(RegsD &r, uint32_t qm) {
#pragma unroll
    for (int g4 = 0; g4 < 4; g4++) {
        if (!((qm >> g4) & 1)) continue;
#pragma unroll
        for (int i = 0; i < 4; i++) {
            const int a = lo_of<J>(4 * g4 + i), b = a | (1 << J);
            double t = r.re[a];
            r.re[a] = r.re[b];
            r.re[b] = t;
            t = r.im[a];
            r.im[a] = r.im[b];
            r.im[b] = t;
        }
    }
}

// General 2x2 m = (U11, U12, U21, U22) as (re, im) pairs.
__device__ __forceinline__ void d_u_pair(RegsD &r, int a, int b, const double *m) {
    const double ar = r.re[a], ai = r.im[a], br = r.re[b], bi = r.im[b];
    r.re[a] = fma(-m[3], bi, fma(m[2], br, fma(-m[1], ai, m[0] * ar)));
    r.im[a] = fma(m[3], br, fma(m[2], bi, fma(m[1], ar, m[0] * ai)));
    r.re[b] = fma(-m[7], bi, fma(m[6], br, fma(-m[5], ai, m[4] * ar)));
    r.im[b] = fma(m[7], br, fma(m[6], bi, fma(m[5], ar, m[4] * ai)));
}

template <int J>
__device__ __forceinline__ void d_u(RegsD &r, uint32_t qm, const double *m) {
#pragma unroll
    for (int g4 = 0; g4 < 4; g4++) {
        if (!((qm >> g4) & 1)) continue;
#pragma unroll
        for (int i = 0; i < 4; i++) {
            const int a = lo_of<J>(4 * g4 + i);
            d_u_pair(r, a, a | (1 << J), m);
        }
    }
}

// Real 2x2 [[a, b], [c, d]] = (m[0], m[2], m[4], m[6]).
template <int J>
__device__ __forceinline__ void d_r(RegsD &r, uint32_t qm, const double *m) {
    const double ma = m[0], mb = m[2], mc = m[4], md = m[6];
#pragma unroll
    for (int g4 = 0; g4 < 4; g4++) {
        if (!((qm >> g4) & 1)) continue;
#pragma unroll
        for (int i = 0; i < 4; i++) {
            const int a = lo_of<J>(4 * g4 + i), b = a | (1 << J);
            const double ar = r.re[a], ai = r.im[a], br = r.re[b], bi = r.im[b];
            r.re[a] = fma(mb, br, ma * ar);
            r.im[a] = fma(mb, bi, ma * ai);
            r.re[b] = fma(md, br, mc * ar);
            r.im[b] = fma(md, bi, mc * ai);
        }
    }
}

// Rotation [[c, -s], [s, c]] as three shears a += t b, b += s a, a += t b
// (m[0] = t, m[1] = s), the same factorisation as the complex64 kernel.
template <int J>
__device__ __forceinline__ void d_rot(RegsD &r, uint32_t qm, const double *m) {
    const double t = m[0], s = m[1];
#pragma unroll
    for (int g4 = 0; g4 < 4; g4++) {
        if (!((qm >> g4) & 1)) continue;
#pragma unroll
        for (int i = 0; i < 4; i++) {
            const int a = lo_of<J>(4 * g4 + i), b = a | (1 << J);
            r.re[a] = fma(r.re[b], t, r.re[a]);
            r.im[a] = fma(r.im[b], t, r.im[a]);
            r.re[b] = fma(r.re[a], s, r.re[b]);
            r.im[b] = fma(r.im[a], s, r.im[b]);
            r.re[a] = fma(r.re[b], t, r.re[a]);
            r.im[a] = fma(r.im[b], t, r.im[a]);
        }
    }
}

// General 2x2 on register bit J for the pairs whose packed-pair index (r >> 1
// of the lower register) is in `pm`, and with `odd` only for odd registers
// (a control on register bit 0).
template <int J>
__device__ __forceinline__ void d_u_ctrl(RegsD &r, uint32_t pm, bool odd, const double *m) {
#pragma unroll
    for (int g = 0; g < 16; g++) {
        const int a = lo_of<J>(g);
        if (!((pm >> (a >> 1)) & 1)) continue;
        if (odd && !(a & 1)) continue;
        d_u_pair(r, a, a | (1 << J), m);
    }
}

// Amplitude x of the register index times entry x of a 32-entry table.
__device__ __forceinline__ void d_table(RegsD &r, const double2 *T, uint32_t qm) {
#pragma unroll
    for (int g4 = 0; g4 < 8; g4++) {
        if (!((qm >> g4) & 1)) continue;
#pragma unroll
        for (int i = 0; i < 4; i++) {
            const int x = 4 * g4 + i;
            const double2 t = T[x];
            const double re = r.re[x], im = r.im[x];
            r.re[x] = fma(-im, t.y, re * t.x);
            r.im[x] = fma(re, t.y, im * t.x);
        }
    }
}

// Amplitudes whose register index has every bit of M set, times f.
template <int M>
__device__ __forceinline__ void d_factor(RegsD &r, double2 f) {
#pragma unroll
    for (int x = 0; x < kR; x++) {
        if ((x & M) != M) continue;
        const double re = r.re[x], im = r.im[x];
        r.re[x] = fma(-im, f.y, re * f.x);
        r.im[x] = fma(re, f.y, im * f.x);
    }
}

__device__ __forceinline__ void d_factor_bit(RegsD &r, int mask, double2 f) {
    switch (mask) {
        case 0: d_factor<0>(r, f); break;
        case 1: d_factor<1>(r, f); break;
        case 2: d_factor<2>(r, f); break;
        case 4: d_factor<4>(r, f); break;
        case 8: d_factor<8>(r, f); break;
        default: d_factor<16>(r, f); break;
    }
}

// Phased Hadamard on register bit J: b <- M b with M = f T[x_b], then the
// pair becomes (a + M b, a - M b).  Without a table (`tab` false) M = f.
template <int J>
__device__ __forceinline__ void d_hph(RegsD &r, uint32_t qm, const double2 *T, bool tab, double2 f,
                                      bool shared) {
    if constexpr (J <= 3) {
        if (tab && shared) {
            // the table depends only on register bits below J (kT2HphShared):
            // the 2^J products F T, once, then one product per pair
            constexpr int NV = 1 << J;
            double2 u[NV];
#pragma unroll
            for (int v = 0; v < NV; v++) u[v] = cxd(f, T[v | NV]);
#pragma unroll
            for (int g8 = 0; g8 < 2; g8++) {
                if (!((qm >> g8) & 1)) continue;
#pragma unroll
                for (int i = 0; i < 8; i++) {
                    const int a = lo_of<J>(8 * g8 + i), b = a | (1 << J);
                    const double2 m = u[b & (NV - 1)];
                    const double br = r.re[b], bi = r.im[b];
                    const double pr = fma(-bi, m.y, br * m.x), pi = fma(br, m.y, bi * m.x);
                    const double ar = r.re[a], ai = r.im[a];
                    r.re[a] = ar + pr;
                    r.im[a] = ai + pi;
                    r.re[b] = ar - pr;
                    r.im[b] = ai - pi;
                }
            }
            return;
        }
    }
#pragma unroll
    for (int g8 = 0; g8 < 2; g8++) {
        if (!((qm >> g8) & 1)) continue;
#pragma unroll
        for (int i = 0; i < 8; i++) {
            const int a = lo_of<J>(8 * g8 + i), b = a | (1 << J);
            const double2 m = tab ? cxd(f, T[b]) : f;
            const double br = r.re[b], bi = r.im[b];
            const double pr = fma(-bi, m.y, br * m.x), pi = fma(br, m.y, bi * m.x);
            const double ar = r.re[a], ai = r.im[a];
            r.re[a] = ar + pr;
            r.im[a] = ai + pi;
            r.re[b] = ar - pr;
            r.im[b] = ai - pi;
        }
    }
}

template <int F, int KIND, int SLOT>
__device__ __forceinline__ void d_gate(RegsD &r, const double *m, uint32_t qm) {
    constexpr int need = KIND == 0 ? 0 : KIND == 1 ? 1 : KIND == 4 ? 4 : 2;  // kFeat* of tile2.cu
    if constexpr ((need & F) != need) {
        return;
    } else if constexpr (KIND == 0) {
        d_h<SLOT>(r, qm);
    } else if constexpr (KIND == 1) {
        d_x<SLOT>(r, qm);
    } else if constexpr (KIND == 2) {
        d_r<SLOT>(r, qm, m);
    } else if constexpr (KIND == 3) {
        d_rot<SLOT>(r, qm, m);
    } else {
        d_u<SLOT>(r, qm, m);
    }
}

extern __shared__ __align__(1024) unsigned char t2d_smem[];

// One tile of the pass: stages, gates, runs, and the write-back.
template <int F, typename Hook>
__device__ __forceinline__ void t2d_run(const T2Args &a, double2 *gstate, uint64_t *rbar, uint32_t &rd, uint64_t base,
                                        const double2 *slotc, Hook hook) {
    const int4 *ins = reinterpret_cast<const int4 *>(t2d_smem + GD::kOffIns);
    const int4 *fac = reinterpret_cast<const int4 *>(t2d_smem + GD::kOffFac);
    const double2 *rows = reinterpret_cast<const double2 *>(t2d_smem + GD::kOffRows);
    const double2 *M = reinterpret_cast<const double2 *>(t2d_smem + GD::kOffMats);  // 4 per record
    const T2LayoutX *lays = reinterpret_cast<const T2LayoutX *>(t2d_smem + GD::kOffLay);
    const double2 *ones = reinterpret_cast<const double2 *>(t2d_smem + GD::kOffOnes);
    double2 *tile = reinterpret_cast<double2 *>(t2d_smem);
    const double2 *statc = reinterpret_cast<const double2 *>(a.statc);
    const int tid = threadIdx.x;
    auto layout = [&](int st) -> const T2LayoutX * { return st < kT2SmemStages ? lays + st : a.layx + st; };
    RegsD r;
    int stage = 0;
    bool live = false;
    auto thread_factor = [&](const int4 fd) -> double2 {
        const uint32_t w0 = (uint32_t)fd.x;
        const int sl = (int16_t)(fd.y & 0xffff), dsl = (int16_t)((uint32_t)fd.y >> 16);
        double2 f = make_double2(1.0, 0.0);
        if (fd.z >= 0)
            f = fd.z < kT2SmemRows ? rows[fd.z * kDThreads + tid] : statc[(size_t)fd.z * kDThreads + tid];
        if (sl >= 0) f = cxd(f, slotc[sl]);
        const uint32_t dmask = (w0 >> kFacDynShift) & 0x1ffu;
        uint32_t dm = dmask & (uint32_t)tid;
        while (dm) {
            const int t = __ffs(dm) - 1;
            dm &= dm - 1;
            f = cxd(f, slotc[dsl + __popc(dmask & ((1u << t) - 1u))]);
        }
        return f;
    };
    auto hph_run = [&](const int4 w, const double2 *&T, double2 &ph) {
        const int e0 = (int16_t)(w.z & 0xffff), e1 = (int16_t)(w.z >> 16);
        T = ones;
        ph = make_double2(1.0, 0.0);
        for (int e = e0; e < e1; e++) {
            const int4 fd = fac[e];
            if ((uint32_t)fd.x & kFacTable)
                T = M + 4 * fd.z;
            else
                ph = thread_factor(fd);
        }
    };
    // the same from the step itself (tileprog.h: kT2HphDirect, kT2HphShared)
    auto hph_direct = [&](const int4 w, const double2 *&T, double2 &ph) {
        const int trec = (int)((uint32_t)w.w & 0xffffu) - 1, row = (int)((uint32_t)w.w >> 16) - 1;
        const int sl = (int16_t)(w.y & 0xffff);
        T = trec >= 0 ? M + 4 * trec : ones;
        ph = make_double2(1.0, 0.0);
        if (row >= 0) ph = row < kT2SmemRows ? rows[row * kDThreads + tid] : statc[(size_t)row * kDThreads + tid];
        if (sl >= 0) ph = cxd(ph, slotc[sl]);
    };
    const int nins = a.nins, last_stage = a.last_stage;
    for (int pc = 0; pc < nins; pc++) {
        const int4 w = ins[pc];
        const uint32_t qm = ~((uint32_t)w.y >> 24);  // all ones at run time, opaque to the compiler
        const double *mrec = reinterpret_cast<const double *>(M + 4 * w.w);
        switch (((uint32_t)w.y >> 16) & 0xffu) {
            case kT2HdStage: {
                if (live) {
                    // every warp has read the previous layout before any overwrites it
                    if (!mbar_wait(rbar, (rd - 1u) & 1u)) atomicExch(a.err, 1);
                    const LaySD L(layout(stage), tid);
#pragma unroll
                    for (int x = 0; x < kR; x++) tile[L.idx(x)] = make_double2(r.re[x], r.im[x]);
                    __syncthreads();
                    stage = w.w;
                    const LaySD L2(layout(stage), tid);
#pragma unroll
                    for (int x = 0; x < kR; x++) {
                        const double2 v = tile[L2.idx(x)];
                        r.re[x] = v.x;
                        r.im[x] = v.y;
                    }
                } else {
                    stage = w.w;
                    const LayD L(layout(stage), tid);
                    if (a.gen) {
                        // the product state H^{hq}|b>, generated (see the complex64 kernel)
                        const bool has = ((a.gen_basis ^ base) & a.gmask & ~a.gen_ghmask) == 0;
                        const uint32_t gneg = (uint32_t)__popcll(base & a.gen_basis & a.gen_ghmask) & 1u;
                        const uint32_t gl = (uint32_t)a.gen_local, hm = a.gen_hmask;
                        const double v = a.gen_val64;
#pragma unroll
                        for (int x = 0; x < kR; x++) {
                            const uint32_t i = (uint32_t)L.idx(x);
                            double val = 0.0;
                            if (has && !((i ^ gl) & ~hm)) val = ((__popc(i & gl & hm) ^ gneg) & 1) ? -v : v;
                            r.re[x] = val;
                            r.im[x] = 0.0;
                        }
                    } else {  // the bulk copies' linear order
#pragma unroll
                        for (int x = 0; x < kR; x++) {
                            const double2 v = tile[L.idx(x)];
                            r.re[x] = v.x;
                            r.im[x] = v.y;
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
                const double s = mrec[0];
#pragma unroll
                for (int x = 0; x < kR; x++) {
                    r.re[x] *= s;
                    r.im[x] *= s;
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
                        d_table(r, M + 4 * fd.z, qm);
                        continue;
                    }
                    d_factor_bit(r, (int)(w0 & 0xffu), thread_factor(fd));
                }
                continue;
            }
#define SV_HPH_CASE(J)                  \
    case kT2Handler + 8 * 5 + J: {      \
        const double2 *T;               \
        double2 ph;                     \
        const int8_t hc = (int8_t)(w.x >> 24); \
        if (hc == kT2HphDirect || hc == kT2HphShared) \
            hph_direct(w, T, ph);       \
        else                            \
            hph_run(w, T, ph);          \
        d_hph<J>(r, qm, T, T != ones, ph, hc == kT2HphShared); \
        continue;                       \
    }
            SV_HPH_CASE(0)
            SV_HPH_CASE(1)
            SV_HPH_CASE(2)
            SV_HPH_CASE(3)
            SV_HPH_CASE(4)
#undef SV_HPH_CASE
#define SV_GATE_CASES(K)                                                   \
    case kT2Handler + 8 * K + 0: d_gate<F, K, 0>(r, mrec, qm); continue;   \
    case kT2Handler + 8 * K + 1: d_gate<F, K, 1>(r, mrec, qm); continue;   \
    case kT2Handler + 8 * K + 2: d_gate<F, K, 2>(r, mrec, qm); continue;   \
    case kT2Handler + 8 * K + 3: d_gate<F, K, 3>(r, mrec, qm); continue;   \
    case kT2Handler + 8 * K + 4: d_gate<F, K, 4>(r, mrec, qm); continue;
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
                if constexpr ((F & 6) != 0) {
                    const uint32_t pm = (uint32_t)w.z & 0xffffu;
                    const bool odd = ((uint32_t)w.z >> 16) != 0;
                    switch (j) {
                        case 0: d_u_ctrl<0>(r, pm, odd, mrec); break;
                        case 1: d_u_ctrl<1>(r, pm, odd, mrec); break;
                        case 2: d_u_ctrl<2>(r, pm, odd, mrec); break;
                        case 3: d_u_ctrl<3>(r, pm, odd, mrec); break;
                        default: d_u_ctrl<4>(r, pm, odd, mrec); break;
                    }
                }
                continue;
            }
#define SV_CTRL_CASE(K)                                   \
    if (kind == K) {                                      \
        switch (j) {                                      \
            case 0: d_gate<F, K, 0>(r, mrec, qm); break;  \
            case 1: d_gate<F, K, 1>(r, mrec, qm); break;  \
            case 2: d_gate<F, K, 2>(r, mrec, qm); break;  \
            case 3: d_gate<F, K, 3>(r, mrec, qm); break;  \
            default: d_gate<F, K, 4>(r, mrec, qm); break; \
        }                                                 \
        continue;                                         \
    }
            SV_CTRL_CASE(2)
            SV_CTRL_CASE(4)
#undef SV_CTRL_CASE
        }
    }
    if (!live) return;
    const T2Epilogue *E = reinterpret_cast<const T2Epilogue *>(t2d_smem + GD::kOffEpi);
    const uint64_t g0 = base + E->glo[tid & 31] + E->ghi[tid >> 5];
    const uint64_t g1 = E->g[0], g2 = E->g[1], g3 = E->g[2], g4 = E->g[3];
#pragma unroll
    for (int x = 0; x < kR; x++) {
        const uint64_t g = g0 + (uint64_t)(x & 1) + ((x & 2) ? g1 : 0) + ((x & 4) ? g2 : 0) +
                           ((x & 8) ? g3 : 0) + ((x & 16) ? g4 : 0);
        __stcs(gstate + g, make_double2(r.re[x], r.im[x]));
    }
}

__device__ __forceinline__ uint64_t tile_base_d(const T2Args &a, uint64_t tile) {
    uint64_t b = 0;
    for (int i = 0; i < a.ngr; i++)
        b |= ((tile >> a.gs[i]) & ((UINT64_C(1) << a.gl[i]) - 1)) << a.gd[i];
    return b;
}

__device__ __forceinline__ void issue_tile_load_d(const T2Args &a, unsigned char *sm, const double2 *state,
                                                  uint64_t tile, uint64_t *bar, int tid) {
    const int nchunks = 1 << (kT2Qubits - a.c);
    const uint32_t chunk_bytes = 16u << a.c;
    const uint64_t base = tile_base_d(a, tile);
    if (tid == 0) {
        fence_async_smem();
        mbar_expect_tx(bar, (uint32_t)GD::kTileBytes);
    }
    __syncwarp();
    for (int j = tid; j < nchunks; j += 32) {
        uint64_t off = 0;
        for (int b = 0; b < kT2Qubits - a.c; b++)
            if ((j >> b) & 1) off |= UINT64_C(1) << a.slot_phys[a.c + b];
        bulk_g2s(sm + (size_t)j * chunk_bytes, state + base + off, chunk_bytes, bar);
    }
}

__device__ __forceinline__ void load_programme_d(const T2Args &a, unsigned char *sm, int tid, int nthreads) {
    int4 *si = reinterpret_cast<int4 *>(sm + GD::kOffIns);
    int4 *sf = reinterpret_cast<int4 *>(sm + GD::kOffFac);
    double2 *sr = reinterpret_cast<double2 *>(sm + GD::kOffRows);
    double2 *smat = reinterpret_cast<double2 *>(sm + GD::kOffMats);
    int4 *slay = reinterpret_cast<int4 *>(sm + GD::kOffLay);
    int4 *sepi = reinterpret_cast<int4 *>(sm + GD::kOffEpi);
    const double2 *mats = reinterpret_cast<const double2 *>(a.mats);
    const double2 *statc = reinterpret_cast<const double2 *>(a.statc);
    for (int i = tid; i < a.nins; i += nthreads) si[i] = __ldg(a.ins + i);
    for (int i = tid; i < a.nfac; i += nthreads) sf[i] = __ldg(a.fac + i);
    for (int i = tid; i < 4 * a.nmats; i += nthreads) smat[i] = __ldg(mats + i);
    const int nl = min(a.nstages, kT2SmemStages) * (int)(sizeof(T2LayoutX) / 16);
    for (int i = tid; i < nl; i += nthreads) slay[i] = __ldg(reinterpret_cast<const int4 *>(a.layx) + i);
    for (int i = tid; i < (int)(sizeof(T2Epilogue) / 16); i += nthreads)
        sepi[i] = __ldg(reinterpret_cast<const int4 *>(a.epi) + i);
    const int nr = min(a.nrows, kT2SmemRows) * kDThreads;
    for (int i = tid; i < nr; i += nthreads) sr[i] = __ldg(statc + i);
    double2 *ones = reinterpret_cast<double2 *>(sm + GD::kOffOnes);
    for (int i = tid; i < 32; i += nthreads) ones[i] = make_double2(1.0, 0.0);
}

// The tile's slot values: each warp sums the 64-bit phase terms of its slots
// over its lanes (exact integer arithmetic), and one lane forms e^{2 pi i u /
// 2^64} as the product of three FP64 table entries (levels 2^-18, 2^-36,
// 2^-54 of a turn).
__device__ __forceinline__ void tile_slots_d(const T2Args &a, double2 *slotc, uint64_t base, int tid) {
    const int warp = tid >> 5, lane = tid & 31;
    const T2SlotTerm64 *sterms = reinterpret_cast<const T2SlotTerm64 *>(a.sterms);
    const double2 *tab = reinterpret_cast<const double2 *>(a.tables);
    for (int sl = warp; sl < a.nslots; sl += kDWarps) {
        const int t0 = __ldg(a.soff + sl), t1 = __ldg(a.soff + sl + 1);
        unsigned long long u = 0;
        for (int t = t0 + lane; t < t1; t += 32) {
            const T2SlotTerm64 st = sterms[t];
            bool on = (base >> st.g0) & 1;
            if (st.g1 >= 0) on = on && ((base >> st.g1) & 1);
            if (on) u += st.theta;
        }
#pragma unroll
        for (int o = 16; o; o >>= 1) u += __shfl_xor_sync(0xffffffffu, u, o);
        if (lane == 0) {
            const double2 x = __ldg(tab + (u >> 46));
            const double2 y = __ldg(tab + (UINT64_C(1) << kTabBits) + ((u >> 28) & kTabMask));
            const double2 z = __ldg(tab + (UINT64_C(2) << kTabBits) + ((u >> 10) & kTabMask));
            slotc[sl] = cxd(cxd(x, y), z);
        }
    }
}

// Persistent CTA over the pass's tiles; tile i+1's copies start once tile i's
// last stage change has read shared memory.
template <int F>
__global__ void __launch_bounds__(kDThreads, 1) k_tile2d(double2 *__restrict__ state, const T2Args a) {
    extern __shared__ __align__(1024) unsigned char sm[];
    double2 *slotc = reinterpret_cast<double2 *>(sm + GD::kOffSlotc);
    uint64_t *bar = reinterpret_cast<uint64_t *>(sm + GD::kOffBar);
    uint64_t *rbar = bar + 1;
    const int tid = threadIdx.x;
    load_programme_d(a, sm, tid, blockDim.x);
    if (tid == 0) {
        mbar_init(bar, 1);
        mbar_init(rbar, kDWarps);
        fence_mbar_init();
    }
    __syncthreads();
    if (!a.gen && tid < 32 && (uint64_t)blockIdx.x < a.ntiles)
        issue_tile_load_d(a, sm, state, blockIdx.x, bar, tid);
    uint32_t parity = 0, rd = 0, buf = 0;
    for (uint64_t tile = blockIdx.x; tile < a.ntiles; tile += gridDim.x) {
        const uint64_t next = tile + gridDim.x;
        const uint64_t base = tile_base_d(a, tile);
        double2 *sc = slotc + buf * kT2MaxSlots;
        tile_slots_d(a, sc, base, tid);
        const bool timed_out = a.gen ? false : !mbar_wait(bar, parity);
        if (__syncthreads_or(timed_out)) {
            if (tid == 0) atomicExch(a.err, 1);
            mbar_wait(bar, parity);  // a second bounded wait for copies in flight
            return;
        }
        auto hook = [&]() {
            if (!a.gen && tid < 32 && next < a.ntiles) {
                if (!mbar_wait(rbar, (rd - 1u) & 1u)) atomicExch(a.err, 1);
                issue_tile_load_d(a, sm, state, next, bar, tid);
            }
        };
        t2d_run<F>(a, state, rbar, rd, base, sc, hook);
        parity ^= 1u;
        buf ^= 1u;
    }
}

}  // namespace

sv_status t2d_launch(sv_state *h, const T2Pass &p, const T2Device &d, const sv_launch_record &meta,
                     int64_t gen_basis) {
    if (p.format != 2 || !p.wide || p.k != kT2Qubits)
        return fail(SV_ERR_ARG, "internal: complex128 register-stage pass not compiled for it");
    SV_TRY(launch_check());
    static bool configured = false;
    if (!configured) {
        for (auto kern : {k_tile2d<0>, k_tile2d<1>, k_tile2d<2>, k_tile2d<7>})
            SV_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)GD::kSmemBytes));
        configured = true;
    }
    T2Args a{};
    t2_fill_args(p, d, h->n, &a);
    if (gen_basis >= 0) t2_set_gen(p, gen_basis, h->basis_h, &a);
    a.tables = reinterpret_cast<const float2 *>(h->tab64);
    a.err = h->t2_err;
    const int need = t2_gate_kinds(p);
    auto kern = need == 0 ? k_tile2d<0> : need == 1 ? k_tile2d<1> : need == 2 ? k_tile2d<2> : k_tile2d<7>;
    int per_sm = 0;
    SV_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kDThreads, GD::kSmemBytes));
    if (per_sm < 1) return fail(SV_ERR_UNSUPPORTED, "complex128 register-stage kernel does not fit");
    h->stats.ctas_per_sm = h->stats.ctas_per_sm ? std::min(h->stats.ctas_per_sm, per_sm) : per_sm;
    const uint64_t grid = std::min<uint64_t>(a.ntiles, (uint64_t)per_sm * h->sm_count);
    const int slot = prof_begin(h);
    kern<<<(unsigned)grid, kDThreads, GD::kSmemBytes, h->stream>>>(reinterpret_cast<double2 *>(h->amps), a);
    SV_CUDA(cudaGetLastError());
    note_launch();
    prof_end(h, slot, meta);
    h->stats.kernels++;
    return SV_OK;
}

}  // namespace sv
