// Register-stage tile kernel (complex64, tiles of 2^13 amplitudes).
//
// Per tile (persistent grid, two CTAs per SM, 256 threads each):
//   1. one warp issues 2^(13-c) bulk copies (TMA, cp.async.bulk) of the
//      tile's contiguous 2^c-amplitude chunks into shared memory, completing
//      on an mbarrier;
//   2. the pass's per-tile diagonal data (global-qubit contributions, which
//      are constants of the tile: Sec. III-B of arxiv 2605.15098) is formed
//      while the copies are in flight;
//   3. the stage programme runs: each thread holds 32 amplitudes as 16
//      packed pairs (re and im of two neighbouring amplitudes), gates on
//      register bits are packed f32x2 arithmetic, gates on lane bits use
//      warp shuffles, a stage change goes through shared memory;
//   4. the tile is written back with bulk copies (TMA store).
// Hadamards are applied unnormalised ([[1,1],[1,-1]]) and the pass ends with
// one multiplication by 2^(-h/2), exact for even h, so the norm carries no
// bias from a rounded 1/sqrt(2).
#include <algorithm>

#include "common.h"
#include "plan.h"
#include "stagecomp.h"
#include "tileprog.h"

namespace sv {
namespace {

constexpr int kTileAmps = 1 << kT2Qubits;
constexpr uint32_t kTileBytes = kTileAmps * 8u;
constexpr int kTab0 = 2048, kTab1 = 2048, kTab2 = 1024;
constexpr int kTabEntries = kTab0 + kTab1 + kTab2;
constexpr size_t kOffTab = kTileBytes;
constexpr size_t kOffLin = kOffTab + (size_t)kTabEntries * 8;
constexpr size_t kOffCst = kOffLin + (size_t)kT2MaxRuns * 16 * 4;
constexpr size_t kOffBar = kOffCst + (size_t)kT2MaxRuns * 4;
constexpr size_t kSmemBytes = kOffBar + 16;
constexpr int kNP = 16;  // packed pairs per thread

struct T2Args {
    uint64_t gmask, ntiles;
    int c, nins, nruns, ntterms;
    int slot_phys[kMaxTileQubits];
    const int4 *ins;      // T2Ins records
    const int4 *stages;   // T2Stage records
    const float4 *mats;   // T2Mat records (two float4 each)
    const int4 *fac;      // T2Factor records
    const uint32_t *stat; // per-thread static phases
    const T2TileTerm *tterms;
    const float2 *tables;
    int *err;
};

// ---------------------------------------------------------------- PTX helpers
__device__ __forceinline__ uint32_t saddr(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(saddr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(saddr(bar)),
                 "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(saddr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ uint64_t now_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// Wait for the phase with a time limit (2 s); false on timeout.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = now_ns();
    while (!mbar_try_wait(bar, parity))
        if (now_ns() - t0 > 2000000000ull) return false;
    return true;
}
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            saddr(dst)),
        "l"(src), "r"(bytes), "r"(saddr(bar))
        : "memory");
}
__device__ __forceinline__ void bulk_s2g(void *dst, const void *src, uint32_t bytes) {
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst),
                 "r"(saddr(src)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_read() {
    asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
}
__device__ __forceinline__ void fence_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ uint64_t pdep(uint64_t v, uint64_t mask) {
    uint64_t r = 0;
    for (uint64_t b = 1; mask; b <<= 1) {
        const uint64_t low = mask & (~mask + 1);
        if (v & b) r |= low;
        mask &= mask - 1;
    }
    return r;
}

// ---------------------------------------------------------------- packed math
__device__ __forceinline__ float2 f2(float v) { return make_float2(v, v); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return fma2(b, f2(-1.f), a); }

// (re, im) of two amplitudes times the complex scalar (fr, fi)
__device__ __forceinline__ void cmul2(float2 &re, float2 &im, float fr, float fi) {
    const float2 nr = fma2(im, f2(-fi), mul2(re, f2(fr)));
    const float2 ni = fma2(im, f2(fr), mul2(re, f2(fi)));
    re = nr;
    im = ni;
}
__device__ __forceinline__ void cmul1(float &re, float &im, float fr, float fi) {
    const float nr = re * fr - im * fi;
    const float ni = re * fi + im * fr;
    re = nr;
    im = ni;
}
__device__ __forceinline__ float2 cx(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

struct Regs {
    float2 re[kNP], im[kNP];
};

// ---------------------------------------------------------------- register-bit gates
// Gate on register bit J >= 1: pairs of packed registers (q, q | 2^(J-1)).
// jc: controlling register bit or -1.
template <int J>
__device__ __forceinline__ void reg_h(Regs &r, int jc) {
#pragma unroll
    for (int q = 0; q < kNP; q++) {
        if constexpr (J >= 1) {
            constexpr int S = 1 << (J - 1);
            if (q & S) continue;
            const int q1 = q | S;
            if (jc >= 1 && !((q >> (jc - 1)) & 1)) continue;
            if (jc == 0) {
                const float ar = r.re[q].y, ai = r.im[q].y, br = r.re[q1].y, bi = r.im[q1].y;
                r.re[q].y = ar + br; r.im[q].y = ai + bi;
                r.re[q1].y = ar - br; r.im[q1].y = ai - bi;
                continue;
            }
            const float2 ar = r.re[q], ai = r.im[q], br = r.re[q1], bi = r.im[q1];
            r.re[q] = add2(ar, br); r.im[q] = add2(ai, bi);
            r.re[q1] = sub2(ar, br); r.im[q1] = sub2(ai, bi);
        } else {
            if (jc >= 1 && !((q >> (jc - 1)) & 1)) continue;
            const float2 a = r.re[q], b = r.im[q];
            r.re[q] = make_float2(a.x + a.y, a.x - a.y);
            r.im[q] = make_float2(b.x + b.y, b.x - b.y);
        }
    }
}

template <int J>
__device__ __forceinline__ void reg_x(Regs &r, int jc) {
#pragma unroll
    for (int q = 0; q < kNP; q++) {
        if constexpr (J >= 1) {
            constexpr int S = 1 << (J - 1);
            if (q & S) continue;
            const int q1 = q | S;
            if (jc >= 1 && !((q >> (jc - 1)) & 1)) continue;
            if (jc == 0) {
                float t = r.re[q].y; r.re[q].y = r.re[q1].y; r.re[q1].y = t;
                t = r.im[q].y; r.im[q].y = r.im[q1].y; r.im[q1].y = t;
                continue;
            }
            float2 t = r.re[q]; r.re[q] = r.re[q1]; r.re[q1] = t;
            t = r.im[q]; r.im[q] = r.im[q1]; r.im[q1] = t;
        } else {
            if (jc >= 1 && !((q >> (jc - 1)) & 1)) continue;
            r.re[q] = make_float2(r.re[q].y, r.re[q].x);
            r.im[q] = make_float2(r.im[q].y, r.im[q].x);
        }
    }
}

template <int J>
__device__ __forceinline__ void reg_u(Regs &r, int jc, const float *m) {
    const float u0r = m[0], u0i = m[1], u1r = m[2], u1i = m[3];
    const float u2r = m[4], u2i = m[5], u3r = m[6], u3i = m[7];
#pragma unroll
    for (int q = 0; q < kNP; q++) {
        if constexpr (J >= 1) {
            constexpr int S = 1 << (J - 1);
            if (q & S) continue;
            const int q1 = q | S;
            if (jc >= 1 && !((q >> (jc - 1)) & 1)) continue;
            if (jc == 0) {
                const float ar = r.re[q].y, ai = r.im[q].y, br = r.re[q1].y, bi = r.im[q1].y;
                r.re[q].y = u0r * ar - u0i * ai + u1r * br - u1i * bi;
                r.im[q].y = u0r * ai + u0i * ar + u1r * bi + u1i * br;
                r.re[q1].y = u2r * ar - u2i * ai + u3r * br - u3i * bi;
                r.im[q1].y = u2r * ai + u2i * ar + u3r * bi + u3i * br;
                continue;
            }
            const float2 ar = r.re[q], ai = r.im[q], br = r.re[q1], bi = r.im[q1];
            r.re[q] = fma2(bi, f2(-u1i), fma2(br, f2(u1r), fma2(ai, f2(-u0i), mul2(ar, f2(u0r)))));
            r.im[q] = fma2(br, f2(u1i), fma2(bi, f2(u1r), fma2(ar, f2(u0i), mul2(ai, f2(u0r)))));
            r.re[q1] = fma2(bi, f2(-u3i), fma2(br, f2(u3r), fma2(ai, f2(-u2i), mul2(ar, f2(u2r)))));
            r.im[q1] = fma2(br, f2(u3i), fma2(bi, f2(u3r), fma2(ar, f2(u2i), mul2(ai, f2(u2r)))));
        } else {
            if (jc >= 1 && !((q >> (jc - 1)) & 1)) continue;
            const float ar = r.re[q].x, ai = r.im[q].x, br = r.re[q].y, bi = r.im[q].y;
            r.re[q].x = u0r * ar - u0i * ai + u1r * br - u1i * bi;
            r.im[q].x = u0r * ai + u0i * ar + u1r * bi + u1i * br;
            r.re[q].y = u2r * ar - u2i * ai + u3r * br - u3i * bi;
            r.im[q].y = u2r * ai + u2i * ar + u3r * bi + u3i * br;
        }
    }
}

// ---------------------------------------------------------------- lane-bit gates (shuffles)
__device__ __forceinline__ void lane_gate(Regs &r, int op, int l, int jc, bool pred,
                                          const float *m) {
    const unsigned FULL = 0xffffffffu;
    const int xm = 1 << l;
    const bool hi = (threadIdx.x >> l) & 1;
    // coefficients for my output: mine * cs + partner * co
    const float csr = hi ? m[6] : m[0], csi = hi ? m[7] : m[1];
    const float cor = hi ? m[4] : m[2], coi = hi ? m[5] : m[3];
    const float sg = hi ? -1.f : 1.f;
#pragma unroll
    for (int q = 0; q < kNP; q++) {
        if (jc >= 1 && !((q >> (jc - 1)) & 1)) continue;
        float2 pr, pi;
        pr.x = __shfl_xor_sync(FULL, r.re[q].x, xm);
        pr.y = __shfl_xor_sync(FULL, r.re[q].y, xm);
        pi.x = __shfl_xor_sync(FULL, r.im[q].x, xm);
        pi.y = __shfl_xor_sync(FULL, r.im[q].y, xm);
        if (!pred) continue;
        float2 nr, ni;
        if (op == T2_H) {
            nr = fma2(r.re[q], f2(sg), pr);
            ni = fma2(r.im[q], f2(sg), pi);
        } else if (op == T2_X) {
            nr = pr;
            ni = pi;
        } else {
            nr = fma2(pi, f2(-coi), fma2(pr, f2(cor), fma2(r.im[q], f2(-csi), mul2(r.re[q], f2(csr)))));
            ni = fma2(pr, f2(coi), fma2(pi, f2(cor), fma2(r.re[q], f2(csi), mul2(r.im[q], f2(csr)))));
        }
        if (jc == 0) {  // control on register bit 0: odd element only
            r.re[q].y = nr.y;
            r.im[q].y = ni.y;
        } else {
            r.re[q] = nr;
            r.im[q] = ni;
        }
    }
}

// ---------------------------------------------------------------- diagonal factors
template <int M>
__device__ __forceinline__ void apply_factor(Regs &r, float fr, float fi) {
#pragma unroll
    for (int q = 0; q < kNP; q++) {
        if constexpr ((M & 1) != 0) {
            if (((2 * q + 1) & M) == M) cmul1(r.re[q].y, r.im[q].y, fr, fi);
        } else {
            if (((2 * q) & M) == M) cmul2(r.re[q], r.im[q], fr, fi);
        }
    }
}

__device__ __forceinline__ void apply_factor_any(Regs &r, int mask, float fr, float fi) {
    switch (mask) {
#define SV_FAC(M) \
    case M: apply_factor<M>(r, fr, fi); break;
        SV_FAC(0) SV_FAC(1) SV_FAC(2) SV_FAC(4) SV_FAC(8) SV_FAC(16)
        SV_FAC(3) SV_FAC(5) SV_FAC(6) SV_FAC(9) SV_FAC(10) SV_FAC(12)
        SV_FAC(17) SV_FAC(18) SV_FAC(20) SV_FAC(24)
#undef SV_FAC
        default: break;
    }
}

// ---------------------------------------------------------------- the kernel
__global__ void __launch_bounds__(kT2Threads, 2) k_tile2(float *__restrict__ state, const T2Args a) {
    extern __shared__ __align__(1024) unsigned char sm[];
    float4 *tile4 = reinterpret_cast<float4 *>(sm);
    float2 *tab = reinterpret_cast<float2 *>(sm + kOffTab);
    uint32_t *lin = reinterpret_cast<uint32_t *>(sm + kOffLin);
    uint32_t *cst = reinterpret_cast<uint32_t *>(sm + kOffCst);
    uint64_t *bar = reinterpret_cast<uint64_t *>(sm + kOffBar);
    const int tid = threadIdx.x;

    for (int i = tid; i < kTabEntries; i += blockDim.x) tab[i] = a.tables[i];
    if (tid == 0) {
        mbar_init(bar, 1);
        fence_mbar_init();
    }
    __syncthreads();

    const int nchunks = 1 << (kT2Qubits - a.c);
    const uint32_t chunk_bytes = 8u << a.c;
    uint32_t parity = 0;
    for (uint64_t tile = blockIdx.x; tile < a.ntiles; tile += gridDim.x) {
        const uint64_t base = pdep(tile, a.gmask);
        if (tid < 32) {
            if (tid == 0) {
                fence_async_smem();
                mbar_expect_tx(bar, kTileBytes);
            }
            __syncwarp();
            for (int j = tid; j < nchunks; j += 32) {
                uint64_t off = 0;
                for (int b = 0; b < kT2Qubits - a.c; b++)
                    if ((j >> b) & 1) off |= UINT64_C(1) << a.slot_phys[a.c + b];
                bulk_g2s(sm + (size_t)j * chunk_bytes, state + 2 * (base + off), chunk_bytes, bar);
            }
        }
        // per-tile diagonal data while the copies are in flight
        for (int i = tid; i < a.nruns * 16; i += blockDim.x) lin[i] = 0u;
        for (int i = tid; i < a.nruns; i += blockDim.x) cst[i] = 0u;
        __syncthreads();
        for (int i = tid; i < a.ntterms; i += blockDim.x) {
            const T2TileTerm t = a.tterms[i];
            bool on = (base >> t.g0) & 1;
            if (t.g1 >= 0) on = on && ((base >> t.g1) & 1);
            if (on) atomicAdd(t.tb >= 0 ? &lin[t.run * 16 + t.tb] : &cst[t.run], t.theta);
        }
        const bool timed_out = !mbar_wait(bar, parity);
        if (__syncthreads_or(timed_out)) {
            if (tid == 0) atomicExch(a.err, 1);
            mbar_wait(bar, parity);  // give copies still in flight a second bounded wait
            return;
        }

        Regs r;
        int bt = 0, s1 = 0, s2 = 0, s3 = 0, s4 = 0;  // current layout: thread base, register strides
        int stage = 0;
        bool live = false;
        auto sidx = [&](int q) {
            return (bt + ((q & 1) ? s1 : 0) + ((q & 2) ? s2 : 0) + ((q & 4) ? s3 : 0) +
                    ((q & 8) ? s4 : 0)) >> 1;
        };
        for (int pc = 0; pc < a.nins; pc++) {
            const int4 w = __ldg(a.ins + pc);
            const int op = w.x & 0xff;
            if (op == T2_STAGE) {
                if (live) {
#pragma unroll
                    for (int q = 0; q < kNP; q++)
                        tile4[sidx(q)] = make_float4(r.re[q].x, r.re[q].y, r.im[q].x, r.im[q].y);
                    __syncthreads();
                }
                stage = w.w;
                const int4 st = __ldg(a.stages + stage);
                auto tbyte = [&](int i) {
                    const int word = i < 4 ? st.x : i < 8 ? st.y : i < 12 ? st.z : st.w;
                    return (word >> (8 * (i & 3))) & 0xff;
                };
                bt = 0;
#pragma unroll
                for (int t = 0; t < 8; t++) bt |= ((tid >> t) & 1) << tbyte(5 + t);
                s1 = 1 << tbyte(1);
                s2 = 1 << tbyte(2);
                s3 = 1 << tbyte(3);
                s4 = 1 << tbyte(4);
#pragma unroll
                for (int q = 0; q < kNP; q++) {
                    const float4 v = tile4[sidx(q)];
                    if (live) {
                        r.re[q] = make_float2(v.x, v.y);
                        r.im[q] = make_float2(v.z, v.w);
                    } else {
                        r.re[q] = make_float2(v.x, v.z);
                        r.im[q] = make_float2(v.y, v.w);
                    }
                }
                live = true;
                continue;
            }
            if (op == T2_SCALE) {
                const float4 mm = __ldg(a.mats + 2 * w.w);
                const float hi = mm.x, lo = mm.y;
#pragma unroll
                for (int q = 0; q < kNP; q++) {
                    r.re[q] = fma2(r.re[q], f2(hi), mul2(r.re[q], f2(lo)));
                    r.im[q] = fma2(r.im[q], f2(hi), mul2(r.im[q], f2(lo)));
                }
                continue;
            }
            if (op == T2_DIAG) {
                const int e0 = (int16_t)(w.z & 0xffff), e1 = (int16_t)(w.z >> 16);
                for (int e = e0; e < e1; e++) {
                    const int4 fd = __ldg(a.fac + e);
                    const uint32_t w0 = (uint32_t)fd.x;
                    const int run = fd.y;
                    float fr, fi;
                    if (!(w0 & 0x100u)) {
                        fr = __int_as_float(fd.z);
                        fi = __int_as_float(fd.w);
                    } else {
                        uint32_t u = __ldg(a.stat + fd.z * 256 + tid);
                        if (w0 & 0x200u) u += cst[run];
                        const int lr = (int)((w0 >> 16) & 0xff) - 1;
                        if (lr >= 0) u += lin[run * 16 + lr];
                        uint32_t dm = (w0 >> 24) & (uint32_t)tid;
                        while (dm) {
                            const int t = __ffs(dm) - 1;
                            dm &= dm - 1;
                            const int8_t *tbp = reinterpret_cast<const int8_t *>(a.stages + stage);
                            u += lin[run * 16 + tbp[5 + t]];
                        }
                        const float2 f0 = tab[u >> 21];
                        const float2 f1 = tab[kTab0 + ((u >> 10) & 2047u)];
                        const float2 fz = tab[kTab0 + kTab1 + (u & 1023u)];
                        const float2 ff = cx(cx(f0, f1), fz);
                        fr = ff.x;
                        fi = ff.y;
                    }
                    apply_factor_any(r, (int)(w0 & 0xffu), fr, fi);
                }
                continue;
            }
            // gates
            const int cls = (w.x >> 8) & 0xff;
            const int j = (int8_t)((w.x >> 16) & 0xff);
            const int ccls = (w.x >> 24) & 0xff;
            const int cidx = (int16_t)(w.y & 0xffff);
            bool pred = true;
            int jc = -1;
            if (ccls == T2C_GLOBAL) {
                if (!((base >> cidx) & 1)) continue;  // tile-uniform
            } else if (ccls == T2C_THREAD) {
                pred = (tid >> cidx) & 1;
            } else if (ccls == T2C_REG) {
                jc = cidx;
            }
            float m[8];
            if (op == T2_GATE) {
                const float4 m0 = __ldg(a.mats + 2 * w.w), m1 = __ldg(a.mats + 2 * w.w + 1);
                m[0] = m0.x; m[1] = m0.y; m[2] = m0.z; m[3] = m0.w;
                m[4] = m1.x; m[5] = m1.y; m[6] = m1.z; m[7] = m1.w;
            } else {
#pragma unroll
                for (int e = 0; e < 8; e++) m[e] = 0.f;
            }
            if (cls == T2C_LANE) {
                lane_gate(r, op, j, jc, pred, m);
                continue;
            }
            if (!pred) continue;
            if (op == T2_H) {
                switch (j) {
                    case 0: reg_h<0>(r, jc); break;
                    case 1: reg_h<1>(r, jc); break;
                    case 2: reg_h<2>(r, jc); break;
                    case 3: reg_h<3>(r, jc); break;
                    default: reg_h<4>(r, jc); break;
                }
            } else if (op == T2_X) {
                switch (j) {
                    case 0: reg_x<0>(r, jc); break;
                    case 1: reg_x<1>(r, jc); break;
                    case 2: reg_x<2>(r, jc); break;
                    case 3: reg_x<3>(r, jc); break;
                    default: reg_x<4>(r, jc); break;
                }
            } else {
                switch (j) {
                    case 0: reg_u<0>(r, jc, m); break;
                    case 1: reg_u<1>(r, jc, m); break;
                    case 2: reg_u<2>(r, jc, m); break;
                    case 3: reg_u<3>(r, jc, m); break;
                    default: reg_u<4>(r, jc, m); break;
                }
            }
        }
        // epilogue: interleaved tile back to shared memory, then TMA store
        if (live) {
#pragma unroll
            for (int q = 0; q < kNP; q++)
                tile4[sidx(q)] = make_float4(r.re[q].x, r.im[q].x, r.re[q].y, r.im[q].y);
        }
        fence_async_smem();
        __syncthreads();
        if (tid < 32) {
            for (int j = tid; j < nchunks; j += 32) {
                uint64_t off = 0;
                for (int b = 0; b < kT2Qubits - a.c; b++)
                    if ((j >> b) & 1) off |= UINT64_C(1) << a.slot_phys[a.c + b];
                bulk_s2g(state + 2 * (base + off), sm + (size_t)j * chunk_bytes, chunk_bytes);
            }
            bulk_commit();
            bulk_wait_read();
        }
        __syncthreads();
        parity ^= 1u;
    }
}

// e^{2 pi i x} for x = j/2^11, j/2^22 (j < 2048) and j/2^32 (j < 1024), FP64 then rounded.
__global__ void k_phase_tables(float2 *t) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= kTabEntries) return;
    double x;
    if (i < kTab0)
        x = (double)i * 0x1p-11;
    else if (i < kTab0 + kTab1)
        x = (double)(i - kTab0) * 0x1p-22;
    else
        x = (double)(i - kTab0 - kTab1) * 0x1p-32;
    double s, c;
    sincospi(2.0 * x, &s, &c);
    t[i] = make_float2((float)c, (float)s);
}

}  // namespace

size_t t2_smem_bytes() { return kSmemBytes; }

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
        SV_CUDA(cudaFuncSetAttribute(k_tile2, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)kSmemBytes));
        configured = true;
    }
    return SV_OK;
}

sv_status t2_launch(sv_state *h, const T2Pass &p, const T2Device &d, const sv_launch_record &meta) {
    T2Args a{};
    a.gmask = p.gmask;
    a.ntiles = UINT64_C(1) << (h->n - p.k);
    a.c = p.c;
    a.nins = (int)p.ins.size();
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
    int per_sm = 0;
    SV_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_tile2, kT2Threads, kSmemBytes));
    if (per_sm < 1) return fail(SV_ERR_UNSUPPORTED, "register-stage tile kernel does not fit");
    const uint64_t grid = std::min<uint64_t>(a.ntiles, (uint64_t)per_sm * h->sm_count);
    const int slot = prof_begin(h);
    k_tile2<<<(unsigned)grid, kT2Threads, kSmemBytes, h->stream>>>(reinterpret_cast<float *>(h->amps), a);
    SV_CUDA(cudaGetLastError());
    note_launch();
    prof_end(h, slot, meta);
    h->stats.kernels++;
    return SV_OK;
}

}  // namespace sv
