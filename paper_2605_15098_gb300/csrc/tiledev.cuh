// Device helpers shared by the register-stage tile kernels (tile2.cu, tile3.cu):
// PTX wrappers for mbarriers and bulk (TMA) copies, packed f32x2 arithmetic,
// register-bit and lane-bit gates on a thread's 32 amplitudes, and diagonal
// factor application.  Included inside an anonymous namespace by each kernel.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "tileprog.h"

namespace sv {
namespace tiledev {

constexpr int kNP = 16;  // packed pairs per thread (32 amplitudes)

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
__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(saddr(bar)) : "memory");
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
// Order this thread's generic-proxy accesses of global memory with the bulk
// copies (async proxy) that follow.
__device__ __forceinline__ void fence_async_global() {
    asm volatile("fence.proxy.async.global;" ::: "memory");
}
__device__ __forceinline__ unsigned ld_acquire(const unsigned *p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
// Wait until *p >= want, with a time limit (2 s), giving up early once *err
// is set (another CTA gave up); false if it gave up.
__device__ __forceinline__ bool wait_count(const unsigned *p, unsigned want, const int *err) {
    if (ld_acquire(p) >= want) return true;
    const uint64_t t0 = now_ns();
    for (;;) {
        __nanosleep(128);
        if (ld_acquire(p) >= want) return true;
        if (*(volatile const int *)err) return false;
        if (now_ns() - t0 > 2000000000ull) return false;
    }
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
// Complex product with its rounding fixed (one product rounded, then a fused
// multiply-add), so that every kernel that forms a value with it gets the same
// bits whatever the compiler's contraction choices.
__device__ __forceinline__ float2 cx(float2 a, float2 b) {
    return make_float2(__fmaf_rn(a.x, b.x, __fmul_rn(-a.y, b.y)), __fmaf_rn(a.x, b.y, __fmul_rn(a.y, b.x)));
}

template <int NP>
struct RegsN {
    float2 re[NP], im[NP];
};
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

// Uncontrolled gates on register bit J for the register-stage kernel.  For
// J >= 1 the 8 butterflies (q, q | 2^(J-1)) are numbered b = 0..7 (q is b with
// a 0 inserted at bit J-1) and taken in two groups of four; `qm` is all ones
// at run time, and testing one of its bits per group keeps each group a
// separate block: four independent butterflies in flight, whatever J, which
// bounds the registers the compiler keeps live.  J = 0 acts inside each
// packed pair, in four groups of four pairs.
template <int J>
__device__ __forceinline__ constexpr int bfly_q(int b) {
    return ((b >> (J - 1)) << J) | (b & ((1 << (J - 1)) - 1));
}

// The butterfly runs in place, a' = a + b then b' = a' - 2b, so no register
// of the pair needs a copy and no operand needs negating; b' equals a - b up
// to one extra rounding of a + b.
template <int J, int NP>
__device__ __forceinline__ void reg_h2(RegsN<NP> &r, uint32_t qm) {
    if constexpr (J >= 1) {
#pragma unroll
        for (int g = 0; g < NP / 8; g++) {
            if (!((qm >> g) & 1)) continue;
#pragma unroll
            for (int i = 0; i < 4; i++) {
                const int q = bfly_q<J>(4 * g + i), q1 = q | (1 << (J - 1));
                r.re[q] = add2(r.re[q], r.re[q1]);
                r.im[q] = add2(r.im[q], r.im[q1]);
                r.re[q1] = fma2(r.re[q1], f2(-2.f), r.re[q]);
                r.im[q1] = fma2(r.im[q1], f2(-2.f), r.im[q]);
            }
        }
    } else {
#pragma unroll
        for (int g4 = 0; g4 < NP / 4; g4++) {
            if (!((qm >> g4) & 1)) continue;
#pragma unroll
            for (int i = 0; i < 4; i++) {
                const int q = 4 * g4 + i;
                const float2 a = r.re[q], b = r.im[q];
                r.re[q] = make_float2(a.x + a.y, a.x - a.y);
                r.im[q] = make_float2(b.x + b.y, b.x - b.y);
            }
        }
    }
}

template <int J, int NP>
__device__ __forceinline__ void reg_x2(RegsN<NP> &r, uint32_t qm) {
    if constexpr (J >= 1) {
#pragma unroll
        for (int g = 0; g < NP / 8; g++) {
            if (!((qm >> g) & 1)) continue;
#pragma unroll
            for (int i = 0; i < 4; i++) {
                const int q = bfly_q<J>(4 * g + i), q1 = q | (1 << (J - 1));
                float2 t = r.re[q]; r.re[q] = r.re[q1]; r.re[q1] = t;
                t = r.im[q]; r.im[q] = r.im[q1]; r.im[q1] = t;
            }
        }
    } else {
#pragma unroll
        for (int g4 = 0; g4 < NP / 4; g4++) {
            if (!((qm >> g4) & 1)) continue;
#pragma unroll
            for (int i = 0; i < 4; i++) {
                const int q = 4 * g4 + i;
                r.re[q] = make_float2(r.re[q].y, r.re[q].x);
                r.im[q] = make_float2(r.im[q].y, r.im[q].x);
            }
        }
    }
}

template <int J, int NP>
__device__ __forceinline__ void reg_u2(RegsN<NP> &r, uint32_t qm, const float *m) {
    const float u0r = m[0], u0i = m[1], u1r = m[2], u1i = m[3];
    const float u2r = m[4], u2i = m[5], u3r = m[6], u3i = m[7];
    if constexpr (J >= 1) {
#pragma unroll
        for (int g = 0; g < NP / 8; g++) {
            if (!((qm >> g) & 1)) continue;
#pragma unroll
            for (int i = 0; i < 4; i++) {
                const int q = bfly_q<J>(4 * g + i), q1 = q | (1 << (J - 1));
                const float2 ar = r.re[q], ai = r.im[q], br = r.re[q1], bi = r.im[q1];
                r.re[q] = fma2(bi, f2(-u1i), fma2(br, f2(u1r), fma2(ai, f2(-u0i), mul2(ar, f2(u0r)))));
                r.im[q] = fma2(br, f2(u1i), fma2(bi, f2(u1r), fma2(ar, f2(u0i), mul2(ai, f2(u0r)))));
                r.re[q1] = fma2(bi, f2(-u3i), fma2(br, f2(u3r), fma2(ai, f2(-u2i), mul2(ar, f2(u2r)))));
                r.im[q1] = fma2(br, f2(u3i), fma2(bi, f2(u3r), fma2(ar, f2(u2i), mul2(ai, f2(u2r)))));
            }
        }
    } else {
#pragma unroll
        for (int g4 = 0; g4 < NP / 4; g4++) {
            if (!((qm >> g4) & 1)) continue;
#pragma unroll
            for (int i = 0; i < 4; i++) {
                const int q = 4 * g4 + i;
                const float ar = r.re[q].x, ai = r.im[q].x, br = r.re[q].y, bi = r.im[q].y;
                r.re[q].x = u0r * ar - u0i * ai + u1r * br - u1i * bi;
                r.im[q].x = u0r * ai + u0i * ar + u1r * bi + u1i * br;
                r.re[q].y = u2r * ar - u2i * ai + u3r * br - u3i * bi;
                r.im[q].y = u2r * ai + u2i * ar + u3r * bi + u3i * br;
            }
        }
    }
}

// Rotation [[c, -s], [s, c]] (c >= 0) on register bit J as three in-place
// shears: a += t b, b += s a, a += t b with t = -s / (1 + c) = (c - 1) / s
// (m[0] = t, m[1] = s).  Their product is the rotation exactly; each shear
// is one multiply-add per plane and no register of the pair is copied.
template <int J, int NP>
__device__ __forceinline__ void reg_rot(RegsN<NP> &r, uint32_t qm, const float *m) {
    const float t = m[0], s = m[1];
    if constexpr (J >= 1) {
#pragma unroll
        for (int g = 0; g < NP / 8; g++) {
            if (!((qm >> g) & 1)) continue;
#pragma unroll
            for (int i = 0; i < 4; i++) {
                const int q = bfly_q<J>(4 * g + i), q1 = q | (1 << (J - 1));
                r.re[q] = fma2(r.re[q1], f2(t), r.re[q]);
                r.im[q] = fma2(r.im[q1], f2(t), r.im[q]);
                r.re[q1] = fma2(r.re[q], f2(s), r.re[q1]);
                r.im[q1] = fma2(r.im[q], f2(s), r.im[q1]);
                r.re[q] = fma2(r.re[q1], f2(t), r.re[q]);
                r.im[q] = fma2(r.im[q1], f2(t), r.im[q]);
            }
        }
    } else {
#pragma unroll
        for (int g4 = 0; g4 < NP / 4; g4++) {
            if (!((qm >> g4) & 1)) continue;
#pragma unroll
            for (int i = 0; i < 4; i++) {
                const int q = 4 * g4 + i;
                float2 &x = r.re[q], &y = r.im[q];
                x.x = fmaf(x.y, t, x.x);
                y.x = fmaf(y.y, t, y.x);
                x.y = fmaf(x.x, s, x.y);
                y.y = fmaf(y.x, s, y.y);
                x.x = fmaf(x.y, t, x.x);
                y.x = fmaf(y.y, t, y.x);
            }
        }
    }
}

// Real 2x2 [[a, b], [c, d]] = (m[0], m[2], m[4], m[6]) on register bit J: the
// real and imaginary planes transform alike, two multiply-adds per output.
template <int J, int NP>
__device__ __forceinline__ void reg_r2(RegsN<NP> &r, uint32_t qm, const float *m) {
    const float a = m[0], b = m[2], c = m[4], d = m[6];
    if constexpr (J >= 1) {
#pragma unroll
        for (int g = 0; g < NP / 8; g++) {
            if (!((qm >> g) & 1)) continue;
#pragma unroll
            for (int i = 0; i < 4; i++) {
                const int q = bfly_q<J>(4 * g + i), q1 = q | (1 << (J - 1));
                const float2 ar = r.re[q], ai = r.im[q], br = r.re[q1], bi = r.im[q1];
                r.re[q] = fma2(br, f2(b), mul2(ar, f2(a)));
                r.im[q] = fma2(bi, f2(b), mul2(ai, f2(a)));
                r.re[q1] = fma2(br, f2(d), mul2(ar, f2(c)));
                r.im[q1] = fma2(bi, f2(d), mul2(ai, f2(c)));
            }
        }
    } else {
#pragma unroll
        for (int g4 = 0; g4 < NP / 4; g4++) {
            if (!((qm >> g4) & 1)) continue;
#pragma unroll
            for (int i = 0; i < 4; i++) {
                const int q = 4 * g4 + i;
                const float ar = r.re[q].x, ai = r.im[q].x, br = r.re[q].y, bi = r.im[q].y;
                r.re[q] = make_float2(a * ar + b * br, c * ar + d * br);
                r.im[q] = make_float2(a * ai + b * bi, c * ai + d * bi);
            }
        }
    }
}

// Gate on register bit j (runtime).
__device__ __forceinline__ void reg_gate(Regs &r, int op, int j, int jc, const float *m) {
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
template <int M, typename R>
__device__ __forceinline__ void apply_factor(R &r, float fr, float fi) {
    constexpr int NP = sizeof(r.re) / sizeof(r.re[0]);
#pragma unroll
    for (int q = 0; q < NP; q++) {
        if constexpr ((M & 1) != 0) {
            if (((2 * q + 1) & M) == M) cmul1(r.re[q].y, r.im[q].y, fr, fi);
        } else {
            if (((2 * q) & M) == M) cmul2(r.re[q], r.im[q], fr, fi);
        }
    }
}

// Masks of at most one register bit (the register-stage kernel's per-thread factors).
template <typename R>
__device__ __forceinline__ void apply_factor_bit(R &r, int mask, float fr, float fi) {
    switch (mask) {
        case 0: apply_factor<0>(r, fr, fi); break;
        case 1: apply_factor<1>(r, fr, fi); break;
        case 2: apply_factor<2>(r, fr, fi); break;
        case 4: apply_factor<4>(r, fr, fi); break;
        case 8: apply_factor<8>(r, fr, fi); break;
        default: apply_factor<16>(r, fr, fi); break;
    }
}

template <typename R>
__device__ __forceinline__ void apply_factor_any(R &r, int mask, float fr, float fi) {
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

}  // namespace tiledev
}  // namespace sv
