// Per-gate kernels: one sweep of HBM per gate (Algorithm 1 of arxiv
// 2605.15098, Sec. III-A, with the control rule of the same section).
//
// Algorithm 1 visits every index j whose bit t is 0 and updates the pair
// (S[j], S[j + 2^t]).  Here the pairs are enumerated directly: the g-th pair
// is g with a 0 inserted at bit t.  A control bit c (run only when bit c of
// j is 1) is a second inserted bit, fixed to 1, so controlled gates only
// touch the half of the state they change.  Diagonal gates (P, CP, CZ, PK,
// CPK) only change amplitudes whose target (and control) bit is 1 and touch
// just those; SWAP(a, b) touches the half with bits a != b.
//
// Memory access: every thread moves 16-byte vectors.  For complex64 a vector
// holds two neighbouring amplitudes (indices 2v, 2v+1); when no gate qubit
// is bit 0 they share every fixed bit and are updated together; a gate on
// bit 0 pairs the two halves of one vector.  For complex128 a vector is one
// amplitude.  Consecutive threads take consecutive vectors, so each warp
// reads and writes whole 512-byte segments.
#include <algorithm>
#include <cmath>

#include "common.h"

namespace sv {
namespace {

constexpr int kThreads = 256;
constexpr int kItems = 4;

struct Fixed {
    int n;
    int pos[3];  // ascending, in vector units
    int val[3];
};

template <typename R>
struct Coef {
    R re[4], im[4];
};

enum Op { OP_U = 0, OP_H = 1, OP_X = 2, OP_PHASE = 3, OP_NEG = 4, OP_SWAP = 5 };

template <typename R, int VB>
struct VecT;
template <>
struct VecT<float, 1> {
    using T = float4;
};
template <>
struct VecT<float, 0> {
    using T = float2;
};
template <>
struct VecT<double, 0> {
    using T = double2;
};

__device__ __forceinline__ uint64_t insert_bits(uint64_t x, const Fixed &f) {
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        if (i < f.n) {
            const int p = f.pos[i];
            const uint64_t lo = x & ((UINT64_C(1) << p) - 1);
            x = ((x >> p) << (p + 1)) | ((uint64_t)f.val[i] << p) | lo;
        }
    }
    return x;
}

template <typename R>
__device__ __forceinline__ R scale_h(R x, const Coef<R> &c) {
    if constexpr (sizeof(R) == 4)
        return fmaf(x, c.re[0], x * c.im[0]);
    else
        return x * c.re[0];
}

// (a, b) <- U (a, b) for one amplitude pair, by kind.
template <typename R, int OP>
__device__ __forceinline__ void pair_update(R &ar, R &ai, R &br, R &bi, const Coef<R> &c) {
    if (OP == OP_U) {
        R xr = c.re[0] * ar - c.im[0] * ai + c.re[1] * br - c.im[1] * bi;
        R xi = c.re[0] * ai + c.im[0] * ar + c.re[1] * bi + c.im[1] * br;
        R yr = c.re[2] * ar - c.im[2] * ai + c.re[3] * br - c.im[3] * bi;
        R yi = c.re[2] * ai + c.im[2] * ar + c.re[3] * bi + c.im[3] * br;
        ar = xr; ai = xi; br = yr; bi = yi;
    } else if (OP == OP_H) {
        // complex64: 1/sqrt(2) = s_hi + s_lo (two floats) so that the product
        // is rounded once, without the bias of a rounded constant
        R xr = ar + br, xi = ai + bi, yr = ar - br, yi = ai - bi;
        ar = scale_h(xr, c); ai = scale_h(xi, c); br = scale_h(yr, c); bi = scale_h(yi, c);
    } else if (OP == OP_X || OP == OP_SWAP) {
        R tr = ar, ti = ai;
        ar = br; ai = bi; br = tr; bi = ti;
    }
}

template <typename R, int OP>
__device__ __forceinline__ void single_update(R &ar, R &ai, const Coef<R> &c) {
    if (OP == OP_PHASE) {
        R xr = ar * c.re[0] - ai * c.im[0];
        R xi = ar * c.im[0] + ai * c.re[0];
        ar = xr; ai = xi;
    } else if (OP == OP_NEG) {
        ar = -ar; ai = -ai;
    }
}

// Pair / single-amplitude kernel over vectors of 2^VB amplitudes.
// units: number of enumerated vectors (or vector pairs); partner: XOR that
// maps the enumerated vector to its partner (0 for single-amplitude ops).
template <typename R, int VB, int OP>
__global__ void __launch_bounds__(kThreads)
k_pergate(R *__restrict__ s, uint64_t units, Fixed fx, uint64_t partner, Coef<R> c) {
    using T = typename VecT<R, VB>::T;
    constexpr int NA = 1 << VB;  // amplitudes per vector
    constexpr bool PAIR = (OP == OP_U || OP == OP_H || OP == OP_X || OP == OP_SWAP);
    T *v = reinterpret_cast<T *>(s);
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t u0 = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; u0 < units;
         u0 += stride * kItems) {
        T a[kItems], b[kItems];
        uint64_t ia[kItems];
#pragma unroll
        for (int k = 0; k < kItems; ++k) {
            const uint64_t u = u0 + (uint64_t)k * stride;
            if (u < units) {
                ia[k] = insert_bits(u, fx);
                a[k] = v[ia[k]];
                if (PAIR) b[k] = v[ia[k] ^ partner];
            }
        }
#pragma unroll
        for (int k = 0; k < kItems; ++k) {
            R *pa = reinterpret_cast<R *>(&a[k]);
            R *pb = reinterpret_cast<R *>(&b[k]);
#pragma unroll
            for (int e = 0; e < NA; ++e) {
                if (PAIR)
                    pair_update<R, OP>(pa[2 * e], pa[2 * e + 1], pb[2 * e], pb[2 * e + 1], c);
                else
                    single_update<R, OP>(pa[2 * e], pa[2 * e + 1], c);
            }
        }
#pragma unroll
        for (int k = 0; k < kItems; ++k) {
            const uint64_t u = u0 + (uint64_t)k * stride;
            if (u < units) {
                v[ia[k]] = a[k];
                if (PAIR) v[ia[k] ^ partner] = b[k];
            }
        }
    }
}

// complex64 gate on qubit 0: the pair is the two halves of one float4.
template <int OP>
__global__ void __launch_bounds__(kThreads)
k_pergate_intra(float *__restrict__ s, uint64_t units, Fixed fx, Coef<float> c) {
    float4 *v = reinterpret_cast<float4 *>(s);
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t u0 = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; u0 < units;
         u0 += stride * kItems) {
        float4 a[kItems];
        uint64_t ia[kItems];
#pragma unroll
        for (int k = 0; k < kItems; ++k) {
            const uint64_t u = u0 + (uint64_t)k * stride;
            if (u < units) {
                ia[k] = insert_bits(u, fx);
                a[k] = v[ia[k]];
            }
        }
#pragma unroll
        for (int k = 0; k < kItems; ++k) pair_update<float, OP>(a[k].x, a[k].y, a[k].z, a[k].w, c);
#pragma unroll
        for (int k = 0; k < kItems; ++k) {
            const uint64_t u = u0 + (uint64_t)k * stride;
            if (u < units) v[ia[k]] = a[k];
        }
    }
}

// The recorded product state H^{hq}|b>: amplitude x is (-1)^{|x & b & hq|} v
// where x agrees with b off hq (v = 2^{-|hq|/2}), 0 elsewhere; two amplitudes
// per thread and 16-byte store.
template <typename R>
__global__ void k_set_product(R *amps, uint64_t npairs, uint64_t b, uint64_t hq, R v) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t p = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; p < npairs; p += stride) {
        R a[2];
        for (int e = 0; e < 2; e++) {
            const uint64_t x = 2 * p + e;
            a[e] = ((x ^ b) & ~hq) ? R(0) : ((__popcll(x & b & hq) & 1) ? -v : v);
        }
        if constexpr (sizeof(R) == 4)
            reinterpret_cast<float4 *>(amps)[p] = make_float4(a[0], 0.f, a[1], 0.f);
        else {
            reinterpret_cast<double2 *>(amps)[2 * p] = make_double2(a[0], 0.0);
            reinterpret_cast<double2 *>(amps)[2 * p + 1] = make_double2(a[1], 0.0);
        }
    }
}

unsigned grid_for(uint64_t units) {
    uint64_t per_block = (uint64_t)kThreads * kItems;
    uint64_t b = (units + per_block - 1) / per_block;
    if (b < 1) b = 1;
    if (b > 0x7fffffffULL) b = 0x7fffffffULL;
    return (unsigned)b;
}

template <typename R>
Coef<R> to_coef(const Mat2 &m) {
    Coef<R> c;
    for (int e = 0; e < 4; e++) {
        c.re[e] = (R)m.re[e];
        c.im[e] = (R)m.im[e];
    }
    return c;
}

// Launch helper: OP chosen at run time.
template <typename R, int VB>
sv_status launch_op(sv_state *h, int op, uint64_t units, const Fixed &fx, uint64_t partner,
                    const Coef<R> &c, const sv_launch_record &meta) {
    R *s = reinterpret_cast<R *>(h->amps);
    dim3 grid(grid_for(units)), block(kThreads);
    const int slot = prof_begin(h);
    switch (op) {
        case OP_U: k_pergate<R, VB, OP_U><<<grid, block, 0, h->stream>>>(s, units, fx, partner, c); break;
        case OP_H: k_pergate<R, VB, OP_H><<<grid, block, 0, h->stream>>>(s, units, fx, partner, c); break;
        case OP_X: k_pergate<R, VB, OP_X><<<grid, block, 0, h->stream>>>(s, units, fx, partner, c); break;
        case OP_PHASE: k_pergate<R, VB, OP_PHASE><<<grid, block, 0, h->stream>>>(s, units, fx, partner, c); break;
        case OP_NEG: k_pergate<R, VB, OP_NEG><<<grid, block, 0, h->stream>>>(s, units, fx, partner, c); break;
        case OP_SWAP: k_pergate<R, VB, OP_SWAP><<<grid, block, 0, h->stream>>>(s, units, fx, partner, c); break;
        default: return fail(SV_ERR_ARG, "internal: bad per-gate op");
    }
    SV_CUDA(cudaGetLastError());
    note_launch();
    prof_end(h, slot, meta);
    h->stats.kernels++;
    return SV_OK;
}

void add_fixed(Fixed &f, int pos, int val) {
    int i = f.n++;
    f.pos[i] = pos;
    f.val[i] = val;
    while (i > 0 && f.pos[i - 1] > f.pos[i]) {  // keep ascending
        int tp = f.pos[i - 1], tv = f.val[i - 1];
        f.pos[i - 1] = f.pos[i];
        f.val[i - 1] = f.val[i];
        f.pos[i] = tp;
        f.val[i] = tv;
        --i;
    }
}

}  // namespace

sv_status init_zero_state(sv_state *h) {
    for (int q = 0; q < 64; q++) h->phys[q] = q;
    h->basis = 0;  // |0...0>, written when something first reads the state
    h->basis_h = 0;
    return SV_OK;
}

sv_status materialize(sv_state *h) {
    if (h->basis < 0) return SV_OK;
    const uint64_t npairs = (UINT64_C(1) << h->n) / 2;
    const uint64_t hq = h->basis_h, b = (uint64_t)h->basis;
    const double v = std::pow(2.0, -0.5 * __builtin_popcountll(hq));
    if (h->n == 1) {  // one pair: the same kernel, one thread
        if (h->dt == SV_C128)
            k_set_product<double><<<1, 1, 0, h->stream>>>((double *)h->amps, 1, b, hq, v);
        else
            k_set_product<float><<<1, 1, 0, h->stream>>>((float *)h->amps, 1, b, hq, (float)v);
    } else {
        const unsigned grid = (unsigned)std::min<uint64_t>((npairs + 255) / 256, (uint64_t)h->sm_count * 8);
        if (h->dt == SV_C128)
            k_set_product<double><<<grid, 256, 0, h->stream>>>((double *)h->amps, npairs, b, hq, v);
        else
            k_set_product<float><<<grid, 256, 0, h->stream>>>((float *)h->amps, npairs, b, hq, (float)v);
    }
    SV_CUDA(cudaGetLastError());
    note_launch();
    h->basis = -1;
    h->basis_h = 0;
    return SV_OK;
}

// Apply one gate given in PHYSICAL qubit positions.
sv_status pergate_apply(sv_state *h, const sv_gate &g) {
    SV_TRY(materialize(h));
    SV_TRY(launch_check());
    const int n = h->n;
    int op;
    Mat2 m{};
    // bits the enumeration fixes (amplitude units): (position, value)
    int fpos[3], fval[3], nf = 0;
    int pair_bit = -1;        // partner differs in this bit (pair ops)
    int swap_a = -1, swap_b = -1;
    double fraction = 1.0;    // share of the state the kernel moves
    switch (g.kind) {
        case SV_X: op = OP_X; break;
        case SV_H: op = OP_H; break;
        case SV_U3: case SV_U: case SV_CU: op = OP_U; break;
        case SV_CZ: op = OP_NEG; break;
        case SV_P: case SV_CP: case SV_PK: case SV_CPK: op = OP_PHASE; break;
        case SV_SWAP: op = OP_SWAP; break;
        default: return fail(SV_ERR_ARG, "internal: kind %d", g.kind);
    }
    if (op != OP_SWAP && op != OP_NEG) m = gate_matrix(g);
    if (op == OP_H) {
        const double r = 0.70710678118654752440084436210485;
        m.re[0] = r;
        m.im[0] = h->dt == SV_C64 ? r - (double)(float)r : 0.0;  // low part for complex64
    }
    if (op == OP_PHASE) {  // coefficient on |1>
        m.re[0] = m.re[3];
        m.im[0] = m.im[3];
    }
    const bool ctrl = is_controlled_kind(g.kind);
    if (op == OP_SWAP) {
        swap_a = g.target;
        swap_b = g.control;
        fpos[nf] = swap_a; fval[nf++] = 1;
        fpos[nf] = swap_b; fval[nf++] = 0;
        fraction = 0.5;
    } else if (op == OP_PHASE || op == OP_NEG) {
        fpos[nf] = g.target; fval[nf++] = 1;
        if (ctrl) { fpos[nf] = g.control; fval[nf++] = 1; }
        fraction = ctrl ? 0.25 : 0.5;
    } else {
        pair_bit = g.target;
        fpos[nf] = g.target; fval[nf++] = 0;
        if (ctrl) { fpos[nf] = g.control; fval[nf++] = 1; }
        fraction = ctrl ? 0.5 : 1.0;
    }
    h->stats.passes++;
    h->stats.touched_bytes += fraction * 2.0 * (double)state_bytes(h);
    sv_launch_record meta{};
    meta.kind = SV_KERNEL_PERGATE;
    meta.pass = h->launch_index++;
    meta.n = n;
    meta.nops = 1;
    meta.ngates = 1;
    meta.dtype = (int32_t)h->dt;
    meta.gate_kind = g.kind;
    meta.bytes = fraction * 2.0 * (double)state_bytes(h);
    meta.feat = UINT64_C(1) << g.target;
    if (is_controlled_kind(g.kind) || g.kind == SV_SWAP) meta.feat |= UINT64_C(1) << g.control;

    if (h->dt == SV_C128) {
        Fixed fx{};
        for (int i = 0; i < nf; i++) add_fixed(fx, fpos[i], fval[i]);
        uint64_t units = UINT64_C(1) << (n - nf);
        uint64_t partner = 0;
        if (pair_bit >= 0) partner = UINT64_C(1) << pair_bit;
        if (op == OP_SWAP) partner = (UINT64_C(1) << swap_a) | (UINT64_C(1) << swap_b);
        return launch_op<double, 0>(h, op, units, fx, partner, to_coef<double>(m), meta);
    }
    // complex64
    bool any0 = false;
    for (int i = 0; i < nf; i++) any0 |= (fpos[i] == 0);
    if (op != OP_SWAP && pair_bit == 0) {
        // pair inside one float4; only the control (never bit 0) is fixed
        Fixed fx{};
        if (ctrl) add_fixed(fx, g.control - 1, 1);
        uint64_t units = UINT64_C(1) << (n - 1 - fx.n);
        dim3 grid(grid_for(units)), block(kThreads);
        float *s = reinterpret_cast<float *>(h->amps);
        Coef<float> c = to_coef<float>(m);
        const int slot = prof_begin(h);
        switch (op) {
            case OP_U: k_pergate_intra<OP_U><<<grid, block, 0, h->stream>>>(s, units, fx, c); break;
            case OP_H: k_pergate_intra<OP_H><<<grid, block, 0, h->stream>>>(s, units, fx, c); break;
            case OP_X: k_pergate_intra<OP_X><<<grid, block, 0, h->stream>>>(s, units, fx, c); break;
            default: return fail(SV_ERR_ARG, "internal: intra op");
        }
        SV_CUDA(cudaGetLastError());
        note_launch();
        prof_end(h, slot, meta);
        h->stats.kernels++;
        return SV_OK;
    }
    if (!any0 && n >= 1 + nf) {
        Fixed fx{};
        for (int i = 0; i < nf; i++) add_fixed(fx, fpos[i] - 1, fval[i]);
        uint64_t units = UINT64_C(1) << (n - 1 - nf);
        uint64_t partner = 0;
        if (pair_bit >= 0) partner = UINT64_C(1) << (pair_bit - 1);
        if (op == OP_SWAP) partner = (UINT64_C(1) << (swap_a - 1)) | (UINT64_C(1) << (swap_b - 1));
        return launch_op<float, 1>(h, op, units, fx, partner, to_coef<float>(m), meta);
    }
    Fixed fx{};
    for (int i = 0; i < nf; i++) add_fixed(fx, fpos[i], fval[i]);
    uint64_t units = UINT64_C(1) << (n - nf);
    uint64_t partner = 0;
    if (pair_bit >= 0) partner = UINT64_C(1) << pair_bit;
    if (op == OP_SWAP) partner = (UINT64_C(1) << swap_a) | (UINT64_C(1) << swap_b);
    return launch_op<float, 0>(h, op, units, fx, partner, to_coef<float>(m), meta);
}

}  // namespace sv
