// General gate set on the per-gate path: multi-controlled U (MCU), two-qubit
// unitaries (U2Q with its three row records) and projective measurement
// with collapse (MEASURE).  Gates arrive with PHYSICAL qubit positions.
//
// MCU is Algorithm 1 (Sec. III-A) with the control rule taken to a set of
// controls: the pair (x, x + 2^t) is updated only when every control bit of
// x is 1, so the kernel enumerates exactly those pairs (2^(n-1-k) of them).
// U2Q updates the four amplitudes that agree off its two qubits.  MEASURE
// sums |amp|^2 over each value of its qubit in FP64 (per-block partials in a
// fixed tree, then the blocks in order), picks the outcome on the device as
// the smallest i with C_i > u C_last for C = (p0, p0 + p1), and collapses the
// state: the other half is zeroed and the kept one divided by sqrt(p_i).  No
// host synchronisation: the outcome goes to a device array that
// sv_last_measurements reads.
#include <algorithm>
#include <cmath>

#include "common.h"

namespace sv {
namespace {

constexpr int kThreads = 256;
constexpr int kMeasBlocks = 1024;  // partial sums of a measurement (2 doubles each)

// Positions (ascending) where the enumeration inserts a bit.
struct Ins {
    int n;
    int8_t pos[40];
};

__device__ __forceinline__ uint64_t insert_zeros(uint64_t u, const Ins &in) {
    for (int i = 0; i < in.n; i++) {
        const int p = in.pos[i];
        u = ((u >> p) << (p + 1)) | (u & ((UINT64_C(1) << p) - 1));
    }
    return u;
}

template <typename R>
struct C2 {
    R re[4], im[4];
};
template <typename R>
struct C4 {
    R re[16], im[16];
};

template <typename R>
__global__ void __launch_bounds__(kThreads)
k_mcu(R *__restrict__ s, uint64_t units, Ins in, uint64_t ones, uint64_t tbit, C2<R> c) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t u = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; u < units; u += stride) {
        const uint64_t x0 = insert_zeros(u, in) | ones, x1 = x0 | tbit;
        const R ar = s[2 * x0], ai = s[2 * x0 + 1], br = s[2 * x1], bi = s[2 * x1 + 1];
        s[2 * x0] = c.re[0] * ar - c.im[0] * ai + c.re[1] * br - c.im[1] * bi;
        s[2 * x0 + 1] = c.re[0] * ai + c.im[0] * ar + c.re[1] * bi + c.im[1] * br;
        s[2 * x1] = c.re[2] * ar - c.im[2] * ai + c.re[3] * br - c.im[3] * bi;
        s[2 * x1 + 1] = c.re[2] * ai + c.im[2] * ar + c.re[3] * bi + c.im[3] * br;
    }
}

template <typename R>
__global__ void __launch_bounds__(kThreads)
k_u2q(R *__restrict__ s, uint64_t units, Ins in, uint64_t ma, uint64_t mb, C4<R> m) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t u = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; u < units; u += stride) {
        const uint64_t x = insert_zeros(u, in);
        const uint64_t idx[4] = {x, x | ma, x | mb, x | ma | mb};
        R vr[4], vi[4];
#pragma unroll
        for (int k = 0; k < 4; k++) {
            vr[k] = s[2 * idx[k]];
            vi[k] = s[2 * idx[k] + 1];
        }
#pragma unroll
        for (int r = 0; r < 4; r++) {
            R yr = 0, yi = 0;
#pragma unroll
            for (int k = 0; k < 4; k++) {
                yr += m.re[4 * r + k] * vr[k] - m.im[4 * r + k] * vi[k];
                yi += m.re[4 * r + k] * vi[k] + m.im[4 * r + k] * vr[k];
            }
            s[2 * idx[r]] = yr;
            s[2 * idx[r] + 1] = yi;
        }
    }
}

// Per-block FP64 sums of |amp|^2 with the measured bit 0 and 1.
template <typename R>
__global__ void __launch_bounds__(kThreads)
k_meas_partial(const R *__restrict__ s, uint64_t N, uint64_t tbit, double *__restrict__ part) {
    __shared__ double sh0[kThreads], sh1[kThreads];
    double p0 = 0.0, p1 = 0.0;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t x = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; x < N; x += stride) {
        const double re = (double)s[2 * x], im = (double)s[2 * x + 1];
        const double q = re * re + im * im;
        if (x & tbit) p1 += q;
        else p0 += q;
    }
    sh0[threadIdx.x] = p0;
    sh1[threadIdx.x] = p1;
    __syncthreads();
    for (int w = kThreads / 2; w; w >>= 1) {
        if ((int)threadIdx.x < w) {
            sh0[threadIdx.x] += sh0[threadIdx.x + w];
            sh1[threadIdx.x] += sh1[threadIdx.x + w];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        part[2 * blockIdx.x] = sh0[0];
        part[2 * blockIdx.x + 1] = sh1[0];
    }
}

// The outcome (smallest i with C_i > u C_last) and the kept half's scale.
__global__ void k_meas_decide(const double *__restrict__ part, int nblocks, double u, double *dec,
                              uint8_t *outcome) {
    double p0 = 0.0, p1 = 0.0;
    for (int b = 0; b < nblocks; b++) {
        p0 += part[2 * b];
        p1 += part[2 * b + 1];
    }
    const double last = p0 + p1;
    const int out = (p0 > u * last) ? 0 : 1;
    const double keep = out ? p1 : p0;
    dec[0] = (double)out;
    dec[1] = keep > 0.0 ? 1.0 / sqrt(keep) : 0.0;
    *outcome = (uint8_t)out;
}

template <typename R>
__global__ void __launch_bounds__(kThreads)
k_meas_collapse(R *__restrict__ s, uint64_t N, uint64_t tbit, const double *__restrict__ dec) {
    const int out = (int)dec[0];
    const R sc = (R)dec[1];
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t x = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; x < N; x += stride) {
        const int bit = (x & tbit) ? 1 : 0;
        if (bit == out) {
            s[2 * x] *= sc;
            s[2 * x + 1] *= sc;
        } else {
            s[2 * x] = R(0);
            s[2 * x + 1] = R(0);
        }
    }
}

unsigned grid_of(uint64_t units, int sm_count) {
    const uint64_t b = (units + kThreads - 1) / kThreads;
    return (unsigned)std::max<uint64_t>(1, std::min<uint64_t>(b, (uint64_t)sm_count * 16));
}

Ins make_ins(uint64_t fixed) {
    Ins in{};
    for (int b = 0; b < 64; b++)
        if ((fixed >> b) & 1) in.pos[in.n++] = (int8_t)b;
    return in;
}

template <typename R>
sv_status launch_general(sv_state *h, const sv_gate *g, sv_launch_record &meta) {
    R *s = reinterpret_cast<R *>(h->amps);
    const int n = h->n;
    const uint64_t N = UINT64_C(1) << n;
    if (g[0].kind == SV_MCU) {
        const uint64_t cm = (uint64_t)g[0].num, tb = UINT64_C(1) << g[0].target;
        const int k = __builtin_popcountll(cm);
        const Mat2 m = gate_matrix(g[0]);
        C2<R> c;
        for (int e = 0; e < 4; e++) {
            c.re[e] = (R)m.re[e];
            c.im[e] = (R)m.im[e];
        }
        const uint64_t units = UINT64_C(1) << (n - 1 - k);
        meta.bytes = 2.0 * std::ldexp(1.0, -k) * (double)state_bytes(h);
        const int slot = prof_begin(h);
        k_mcu<R><<<grid_of(units, h->sm_count), kThreads, 0, h->stream>>>(s, units, make_ins(cm | tb), cm, tb, c);
        SV_CUDA(cudaGetLastError());
        note_launch();
        prof_end(h, slot, meta);
    } else if (g[0].kind == SV_U2Q) {
        const uint64_t ma = UINT64_C(1) << g[0].target, mb = UINT64_C(1) << g[0].control;
        C4<R> m;
        for (int r = 0; r < 4; r++)
            for (int k = 0; k < 4; k++) {
                m.re[4 * r + k] = (R)g[r].p[2 * k];
                m.im[4 * r + k] = (R)g[r].p[2 * k + 1];
            }
        const uint64_t units = N / 4;
        meta.bytes = 2.0 * (double)state_bytes(h);
        const int slot = prof_begin(h);
        k_u2q<R><<<grid_of(units, h->sm_count), kThreads, 0, h->stream>>>(s, units, make_ins(ma | mb), ma, mb, m);
        SV_CUDA(cudaGetLastError());
        note_launch();
        prof_end(h, slot, meta);
    } else {  // SV_MEASURE
        SV_TRY(ensure_meas(h, h->nmeas + 1));
        const uint64_t tb = UINT64_C(1) << g[0].target;
        double *part = reinterpret_cast<double *>(h->small);
        double *dec = part + 2 * kMeasBlocks;
        const int nb = (int)std::min<uint64_t>(kMeasBlocks, grid_of(N, h->sm_count));
        meta.bytes = 3.0 * (double)state_bytes(h);  // one read to sum, one read and write to collapse
        const int slot = prof_begin(h);
        k_meas_partial<R><<<nb, kThreads, 0, h->stream>>>(s, N, tb, part);
        k_meas_decide<<<1, 1, 0, h->stream>>>(part, nb, g[0].p[0], dec, h->meas_dev + h->nmeas);
        k_meas_collapse<R><<<grid_of(N, h->sm_count), kThreads, 0, h->stream>>>(s, N, tb, dec);
        SV_CUDA(cudaGetLastError());
        note_launch(3);
        prof_end(h, slot, meta);
        h->nmeas++;
    }
    h->stats.kernels++;
    return SV_OK;
}

}  // namespace

int general_records(int kind) { return kind == SV_U2Q ? 4 : 1; }

bool is_general_kind(int kind) { return kind == SV_MCU || kind == SV_U2Q || kind == SV_MEASURE; }

sv_status general_apply(sv_state *h, const sv_gate *g) {
    static_assert(2 * kMeasBlocks * sizeof(double) + 64 <= 64 * 1024, "measurement scratch fits the small area");
    SV_TRY(materialize(h));
    SV_TRY(resolve_norm(h));
    SV_TRY(launch_check());
    sv_launch_record meta{};
    meta.kind = SV_KERNEL_PERGATE;
    meta.pass = h->launch_index++;
    meta.n = h->n;
    meta.nops = 1;
    meta.ngates = 1;
    meta.dtype = (int32_t)h->dt;
    meta.gate_kind = g[0].kind;
    meta.feat = UINT64_C(1) << g[0].target;
    if (g[0].kind == SV_MCU) meta.feat |= (uint64_t)g[0].num;
    if (g[0].kind == SV_U2Q) meta.feat |= UINT64_C(1) << g[0].control;
    const sv_status st = h->dt == SV_C128 ? launch_general<double>(h, g, meta)
                                          : launch_general<float>(h, g, meta);
    if (st != SV_OK) return st;
    h->stats.passes++;
    h->stats.touched_bytes += meta.bytes;
    return SV_OK;
}

sv_status ensure_meas(sv_state *h, size_t count) {
    if (count <= h->meas_cap) return SV_OK;
    const size_t cap = std::max<size_t>(2 * count, 256);
    uint8_t *p = nullptr;
    if (dev_malloc(&p, cap) != cudaSuccess) {
        cudaGetLastError();
        return fail(SV_ERR_OOM, "cannot allocate the measurement outcomes (%zu bytes)", cap);
    }
    if (h->meas_dev) {
        SV_CUDA(cudaMemcpyAsync(p, h->meas_dev, h->nmeas, cudaMemcpyDeviceToDevice, h->stream));
        SV_CUDA(cudaStreamSynchronize(h->stream));
        cudaFree(h->meas_dev);
    }
    h->meas_dev = p;
    h->meas_cap = cap;
    return SV_OK;
}

}  // namespace sv
