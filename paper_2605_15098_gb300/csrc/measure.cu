// Read-out kernels: FP64 marginal probabilities, renormalisation, argmax and
// inverse-CDF sampling (the measured bitstring of Sec. IV-A, arxiv 2605.15098).
//
// All sums run in a fixed order, so a call returns the same bits every time:
//   1. partial[g][m] = sum of |amp|^2 over the g-th slice of the amplitudes
//      that map to outcome m, summed in increasing index order;
//   2. p[m] = sum over g of partial[g][m], in g order;
//   3. total = fixed two-level tree over p; p[m] /= total.
// Sampling builds the inclusive CDF in blocks of 1024 outcomes (in-block
// running sums in index order, block totals accumulated in block order) and
// binary-searches the smallest i with C_i > u * C_last for each shot.
#include <algorithm>

#include "common.h"

namespace sv {
namespace {

constexpr int kRedThreads = 256;

struct MargArgs {
    int n;
    int m;                    // outcome bits
    uint64_t mask;            // physical bits of the outcome
    uint64_t rest;            // physical bits summed over (within n)
    uint64_t upper;           // layout R: rest bits above the 5 lane bits
    int spos[34];             // outcome physical bits, ascending
    int out_bit[34];          // logical output bit of spos[k]
    uint64_t per_group;       // enumerated rest values per group
    int groups_log2;
};

__device__ __forceinline__ uint64_t pdep_mask(uint64_t v, uint64_t mask) {
    uint64_t r = 0;
    for (uint64_t b = 1; mask; b <<= 1) {
        uint64_t low = mask & (~mask + 1);
        if (v & b) r |= low;
        mask &= mask - 1;
    }
    return r;
}

// Running sum of |amp|^2.  complex128: FP64.  complex64: the squares of the
// FP32 components are formed exactly (product plus fmaf remainder) and added
// with error-free FP32 sums into a (hi, lo) pair, converted to FP64 once per
// thread: the result is the FP64-rounded exact sum to within about 2^-44
// relative, at FP32 instruction cost (GB300 issues FP64 at 1/64 of FP32).
template <typename R>
struct ProbAcc;

// Amplitude loads a reduction thread keeps in flight before accumulating
// them (in order): enough bytes in flight per SM to cover HBM latency.
constexpr int kLoadBatch = 8;

template <>
struct ProbAcc<double> {
    using V = double2;
    double acc = 0.0;
    __device__ static V load(const double *s, uint64_t x) {
        return reinterpret_cast<const double2 *>(s)[x];
    }
    __device__ void add(V v) { acc += v.x * v.x + v.y * v.y; }
    __device__ void add(const double *s, uint64_t x) { add(load(s, x)); }
    __device__ double value() const { return acc; }
};

template <>
struct ProbAcc<float> {
    float hi = 0.f, lo = 0.f;
    __device__ void two_sum(float b) {
        const float t = hi + b;
        const float bb = t - hi;
        lo += (hi - (t - bb)) + (b - bb);
        hi = t;
    }
    using V = float2;
    __device__ static V load(const float *s, uint64_t x) {
        return reinterpret_cast<const float2 *>(s)[x];
    }
    __device__ void add(V v) {
        const float pr = v.x * v.x, pi = v.y * v.y;
        lo += fmaf(v.x, v.x, -pr) + fmaf(v.y, v.y, -pi);
        two_sum(pr);
        two_sum(pi);
    }
    __device__ void add(const float *s, uint64_t x) { add(load(s, x)); }
    __device__ double value() const { return (double)hi + (double)lo; }
};

// Layout M: outcome bit 0 is physical bit 0, so consecutive threads (consecutive
// physical-order outcomes) read neighbouring amplitudes.
template <typename R>
__global__ void __launch_bounds__(kRedThreads)
k_marg_m(const R *__restrict__ s, MargArgs a, double *__restrict__ partial) {
    const uint64_t outcomes = UINT64_C(1) << a.m;
    const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (tid >= (outcomes << a.groups_log2)) return;
    const uint64_t mp = tid & (outcomes - 1);
    const uint64_t g = tid >> a.m;
    uint64_t xm = 0, ml = 0;
    for (int k = 0; k < a.m; k++) {
        if ((mp >> k) & 1) {
            xm |= UINT64_C(1) << a.spos[k];
            ml |= UINT64_C(1) << a.out_bit[k];
        }
    }
    uint64_t xr = pdep_mask(g * a.per_group, a.rest);
    ProbAcc<R> acc;
    uint64_t i = 0;
    // kLoadBatch loads in flight per thread, then accumulated in order
    for (; i + kLoadBatch <= a.per_group; i += kLoadBatch) {
        typename ProbAcc<R>::V v[kLoadBatch];
#pragma unroll
        for (int k = 0; k < kLoadBatch; k++) {
            v[k] = ProbAcc<R>::load(s, xm | xr);
            xr = ((xr | ~a.rest) + 1) & a.rest;
        }
#pragma unroll
        for (int k = 0; k < kLoadBatch; k++) acc.add(v[k]);
    }
    for (; i < a.per_group; i++) {
        acc.add(s, xm | xr);
        xr = ((xr | ~a.rest) + 1) & a.rest;
    }
    partial[g * outcomes + ml] = acc.value();
}

// Layout M, complex64: each thread takes the two outcomes that differ in
// physical bit 0 (one 16-byte load covers both amplitudes), each summed in
// the same order as k_marg_m.
__global__ void __launch_bounds__(kRedThreads)
k_marg_m2(const float *__restrict__ s, MargArgs a, double *__restrict__ partial) {
    const uint64_t outcomes = UINT64_C(1) << a.m;
    const uint64_t half = outcomes >> 1;
    const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (tid >= (half << a.groups_log2)) return;
    const uint64_t mp = (tid & (half - 1)) << 1;
    const uint64_t g = tid >> (a.m - 1);
    uint64_t xm = 0, ml = 0;
    for (int k = 1; k < a.m; k++) {
        if ((mp >> k) & 1) {
            xm |= UINT64_C(1) << a.spos[k];
            ml |= UINT64_C(1) << a.out_bit[k];
        }
    }
    const uint64_t ml1 = ml | (UINT64_C(1) << a.out_bit[0]);
    uint64_t xr = pdep_mask(g * a.per_group, a.rest);
    ProbAcc<float> acc0, acc1;
    const float4 *s4 = reinterpret_cast<const float4 *>(s);
    uint64_t i = 0;
    for (; i + kLoadBatch <= a.per_group; i += kLoadBatch) {
        float4 v[kLoadBatch];
#pragma unroll
        for (int k = 0; k < kLoadBatch; k++) {
            v[k] = s4[(xm | xr) >> 1];
            xr = ((xr | ~a.rest) + 1) & a.rest;
        }
#pragma unroll
        for (int k = 0; k < kLoadBatch; k++) {
            acc0.add(make_float2(v[k].x, v[k].y));
            acc1.add(make_float2(v[k].z, v[k].w));
        }
    }
    for (; i < a.per_group; i++) {
        const float4 v = s4[(xm | xr) >> 1];
        acc0.add(make_float2(v.x, v.y));
        acc1.add(make_float2(v.z, v.w));
        xr = ((xr | ~a.rest) + 1) & a.rest;
    }
    partial[g * outcomes + ml] = acc0.value();
    partial[g * outcomes + ml1] = acc1.value();
}

// Layout R: the lowest physical bits are summed over; one warp per
// (group, outcome), lanes take the five lowest rest bits.
template <typename R>
__global__ void __launch_bounds__(kRedThreads)
k_marg_r(const R *__restrict__ s, MargArgs a, double *__restrict__ partial) {
    const uint64_t outcomes = UINT64_C(1) << a.m;
    const uint64_t warp = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (warp >= (outcomes << a.groups_log2)) return;
    const uint64_t mp = warp & (outcomes - 1);
    const uint64_t g = warp >> a.m;
    uint64_t xm = 0, ml = 0;
    for (int k = 0; k < a.m; k++) {
        if ((mp >> k) & 1) {
            xm |= UINT64_C(1) << a.spos[k];
            ml |= UINT64_C(1) << a.out_bit[k];
        }
    }
    const uint64_t lane_bits = a.rest & ~a.upper;
    const uint64_t xl = pdep_mask((uint64_t)lane, lane_bits);
    uint64_t xo = pdep_mask(g * a.per_group, a.upper);
    ProbAcc<R> pa;
    uint64_t i = 0;
    for (; i + kLoadBatch <= a.per_group; i += kLoadBatch) {
        typename ProbAcc<R>::V v[kLoadBatch];
#pragma unroll
        for (int k = 0; k < kLoadBatch; k++) {
            v[k] = ProbAcc<R>::load(s, xm | xo | xl);
            xo = ((xo | ~a.upper) + 1) & a.upper;
        }
#pragma unroll
        for (int k = 0; k < kLoadBatch; k++) pa.add(v[k]);
    }
    for (; i < a.per_group; i++) {
        pa.add(s, xm | xo | xl);
        xo = ((xo | ~a.upper) + 1) & a.upper;
    }
    double acc = pa.value();
#pragma unroll
    for (int off = 16; off; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
    if (lane == 0) partial[g * outcomes + ml] = acc;
}

__global__ void k_sum_groups(const double *__restrict__ partial, uint64_t outcomes, int groups,
                             double *__restrict__ out) {
    const uint64_t m = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= outcomes) return;
    double acc = 0.0;
    for (int g = 0; g < groups; g++) acc += partial[(uint64_t)g * outcomes + m];
    out[m] = acc;
}

// Block sums of x[0..len) (each thread sums a strided slice, then a fixed tree).
__global__ void __launch_bounds__(kRedThreads)
k_block_sum(const double *__restrict__ x, uint64_t len, double *__restrict__ sums) {
    __shared__ double sh[kRedThreads];
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    double acc = 0.0;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < len; i += stride)
        acc += x[i];
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int w = kRedThreads / 2; w; w >>= 1) {
        if ((int)threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) sums[blockIdx.x] = sh[0];
}

// Total of the block sums in a fixed order (one warp: lane l sums entries
// l, l + 32, ... in order, then a fixed shuffle tree), so every call gets the
// same bits.
__device__ __forceinline__ double ordered_total(const double *__restrict__ sums, int nsums) {
    double t = 0.0;
    for (int i = threadIdx.x & 31; i < nsums; i += 32) t += sums[i];
#pragma unroll
    for (int off = 16; off; off >>= 1) t += __shfl_xor_sync(0xffffffffu, t, off);
    return t;
}

__global__ void k_total(const double *__restrict__ sums, int nsums, double *__restrict__ total) {
    const double t = ordered_total(sums, nsums);
    if (threadIdx.x == 0) *total = t;
}

__global__ void k_normalise(double *__restrict__ p, uint64_t len, const double *__restrict__ total) {
    const double t = *total;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < len; i += stride)
        p[i] = p[i] / t;
}

// v[0] /= total (the same ordered total as the normalisation uses).
__global__ void k_div_total(double *v, const double *__restrict__ sums, int nsums) {
    const double t = ordered_total(sums, nsums);
    if (threadIdx.x == 0) v[0] = v[0] / t;
}

// argmax: (value, lowest index) per block, then one block over the partials.
__device__ __forceinline__ void better(double &v, uint64_t &i, double v2, uint64_t i2) {
    if (v2 > v || (v2 == v && i2 < i)) {
        v = v2;
        i = i2;
    }
}

// Output index of the entry at position i of a marginal ordered as p says.
__device__ __forceinline__ uint64_t output_index(uint64_t i, const OutPerm &p) {
    if (!p.m) return i;
    uint64_t r = 0;
    for (int k = 0; k < p.m; k++) r |= ((i >> k) & 1) << p.bit[k];
    return r;
}

__global__ void __launch_bounds__(kRedThreads)
k_argmax(const double *__restrict__ x, const uint64_t *__restrict__ xi, uint64_t len,
         double *__restrict__ ov, uint64_t *__restrict__ oi, const OutPerm perm) {
    __shared__ double sv_[kRedThreads];
    __shared__ uint64_t si[kRedThreads];
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    double v = -1.0;
    uint64_t idx = ~UINT64_C(0);
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < len; i += stride) {
        const double xv = x[i];
        // the output index (for ties: the lowest wins) only for a candidate
        if (xv >= v) better(v, idx, xv, xi ? xi[i] : output_index(i, perm));
    }
    sv_[threadIdx.x] = v;
    si[threadIdx.x] = idx;
    __syncthreads();
    for (int w = kRedThreads / 2; w; w >>= 1) {
        if ((int)threadIdx.x < w) {
            double v2 = sv_[threadIdx.x + w];
            uint64_t i2 = si[threadIdx.x + w];
            double v1 = sv_[threadIdx.x];
            uint64_t i1 = si[threadIdx.x];
            better(v1, i1, v2, i2);
            sv_[threadIdx.x] = v1;
            si[threadIdx.x] = i1;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        ov[blockIdx.x] = sv_[0];
        oi[blockIdx.x] = si[0];
    }
}

// CDF, step 1: one thread per block of 1024 outcomes.
__global__ void k_cdf_blocks(const double *__restrict__ p, uint64_t len, double *__restrict__ cdf,
                             double *__restrict__ btot) {
    const uint64_t b = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const uint64_t b0 = b * 1024;
    if (b0 >= len) return;
    const uint64_t b1 = b0 + 1024 < len ? b0 + 1024 : len;
    double run = 0.0;
    for (uint64_t i = b0; i < b1; i++) {
        run += p[i];
        cdf[i] = run;
    }
    btot[b] = run;
}

// CDF, step 2: exclusive running total over blocks, in block order.
__global__ void k_cdf_scan(double *__restrict__ btot, uint64_t nb) {
    double before = 0.0;
    for (uint64_t b = 0; b < nb; b++) {
        double t = btot[b];
        btot[b] = before;
        before += t;
    }
}

// CDF, step 3: C_i = (total before the block) + (in-block running sum).
__global__ void k_cdf_add(double *__restrict__ cdf, uint64_t len, const double *__restrict__ before) {
    const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < len) cdf[i] = before[i / 1024] + cdf[i];
}

__global__ void k_sample(const double *__restrict__ cdf, uint64_t len, const double *__restrict__ u,
                         uint64_t shots, uint64_t *__restrict__ out) {
    const uint64_t s = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= shots) return;
    const double target = u[s] * cdf[len - 1];
    uint64_t lo = 0, hi = len - 1;  // answer in [lo, hi]
    while (lo < hi) {
        uint64_t mid = lo + (hi - lo) / 2;
        if (cdf[mid] > target)
            hi = mid;
        else
            lo = mid + 1;
    }
    out[s] = lo;
}

unsigned blocks_for(uint64_t work, int threads) {
    uint64_t b = (work + threads - 1) / threads;
    return (unsigned)std::max<uint64_t>(1, std::min<uint64_t>(b, 0x7fffffffULL));
}

}  // namespace

sv_status ensure_scratch(sv_state *h, size_t bytes) {
    if (bytes <= h->scratch_cap) return SV_OK;
    if (h->scratch) {
        SV_CUDA(cudaStreamSynchronize(h->stream));
        cudaFree(h->scratch);
        h->scratch = nullptr;
        h->scratch_cap = 0;
    }
    size_t cap = std::max<size_t>(bytes, (size_t)1 << 20);
    if (dev_malloc(&h->scratch, cap) != cudaSuccess) {
        cudaGetLastError();
        h->scratch = nullptr;
        return fail(SV_ERR_OOM, "cannot allocate %zu bytes of device scratch", cap);
    }
    h->scratch_cap = cap;
    return SV_OK;
}

sv_status ensure_probs(sv_state *h, size_t bytes) {
    if (bytes <= h->probs_cap) return SV_OK;
    if (h->probs) {
        SV_CUDA(cudaStreamSynchronize(h->stream));
        cudaFree(h->probs);
        h->probs = nullptr;
        h->probs_cap = 0;
    }
    size_t cap = std::max<size_t>(bytes, (size_t)1 << 16);
    if (dev_malloc(&h->probs, cap) != cudaSuccess) {
        cudaGetLastError();
        h->probs = nullptr;
        return fail(SV_ERR_OOM, "cannot allocate %zu bytes for probabilities", cap);
    }
    h->probs_cap = cap;
    return SV_OK;
}

// pos[j]: physical bit of output bit j.
sv_status marginal_device(sv_state *h, const int *pos, int m, double *dev_out, bool normalise,
                          const double **sums_out, int *nsums_out, OutPerm *perm_out) {
    SV_TRY(materialize(h));
    const int n = h->n;
    MargArgs a{};
    a.n = n;
    a.m = m;
    // outcome bits sorted by physical position
    int order[34];
    for (int j = 0; j < m; j++) order[j] = j;
    std::sort(order, order + m, [&](int x, int y) { return pos[x] < pos[y]; });
    for (int k = 0; k < m; k++) {
        a.spos[k] = pos[order[k]];
        a.out_bit[k] = perm_out ? k : order[k];
        a.mask |= UINT64_C(1) << pos[order[k]];
    }
    if (perm_out) {
        perm_out->m = m;
        for (int k = 0; k < m; k++) perm_out->bit[k] = (int8_t)order[k];
    }
    const uint64_t all = (n == 64) ? ~UINT64_C(0) : ((UINT64_C(1) << n) - 1);
    a.rest = all & ~a.mask;
    const int rbits = n - m;
    const uint64_t outcomes = UINT64_C(1) << m;
    const bool layout_r = (a.mask & 1) == 0 && rbits >= 5;
    const int target_log2 = 19;  // ~5e5 threads (layout M) or lanes (layout R)
    int gl;
    if (layout_r) {
        uint64_t up = a.rest;
        for (int i = 0; i < 5; i++) up &= up - 1;  // drop the 5 lowest rest bits
        a.upper = up;
        int ubits = rbits - 5;
        gl = std::max(0, std::min(ubits, target_log2 - 5 - m));
        a.per_group = UINT64_C(1) << (ubits - gl);
    } else {
        gl = std::max(0, std::min(rbits, target_log2 - m));
        a.per_group = UINT64_C(1) << (rbits - gl);
    }
    a.groups_log2 = gl;
    const uint64_t groups = UINT64_C(1) << gl;

    double *partial = dev_out;
    size_t need = 0;
    if (groups > 1) need += groups * outcomes * sizeof(double);
    const int nsum_blocks = (int)std::min<uint64_t>(1024, blocks_for(outcomes, kRedThreads));
    const size_t sums_off = (need + 255) & ~(size_t)255;
    need = sums_off + (nsum_blocks + 1) * sizeof(double);
    SV_TRY(ensure_scratch(h, need));
    if (groups > 1) partial = reinterpret_cast<double *>(h->scratch);
    double *sums = reinterpret_cast<double *>(reinterpret_cast<char *>(h->scratch) + sums_off);

    // complex64 with physical bit 0 an outcome bit: two outcomes per thread
    const bool pairs = !layout_r && h->dt == SV_C64 && m >= 1 && a.spos[0] == 0;
    const uint64_t work = layout_r ? (outcomes << gl) * 32 : pairs ? ((outcomes >> 1) << gl) : (outcomes << gl);
    const unsigned grid = blocks_for(work, kRedThreads);
    if (h->dt == SV_C128) {
        const double *s = reinterpret_cast<const double *>(h->amps);
        if (layout_r)
            k_marg_r<double><<<grid, kRedThreads, 0, h->stream>>>(s, a, partial);
        else
            k_marg_m<double><<<grid, kRedThreads, 0, h->stream>>>(s, a, partial);
    } else {
        const float *s = reinterpret_cast<const float *>(h->amps);
        if (layout_r)
            k_marg_r<float><<<grid, kRedThreads, 0, h->stream>>>(s, a, partial);
        else if (pairs)
            k_marg_m2<<<grid, kRedThreads, 0, h->stream>>>(s, a, partial);
        else
            k_marg_m<float><<<grid, kRedThreads, 0, h->stream>>>(s, a, partial);
    }
    SV_CUDA(cudaGetLastError());
    note_launch();
    if (groups > 1) {
        k_sum_groups<<<blocks_for(outcomes, kRedThreads), kRedThreads, 0, h->stream>>>(
            partial, outcomes, (int)groups, dev_out);
        SV_CUDA(cudaGetLastError());
    note_launch();
    }
    k_block_sum<<<nsum_blocks, kRedThreads, 0, h->stream>>>(dev_out, outcomes, sums);
    SV_CUDA(cudaGetLastError());
    note_launch();
    if (sums_out) *sums_out = sums;
    if (nsums_out) *nsums_out = nsum_blocks;
    if (!normalise) return SV_OK;
    double *total = sums + nsum_blocks;
    k_total<<<1, 32, 0, h->stream>>>(sums, nsum_blocks, total);
    SV_CUDA(cudaGetLastError());
    note_launch();
    k_normalise<<<std::min<unsigned>(blocks_for(outcomes, kRedThreads), 4096), kRedThreads, 0,
                  h->stream>>>(dev_out, outcomes, total);
    SV_CUDA(cudaGetLastError());
    note_launch();
    return SV_OK;
}

sv_status argmax_device(sv_state *h, const double *dev_p, uint64_t len, uint64_t *host_idx,
                        double *host_p, const double *sums, int nsums, const OutPerm *perm) {
    OutPerm ident{};
    const OutPerm pm = perm ? *perm : ident;
    const int nb = (int)std::min<uint64_t>(1024, blocks_for(len, kRedThreads));
    char *base = reinterpret_cast<char *>(h->small);
    double *bv = reinterpret_cast<double *>(base);
    uint64_t *bi = reinterpret_cast<uint64_t *>(base + 8192);
    double *fv = reinterpret_cast<double *>(base + 16384);
    uint64_t *fi = reinterpret_cast<uint64_t *>(base + 16384 + 64);
    k_argmax<<<nb, kRedThreads, 0, h->stream>>>(dev_p, nullptr, len, bv, bi, pm);
    SV_CUDA(cudaGetLastError());
    note_launch();
    k_argmax<<<1, kRedThreads, 0, h->stream>>>(bv, bi, (uint64_t)nb, fv, fi, ident);
    SV_CUDA(cudaGetLastError());
    note_launch();
    if (sums) {  // unnormalised marginal: p = max / total, the total in the normalisation's order
        k_div_total<<<1, 32, 0, h->stream>>>(fv, sums, nsums);
        SV_CUDA(cudaGetLastError());
        note_launch();
    }
    double v;
    uint64_t i;
    SV_CUDA(cudaMemcpyAsync(&v, fv, sizeof v, cudaMemcpyDeviceToHost, h->stream));
    SV_CUDA(cudaMemcpyAsync(&i, fi, sizeof i, cudaMemcpyDeviceToHost, h->stream));
    SV_TRY(finish_sync(h));
    *host_idx = i;
    if (host_p) *host_p = v;
    return SV_OK;
}

sv_status sample_device(sv_state *h, const double *dev_p, uint64_t len, const double *host_u,
                        size_t shots, uint64_t *host_out) {
    const uint64_t nb = (len + 1023) / 1024;
    size_t off_cdf = 0;
    size_t off_bt = (len * sizeof(double) + 255) & ~(size_t)255;
    size_t off_u = (off_bt + nb * sizeof(double) + 255) & ~(size_t)255;
    size_t off_o = (off_u + shots * sizeof(double) + 255) & ~(size_t)255;
    size_t need = off_o + shots * sizeof(uint64_t);
    SV_TRY(ensure_scratch(h, need));
    char *base = reinterpret_cast<char *>(h->scratch);
    double *cdf = reinterpret_cast<double *>(base + off_cdf);
    double *bt = reinterpret_cast<double *>(base + off_bt);
    double *du = reinterpret_cast<double *>(base + off_u);
    uint64_t *dout = reinterpret_cast<uint64_t *>(base + off_o);
    k_cdf_blocks<<<blocks_for(nb, 128), 128, 0, h->stream>>>(dev_p, len, cdf, bt);
    SV_CUDA(cudaGetLastError());
    note_launch();
    k_cdf_scan<<<1, 1, 0, h->stream>>>(bt, nb);
    SV_CUDA(cudaGetLastError());
    note_launch();
    k_cdf_add<<<blocks_for(len, kRedThreads), kRedThreads, 0, h->stream>>>(cdf, len, bt);
    SV_CUDA(cudaGetLastError());
    note_launch();
    if (shots) {
        SV_CUDA(cudaMemcpyAsync(du, host_u, shots * sizeof(double), cudaMemcpyHostToDevice,
                                h->stream));
        k_sample<<<blocks_for(shots, 128), 128, 0, h->stream>>>(cdf, len, du, shots, dout);
        SV_CUDA(cudaGetLastError());
    note_launch();
        SV_CUDA(cudaMemcpyAsync(host_out, dout, shots * sizeof(uint64_t), cudaMemcpyDeviceToHost,
                                h->stream));
    }
    return finish_sync(h);
}

}  // namespace sv
