// Allocation-free marginal probabilities: sv_marginal_noalloc.
//
// Some callers cannot call cudaMalloc at the point where they want a
// read-out: a serving runtime that reserves all device memory up front and
// forbids further allocation, or host code that must not take the implicit
// device-wide synchronisation a cudaMalloc / cudaFree may cause.  For them
// this entry point computes the renormalised FP64 marginal that
// sv_probabilities_device computes, but takes the state buffer, the qubit map
// and the output buffer from the caller and keeps its partial sums in a fixed
// device array that lives in this file, so it allocates nothing.  The two
// agree to about 1e-13, not bit for bit: this file squares complex64
// components in FP64 and adds its groups in another order than measure.cu.
//
// The array's device address is looked up once per device and kept for the
// life of the process.  A cudaDeviceReset of that device unloads the module
// and ends the array's life, so the kept address is then stale: do not call
// this entry point on a device after resetting it.
//
// The array is shared by every call in the process on a given device and
// keeps the last call's contents.  Every slot a call reads has been written
// earlier in the same call, so nothing needs clearing; but two calls whose
// kernels overlap on the GPU (for example on two streams) race on it and
// must be ordered by the caller.
#include <algorithm>
#include <mutex>

#include "common.h"

namespace {

// Partial sums of the two-level reduction (1 MiB) plus 1024 block totals.
constexpr uint64_t kPartialDoubles = UINT64_C(1) << 17;
constexpr int kBlockSums = 1024;
static __device__ __align__(256) double g_noalloc_scratch[kPartialDoubles + kBlockSums];

constexpr int kThreads = 256;
constexpr int kMaxDevices = 64;
std::mutex g_setup_mu;
double *g_scratch_addr[kMaxDevices] = {};

struct Args {
    int m;
    uint64_t rest, upper;
    int spos[34];
    int out_bit[34];
    uint64_t per_group;
    int groups_log2;
};

__device__ __forceinline__ uint64_t deposit(uint64_t v, uint64_t mask) {
    uint64_t r = 0;
    for (uint64_t b = 1; mask; b <<= 1) {
        const uint64_t low = mask & (~mask + 1);
        if (v & b) r |= low;
        mask &= mask - 1;
    }
    return r;
}

template <typename R>
__device__ __forceinline__ double prob(const R *s, uint64_t x) {
    const double re = (double)s[2 * x], im = (double)s[2 * x + 1];
    return re * re + im * im;
}

__device__ __forceinline__ void outcome_bits(const Args &a, uint64_t mp, uint64_t *xm, uint64_t *ml) {
    uint64_t x = 0, o = 0;
    for (int k = 0; k < a.m; k++)
        if ((mp >> k) & 1) {
            x |= UINT64_C(1) << a.spos[k];
            o |= UINT64_C(1) << a.out_bit[k];
        }
    *xm = x;
    *ml = o;
}

// One thread per (group, outcome); outcome bit 0 is physical bit 0.
template <typename R>
__global__ void __launch_bounds__(kThreads)
k_na_marg_m(const R *__restrict__ s, Args a, double *__restrict__ dst) {
    const uint64_t outcomes = UINT64_C(1) << a.m;
    const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (tid >= (outcomes << a.groups_log2)) return;
    uint64_t xm, ml;
    outcome_bits(a, tid & (outcomes - 1), &xm, &ml);
    const uint64_t g = tid >> a.m;
    uint64_t xr = deposit(g * a.per_group, a.rest);
    double acc = 0.0;
    for (uint64_t i = 0; i < a.per_group; i++) {
        acc += prob(s, xm | xr);
        xr = ((xr | ~a.rest) + 1) & a.rest;
    }
    // dst is the static array when groups > 1, the caller's output otherwise
    dst[g * outcomes + ml] = acc;
}

// One warp per (group, outcome); lanes take the five lowest summed bits.
template <typename R>
__global__ void __launch_bounds__(kThreads)
k_na_marg_r(const R *__restrict__ s, Args a, double *__restrict__ dst) {
    const uint64_t outcomes = UINT64_C(1) << a.m;
    const uint64_t warp = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (warp >= (outcomes << a.groups_log2)) return;
    uint64_t xm, ml;
    outcome_bits(a, warp & (outcomes - 1), &xm, &ml);
    const uint64_t g = warp >> a.m;
    const uint64_t xl = deposit((uint64_t)lane, a.rest & ~a.upper);
    uint64_t xo = deposit(g * a.per_group, a.upper);
    double acc = 0.0;
    for (uint64_t i = 0; i < a.per_group; i++) {
        acc += prob(s, xm | xo | xl);
        xo = ((xo | ~a.upper) + 1) & a.upper;
    }
#pragma unroll
    for (int off = 16; off; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
    if (lane == 0) dst[g * outcomes + ml] = acc;
}

// out[m] = sum over groups of the static partial sums, in group order.
__global__ void k_na_sum_groups(uint64_t outcomes, int groups, double *__restrict__ out) {
    const uint64_t m = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= outcomes) return;
    double acc = 0.0;
    for (int g = 0; g < groups; g++) acc += g_noalloc_scratch[(uint64_t)g * outcomes + m];
    out[m] = acc;
}

// Block totals of out[] into the tail of the static array (fixed tree).
__global__ void __launch_bounds__(kThreads)
k_na_block_sum(const double *__restrict__ x, uint64_t len) {
    __shared__ double sh[kThreads];
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    double acc = 0.0;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < len; i += stride)
        acc += x[i];
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int w = kThreads / 2; w; w >>= 1) {
        if ((int)threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) g_noalloc_scratch[kPartialDoubles + blockIdx.x] = sh[0];
}

__global__ void k_na_normalise(double *__restrict__ p, uint64_t len, int nsums) {
    __shared__ double total;
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int i = 0; i < nsums; i++) t += g_noalloc_scratch[kPartialDoubles + i];
        total = t;
    }
    __syncthreads();
    const double t = total;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < len; i += stride)
        p[i] = p[i] / t;
}

unsigned nblocks(uint64_t work) {
    const uint64_t b = (work + kThreads - 1) / kThreads;
    return (unsigned)std::max<uint64_t>(1, std::min<uint64_t>(b, 0x7fffffffULL));
}

// Device address of the static array on the current device (set-up once
// per device, with that device current).
sv_status scratch_address(double **out) {
    int dev = 0;
    SV_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return sv::fail(SV_ERR_UNSUPPORTED, "device %d", dev);
    std::lock_guard<std::mutex> lock(g_setup_mu);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p)
            return sv::fail(SV_ERR_CUDA, "cudaGetSymbolAddress(g_noalloc_scratch) failed: %s",
                            cudaGetErrorString(e));
        g_scratch_addr[dev] = reinterpret_cast<double *>(p);
    }
    *out = g_scratch_addr[dev];
    return SV_OK;
}

}  // namespace

using sv::fail;

extern "C" sv_status sv_marginal_noalloc(const void *dev_amps, int n, sv_dtype dt,
                                         const int *host_phys_of_logical, uint64_t qubit_mask,
                                         double *dev_out, void *cuda_stream) {
    sv::clear_error();
    if (!dev_amps || !dev_out) return fail(SV_ERR_ARG, "NULL device pointer");
    if (n < 1 || n > 34) return fail(SV_ERR_ARG, "n=%d outside 1..34", n);
    if (dt != SV_C64 && dt != SV_C128) return fail(SV_ERR_ARG, "unknown dtype %d", (int)dt);
    if (!qubit_mask) return fail(SV_ERR_ARG, "qubit_mask is empty");
    if (qubit_mask >> n) return fail(SV_ERR_ARG, "qubit_mask has bits beyond n=%d", n);
    const int m = __builtin_popcountll(qubit_mask);
    if (m > 30) return fail(SV_ERR_ARG, "qubit_mask selects more than 30 qubits");
    if ((uintptr_t)dev_amps % 16) return fail(SV_ERR_ARG, "dev_amps not 16-byte aligned");
    int phys[64];
    bool seen[64] = {};
    for (int q = 0; q < n; q++) {
        phys[q] = host_phys_of_logical ? host_phys_of_logical[q] : q;
        if (phys[q] < 0 || phys[q] >= n || seen[phys[q]])
            return fail(SV_ERR_ARG, "qubit map is not a permutation of 0..%d", n - 1);
        seen[phys[q]] = true;
    }
    // outcome bit j <-> physical position of the j-th lowest logical qubit of the mask
    int pos[34], order[34];
    int j = 0;
    for (int q = 0; q < n; q++)
        if ((qubit_mask >> q) & 1) pos[j++] = phys[q];
    for (int i = 0; i < m; i++) order[i] = i;
    std::sort(order, order + m, [&](int x, int y) { return pos[x] < pos[y]; });
    Args a{};
    a.m = m;
    uint64_t maskp = 0;
    for (int k = 0; k < m; k++) {
        a.spos[k] = pos[order[k]];
        a.out_bit[k] = order[k];
        maskp |= UINT64_C(1) << pos[order[k]];
    }
    a.rest = ((UINT64_C(1) << n) - 1) & ~maskp;
    const int rbits = n - m;
    const uint64_t outcomes = UINT64_C(1) << m;
    const bool layout_r = (maskp & 1) == 0 && rbits >= 5;
    // groups: as many as the static array holds, up to ~2^19 threads of work
    const int cap_log2 = 17 - std::min(m, 17);  // groups * outcomes <= 2^17
    int gl;
    if (layout_r) {
        uint64_t up = a.rest;
        for (int i = 0; i < 5; i++) up &= up - 1;
        a.upper = up;
        gl = std::max(0, std::min({rbits - 5, 19 - 5 - m, cap_log2}));
        a.per_group = UINT64_C(1) << (rbits - 5 - gl);
    } else {
        gl = std::max(0, std::min({rbits, 19 - m, cap_log2}));
        a.per_group = UINT64_C(1) << (rbits - gl);
    }
    a.groups_log2 = gl;
    const uint64_t groups = UINT64_C(1) << gl;
    if (groups > 1 && groups * outcomes > kPartialDoubles)
        return fail(SV_ERR_ARG, "partial sums need %llu doubles, the static array holds %llu",
                    (unsigned long long)(groups * outcomes), (unsigned long long)kPartialDoubles);

    double *scratch = nullptr;
    sv_status st = scratch_address(&scratch);
    if (st != SV_OK) return st;
    cudaStream_t stream = reinterpret_cast<cudaStream_t>(cuda_stream);
    double *dst = groups > 1 ? scratch : dev_out;
    const uint64_t work = layout_r ? (outcomes << gl) * 32 : (outcomes << gl);
    if (dt == SV_C128) {
        const double *s = reinterpret_cast<const double *>(dev_amps);
        if (layout_r)
            k_na_marg_r<double><<<nblocks(work), kThreads, 0, stream>>>(s, a, dst);
        else
            k_na_marg_m<double><<<nblocks(work), kThreads, 0, stream>>>(s, a, dst);
    } else {
        const float *s = reinterpret_cast<const float *>(dev_amps);
        if (layout_r)
            k_na_marg_r<float><<<nblocks(work), kThreads, 0, stream>>>(s, a, dst);
        else
            k_na_marg_m<float><<<nblocks(work), kThreads, 0, stream>>>(s, a, dst);
    }
    SV_CUDA(cudaGetLastError());
    sv::note_launch();
    if (groups > 1) {
        k_na_sum_groups<<<nblocks(outcomes), kThreads, 0, stream>>>(outcomes, (int)groups, dev_out);
        SV_CUDA(cudaGetLastError());
        sv::note_launch();
    }
    const int nsum = (int)std::min<uint64_t>(kBlockSums, nblocks(outcomes));
    k_na_block_sum<<<nsum, kThreads, 0, stream>>>(dev_out, outcomes);
    SV_CUDA(cudaGetLastError());
    sv::note_launch();
    k_na_normalise<<<std::min<unsigned>(nblocks(outcomes), 4096), kThreads, 0, stream>>>(
        dev_out, outcomes, nsum);
    SV_CUDA(cudaGetLastError());
    sv::note_launch();
    return SV_OK;
}
