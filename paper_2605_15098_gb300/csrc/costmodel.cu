// Cost model: a 3-layer MLP that predicts the duration of a launch.
//
// Training and inference run in the kernels below, in FP32:
//  * k_mlp_forward: inference, 64 samples per CTA step;
//  * k_mlp_grad: forward and backward over a slice of a minibatch; each CTA
//    keeps the gradient of the parameters it owns in registers across its
//    chunks of 64 samples and writes one partial gradient vector;
//  * k_mlp_adam: sums the partial gradients in a fixed order and applies one
//    Adam step (Kingma and Ba 2015, Algorithm 1), or only returns the
//    gradient.
// The network is small (7,617 parameters), so the work is kept on the CUDA
// cores; activations of a 64-sample chunk live in shared memory.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>

#include "common.h"

namespace sv {
namespace {

constexpr int NF = SV_COST_FEATURES;
constexpr int HD = SV_COST_HIDDEN;
constexpr int NP = SV_COST_PARAMS;
constexpr int OW1 = 0;
constexpr int OB1 = OW1 + NF * HD;
constexpr int OW2 = OB1 + HD;
constexpr int OB2 = OW2 + HD * HD;
constexpr int OW3 = OB2 + HD;
constexpr int OB3 = OW3 + HD;
static_assert(OB3 + 1 == NP, "parameter layout");

constexpr int kThreads = 256;
constexpr int kRows = 64;             // samples per chunk
constexpr int kW2Stride = HD + 1;     // padded rows of W2 in shared memory
constexpr int kOwn = (NP + kThreads - 1) / kThreads;  // parameters per thread

// Shared-memory layout (floats).
struct Smem {
    static constexpr int w1 = 0;
    static constexpr int b1 = w1 + NF * HD;
    static constexpr int w2 = b1 + HD;
    static constexpr int b2 = w2 + HD * kW2Stride;
    static constexpr int w3 = b2 + HD;
    static constexpr int b3 = w3 + HD;
    static constexpr int x = b3 + 4;
    static constexpr int h1 = x + kRows * NF;
    static constexpr int h2 = h1 + kRows * HD;
    static constexpr int d2 = h2 + kRows * HD;
    static constexpr int d1 = d2 + kRows * HD;
    static constexpr int dy = d1 + kRows * HD;
    static constexpr int red = dy + kRows;
    static constexpr int fwd_total = d2;          // inference needs x, h1, h2
    static constexpr int total = red + kThreads;  // training
};

__device__ void load_params(float *sm, const float *__restrict__ P) {
    for (int i = threadIdx.x; i < NF * HD; i += blockDim.x) sm[Smem::w1 + i] = P[OW1 + i];
    for (int i = threadIdx.x; i < HD * HD; i += blockDim.x)
        sm[Smem::w2 + (i / HD) * kW2Stride + (i % HD)] = P[OW2 + i];
    for (int i = threadIdx.x; i < HD; i += blockDim.x) {
        sm[Smem::b1 + i] = P[OB1 + i];
        sm[Smem::b2 + i] = P[OB2 + i];
        sm[Smem::w3 + i] = P[OW3 + i];
    }
    if (threadIdx.x == 0) sm[Smem::b3] = P[OB3];
}

// Rows [0, rows) of the chunk: x, then h1 = relu(x W1 + b1), h2 = relu(h1 W2 + b2).
// Thread t computes column j = t % 64 of rows t/64, t/64 + 4, ...
__device__ void forward_hidden(float *sm) {
    const int j = threadIdx.x & (HD - 1);
    const int r0 = threadIdx.x >> 6;
    constexpr int R = kRows / (kThreads / HD);  // 16 rows per thread
    float acc[R];
#pragma unroll
    for (int r = 0; r < R; r++) acc[r] = sm[Smem::b1 + j];
    for (int i = 0; i < NF; i++) {
        const float w = sm[Smem::w1 + i * HD + j];
#pragma unroll
        for (int r = 0; r < R; r++) acc[r] = fmaf(sm[Smem::x + (r0 + 4 * r) * NF + i], w, acc[r]);
    }
#pragma unroll
    for (int r = 0; r < R; r++) sm[Smem::h1 + (r0 + 4 * r) * HD + j] = fmaxf(acc[r], 0.f);
    __syncthreads();
#pragma unroll
    for (int r = 0; r < R; r++) acc[r] = sm[Smem::b2 + j];
    for (int i = 0; i < HD; i++) {
        const float w = sm[Smem::w2 + i * kW2Stride + j];
#pragma unroll
        for (int r = 0; r < R; r++) acc[r] = fmaf(sm[Smem::h1 + (r0 + 4 * r) * HD + i], w, acc[r]);
    }
#pragma unroll
    for (int r = 0; r < R; r++) sm[Smem::h2 + (r0 + 4 * r) * HD + j] = fmaxf(acc[r], 0.f);
    __syncthreads();
}

// y for row t/4 (4 threads per row, 16 columns each, reduced by shuffles);
// valid in the thread with t % 4 == 0.
__device__ float forward_out(const float *sm) {
    const int row = threadIdx.x >> 2, q = threadIdx.x & 3;
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < HD / 4; c++) {
        const int j = q * (HD / 4) + c;
        s = fmaf(sm[Smem::h2 + row * HD + j], sm[Smem::w3 + j], s);
    }
    s += __shfl_down_sync(0xffffffffu, s, 2);
    s += __shfl_down_sync(0xffffffffu, s, 1);
    return s + sm[Smem::b3];
}

__device__ void load_rows(float *sm, const float *__restrict__ X, const int *__restrict__ idx,
                          long long first, long long count) {
    for (int e = threadIdx.x; e < kRows * NF; e += blockDim.x) {
        const int r = e / NF, f = e % NF;
        const long long s = first + r;
        float v = 0.f;
        if (s < count) {
            const long long row = idx ? idx[s] : s;
            v = X[row * NF + f];
        }
        sm[Smem::x + e] = v;
    }
}

__global__ void __launch_bounds__(kThreads)
k_mlp_forward(const float *__restrict__ X, const float *__restrict__ P, float *__restrict__ Y,
              long long count) {
    extern __shared__ float sm[];
    load_params(sm, P);
    const long long chunks = (count + kRows - 1) / kRows;
    for (long long ch = blockIdx.x; ch < chunks; ch += gridDim.x) {
        __syncthreads();
        load_rows(sm, X, nullptr, ch * kRows, count);
        __syncthreads();
        forward_hidden(sm);
        const float y = forward_out(sm);
        const long long s = ch * kRows + (threadIdx.x >> 2);
        if ((threadIdx.x & 3) == 0 && s < count) Y[s] = y;
    }
}

// Forward and backward over chunks blockIdx.x, blockIdx.x + gridDim.x, ...
// of the `count` samples (rows idx[s] of X when idx is given).  The loss is
// the mean over `count` (inv_n = 1 / count).  Thread t owns parameters
// t, t + 256, ...; their gradient stays in registers until the end.
__global__ void __launch_bounds__(kThreads)
k_mlp_grad(const float *__restrict__ X, const float *__restrict__ T, const int *__restrict__ idx,
           long long count, float inv_n, const float *__restrict__ P, float *__restrict__ Gpart,
           float *__restrict__ Lpart) {
    extern __shared__ float sm[];
    load_params(sm, P);
    float acc[kOwn];
#pragma unroll
    for (int r = 0; r < kOwn; r++) acc[r] = 0.f;
    float lsum = 0.f;
    const int t = threadIdx.x;
    const long long chunks = (count + kRows - 1) / kRows;
    for (long long ch = blockIdx.x; ch < chunks; ch += gridDim.x) {
        __syncthreads();
        load_rows(sm, X, idx, ch * kRows, count);
        __syncthreads();
        forward_hidden(sm);
        const float y = forward_out(sm);
        if ((t & 3) == 0) {
            const int row = t >> 2;
            const long long s = ch * kRows + row;
            float d = 0.f;
            if (s < count) {
                const float e = y - T[idx ? idx[s] : s];
                lsum = fmaf(e * e, inv_n, lsum);
                d = 2.f * e * inv_n;
            }
            sm[Smem::dy + row] = d;
        }
        __syncthreads();
        // dL/dz2 = dy * W3 * relu'(z2)
        for (int e = t; e < kRows * HD; e += kThreads) {
            const int b = e / HD, j = e % HD;
            sm[Smem::d2 + e] = sm[Smem::h2 + e] > 0.f ? sm[Smem::dy + b] * sm[Smem::w3 + j] : 0.f;
        }
        __syncthreads();
        // dL/dz1 = (dL/dz2 W2^T) * relu'(z1)
        {
            const int i = t & (HD - 1);
            const int r0 = t >> 6;
            constexpr int R = kRows / (kThreads / HD);
            float a[R];
#pragma unroll
            for (int r = 0; r < R; r++) a[r] = 0.f;
            for (int j = 0; j < HD; j++) {
                const float w = sm[Smem::w2 + i * kW2Stride + j];
#pragma unroll
                for (int r = 0; r < R; r++) a[r] = fmaf(sm[Smem::d2 + (r0 + 4 * r) * HD + j], w, a[r]);
            }
#pragma unroll
            for (int r = 0; r < R; r++) {
                const int e = (r0 + 4 * r) * HD + i;
                sm[Smem::d1 + e] = sm[Smem::h1 + e] > 0.f ? a[r] : 0.f;
            }
        }
        __syncthreads();
        // accumulate the owned parameters' gradients over the chunk
#pragma unroll
        for (int r = 0; r < kOwn; r++) {
            const int p = t + kThreads * r;
            if (p >= NP) break;
            float s = 0.f;
            if (p < OB1) {
                const int i = p / HD, j = p % HD;
                for (int b = 0; b < kRows; b++) s = fmaf(sm[Smem::x + b * NF + i], sm[Smem::d1 + b * HD + j], s);
            } else if (p < OW2) {
                const int j = p - OB1;
                for (int b = 0; b < kRows; b++) s += sm[Smem::d1 + b * HD + j];
            } else if (p < OB2) {
                const int q = p - OW2, i = q / HD, j = q % HD;
                for (int b = 0; b < kRows; b++) s = fmaf(sm[Smem::h1 + b * HD + i], sm[Smem::d2 + b * HD + j], s);
            } else if (p < OW3) {
                const int j = p - OB2;
                for (int b = 0; b < kRows; b++) s += sm[Smem::d2 + b * HD + j];
            } else if (p < OB3) {
                const int j = p - OW3;
                for (int b = 0; b < kRows; b++) s = fmaf(sm[Smem::h2 + b * HD + j], sm[Smem::dy + b], s);
            } else {
                for (int b = 0; b < kRows; b++) s += sm[Smem::dy + b];
            }
            acc[r] += s;
        }
    }
#pragma unroll
    for (int r = 0; r < kOwn; r++) {
        const int p = t + kThreads * r;
        if (p < NP) Gpart[(size_t)blockIdx.x * NP + p] = acc[r];
    }
    __syncthreads();
    sm[Smem::red + t] = lsum;
    __syncthreads();
    if (t == 0) {
        float s = 0.f;
        for (int i = 0; i < kThreads; i++) s += sm[Smem::red + i];
        Lpart[blockIdx.x] = s;
    }
}

// Sum the G partial gradients (in block order) and, when lr > 0, take one
// Adam step; bc1 = 1 - beta1^t and bc2 = 1 - beta2^t come from the host.
__global__ void k_mlp_adam(const float *__restrict__ Gpart, int G, float *__restrict__ P,
                           float *__restrict__ M, float *__restrict__ V, float lr, float beta1,
                           float beta2, float eps, float bc1, float bc2, float *__restrict__ gout,
                           const float *__restrict__ Lpart, double *__restrict__ loss_acc,
                           double loss_w) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p < NP) {
        float g = 0.f;
        for (int b = 0; b < G; b++) g += Gpart[(size_t)b * NP + p];
        if (gout) gout[p] = g;
        if (lr > 0.f) {
            const float m = beta1 * M[p] + (1.f - beta1) * g;
            const float v = beta2 * V[p] + (1.f - beta2) * g * g;
            M[p] = m;
            V[p] = v;
            P[p] -= lr * (m / bc1) / (sqrtf(v / bc2) + eps);
        }
    }
    if (p == 0 && loss_acc) {
        double s = 0.0;
        for (int b = 0; b < G; b++) s += Lpart[b];
        *loss_acc += s * loss_w;
    }
}

}  // namespace
}  // namespace sv

// ---- host side ------------------------------------------------------------

struct sv_cost_model_s {
    int device = 0;
    int sm_count = 0;
    cudaStream_t stream = nullptr;
    float *P = nullptr, *M = nullptr, *V = nullptr;  // parameters, Adam moments
    long long step = 0;                              // Adam steps taken
    // growable work buffers
    float *X = nullptr, *T = nullptr, *Y = nullptr, *G = nullptr, *L = nullptr, *gout = nullptr;
    int *idx = nullptr;
    double *loss = nullptr;
    size_t x_cap = 0, g_cap = 0;
};

namespace sv {
namespace {

uint64_t splitmix_next(uint64_t &s) {
    uint64_t z = (s += 0x9E3779B97F4A7C15ULL);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

double splitmix_uniform(uint64_t &s) { return (double)(splitmix_next(s) >> 11) * 0x1p-53; }

size_t smem_train() { return (size_t)Smem::total * sizeof(float); }
size_t smem_fwd() { return (size_t)Smem::fwd_total * sizeof(float); }

sv_status ensure_rows(sv_cost_model_s *m, size_t count) {
    if (count <= m->x_cap) return SV_OK;
    cudaFree(m->X);
    cudaFree(m->T);
    cudaFree(m->Y);
    cudaFree(m->idx);
    m->X = m->T = m->Y = nullptr;
    m->idx = nullptr;
    m->x_cap = 0;
    const size_t cap = std::max<size_t>(count, 1024);
    if (dev_malloc(&m->X, cap * NF * sizeof(float)) != cudaSuccess ||
        dev_malloc(&m->T, cap * sizeof(float)) != cudaSuccess ||
        dev_malloc(&m->Y, cap * sizeof(float)) != cudaSuccess ||
        dev_malloc(&m->idx, cap * sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        return fail(SV_ERR_OOM, "cost model: cannot allocate %zu sample rows", cap);
    }
    m->x_cap = cap;
    return SV_OK;
}

sv_status ensure_partials(sv_cost_model_s *m, size_t blocks) {
    if (blocks <= m->g_cap) return SV_OK;
    cudaFree(m->G);
    cudaFree(m->L);
    m->G = m->L = nullptr;
    m->g_cap = 0;
    if (dev_malloc(&m->G, blocks * NP * sizeof(float)) != cudaSuccess ||
        dev_malloc(&m->L, blocks * sizeof(float)) != cudaSuccess) {
        cudaGetLastError();
        return fail(SV_ERR_OOM, "cost model: cannot allocate gradient partials");
    }
    m->g_cap = blocks;
    return SV_OK;
}

int grad_blocks(const sv_cost_model_s *m, long long count) {
    const long long chunks = (count + kRows - 1) / kRows;
    return (int)std::max<long long>(1, std::min<long long>(chunks, 2LL * m->sm_count));
}

// One gradient evaluation over `count` samples (rows idx[first..] of the
// resident X when use_idx), followed by an Adam step when lr > 0.
sv_status grad_step(sv_cost_model_s *m, const int *idx, long long count, float lr, float b1,
                    float b2, float eps, float *gout, double loss_w) {
    const int G = grad_blocks(m, count);
    SV_TRY(ensure_partials(m, G));
    k_mlp_grad<<<G, kThreads, smem_train(), m->stream>>>(m->X, m->T, idx, count,
                                                        1.0f / (float)count, m->P, m->G, m->L);
    SV_CUDA(cudaGetLastError());
    note_launch();
    float bc1 = 1.f, bc2 = 1.f;
    if (lr > 0.f) {
        m->step++;
        bc1 = (float)(1.0 - std::pow((double)b1, (double)m->step));
        bc2 = (float)(1.0 - std::pow((double)b2, (double)m->step));
    }
    k_mlp_adam<<<(NP + 255) / 256, 256, 0, m->stream>>>(m->G, G, m->P, m->M, m->V, lr, b1, b2, eps,
                                                        bc1, bc2, gout, m->L, m->loss, loss_w);
    SV_CUDA(cudaGetLastError());
    note_launch();
    return SV_OK;
}

}  // namespace

// Features of one launch: see sv.h.  The same function describes candidate
// passes at planning time and recorded launches at training time.
void cost_features(const sv_launch_record &r, float *f) {
    for (int i = 0; i < NF; i++) f[i] = 0.f;
    for (int q = 0; q < 32; q++) f[q] = (float)((r.feat >> q) & 1);
    int top = -1;
    for (int q = 63; q >= 0; q--)
        if ((r.feat >> q) & 1) {
            top = q;
            break;
        }
    const int k = r.k > 0 ? r.k : 13;
    f[32 + (top < 5 ? 0 : top < 10 ? 1 : top < k ? 2 : 3)] = 1.f;
    f[36] = r.generated ? 1.f : 0.f;  // generated its state: no reads
    f[37] = r.dtype == SV_C128 ? 1.f : 0.f;
    int fam = 0;  // per-gate
    if (r.kind == SV_KERNEL_REMAP) fam = 4;
    else if (r.kind == SV_KERNEL_FUSED || r.gate_kind == -3) fam = 3;
    else if (r.kind == SV_KERNEL_TILE) fam = r.gate_kind == -2 ? 2 : 1;
    f[38 + fam] = 1.f;
    auto lg = [](double v) { return (float)std::log2(1.0 + std::max(0.0, v)); };
    f[43] = lg(r.ngates) / 8.f;
    f[44] = lg(r.nins) / 10.f;
    f[45] = lg(r.stages) / 6.f;
    f[46] = lg(r.blocks) / 8.f;
    f[47] = (float)r.c / 16.f;
    f[48] = (float)(r.n - 20) / 10.f;
    f[49] = (float)r.k / 16.f;
    f[50] = lg(r.nfactors) / 10.f;
    f[51] = (float)std::max(0, r.k - r.c) / 16.f;
}

// Predict `count` rows already in m->X; results to host_y.
sv_status cost_predict_rows(sv_cost_model_s *m, size_t count, float *host_y) {
    if (!count) return SV_OK;
    const long long chunks = ((long long)count + kRows - 1) / kRows;
    const int grid = (int)std::min<long long>(chunks, 2LL * m->sm_count);
    k_mlp_forward<<<grid, kThreads, smem_fwd(), m->stream>>>(m->X, m->P, m->Y, (long long)count);
    SV_CUDA(cudaGetLastError());
    note_launch();
    SV_CUDA(cudaMemcpyAsync(host_y, m->Y, count * sizeof(float), cudaMemcpyDeviceToHost, m->stream));
    SV_CUDA(cudaStreamSynchronize(m->stream));
    return SV_OK;
}

sv_status cost_predict(sv_cost_model_s *m, const float *host_x, size_t count, float *host_y) {
    if (!count) return SV_OK;
    SV_TRY(ensure_rows(m, count));
    SV_CUDA(cudaMemcpyAsync(m->X, host_x, count * NF * sizeof(float), cudaMemcpyHostToDevice,
                            m->stream));
    return cost_predict_rows(m, count, host_y);
}

}  // namespace sv

using namespace sv;

extern "C" {

sv_status sv_cost_features(const sv_launch_record *rec, float *host_out) {
    clear_error();
    if (!rec || !host_out) return fail(SV_ERR_ARG, "NULL argument");
    cost_features(*rec, host_out);
    return SV_OK;
}

sv_status sv_cost_model_destroy(sv_cost_model m) {
    clear_error();
    if (!m) return SV_OK;
    if (m->stream) cudaStreamSynchronize(m->stream);
    cudaFree(m->P);
    cudaFree(m->M);
    cudaFree(m->V);
    cudaFree(m->X);
    cudaFree(m->T);
    cudaFree(m->Y);
    cudaFree(m->G);
    cudaFree(m->L);
    cudaFree(m->gout);
    cudaFree(m->idx);
    cudaFree(m->loss);
    if (m->stream) cudaStreamDestroy(m->stream);
    delete m;
    return SV_OK;
}

sv_status sv_cost_model_create(uint64_t seed, sv_cost_model *out) {
    clear_error();
    if (!out) return fail(SV_ERR_ARG, "NULL argument");
    *out = nullptr;
    auto *m = new sv_cost_model_s();
    auto bail = [&](sv_status st) {
        sv_cost_model_destroy(m);
        return st;
    };
    cudaError_t e = cudaGetDevice(&m->device);
    if (e == cudaSuccess)
        e = cudaDeviceGetAttribute(&m->sm_count, cudaDevAttrMultiProcessorCount, m->device);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&m->stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = dev_malloc(&m->P, NP * sizeof(float));
    if (e == cudaSuccess) e = dev_malloc(&m->M, NP * sizeof(float));
    if (e == cudaSuccess) e = dev_malloc(&m->V, NP * sizeof(float));
    if (e == cudaSuccess) e = dev_malloc(&m->gout, NP * sizeof(float));
    if (e == cudaSuccess) e = dev_malloc(&m->loss, sizeof(double));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_mlp_grad, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem_train());
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_mlp_forward, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem_fwd());
    if (e != cudaSuccess) {
        cudaGetLastError();
        return bail(fail(SV_ERR_CUDA, "cost model: %s", cudaGetErrorString(e)));
    }
    // He-uniform weights: U(-sqrt(6 / fan_in), +sqrt(6 / fan_in)); zero biases
    std::vector<float> p(NP, 0.f);
    uint64_t s = seed;
    auto fill = [&](int off, int cnt, int fan_in) {
        const double a = std::sqrt(6.0 / fan_in);
        for (int i = 0; i < cnt; i++) p[off + i] = (float)((2.0 * splitmix_uniform(s) - 1.0) * a);
    };
    fill(OW1, NF * HD, NF);
    fill(OW2, HD * HD, HD);
    fill(OW3, HD, HD);
    if (cudaMemcpy(m->P, p.data(), NP * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemset(m->M, 0, NP * sizeof(float)) != cudaSuccess ||
        cudaMemset(m->V, 0, NP * sizeof(float)) != cudaSuccess) {
        cudaGetLastError();
        return bail(fail(SV_ERR_CUDA, "cost model: cannot initialise parameters"));
    }
    *out = m;
    return SV_OK;
}

sv_status sv_cost_model_get_params(sv_cost_model m, float *host_params) {
    clear_error();
    if (!m || !host_params) return fail(SV_ERR_ARG, "NULL argument");
    SV_CUDA(cudaMemcpyAsync(host_params, m->P, NP * sizeof(float), cudaMemcpyDeviceToHost, m->stream));
    SV_CUDA(cudaStreamSynchronize(m->stream));
    return SV_OK;
}

sv_status sv_cost_model_set_params(sv_cost_model m, const float *host_params) {
    clear_error();
    if (!m || !host_params) return fail(SV_ERR_ARG, "NULL argument");
    for (int i = 0; i < NP; i++)
        if (!std::isfinite(host_params[i])) return fail(SV_ERR_ARG, "parameter %d is not finite", i);
    SV_CUDA(cudaMemcpyAsync(m->P, host_params, NP * sizeof(float), cudaMemcpyHostToDevice, m->stream));
    SV_CUDA(cudaMemsetAsync(m->M, 0, NP * sizeof(float), m->stream));
    SV_CUDA(cudaMemsetAsync(m->V, 0, NP * sizeof(float), m->stream));
    SV_CUDA(cudaStreamSynchronize(m->stream));
    m->step = 0;
    return SV_OK;
}

sv_status sv_cost_model_predict(sv_cost_model m, const float *host_x, size_t count, float *host_y) {
    clear_error();
    if (!m || (count && (!host_x || !host_y))) return fail(SV_ERR_ARG, "NULL argument");
    return cost_predict(m, host_x, count, host_y);
}

sv_status sv_cost_model_gradient(sv_cost_model m, const float *host_x, const float *host_t,
                                 size_t count, float *host_grad, double *host_loss) {
    clear_error();
    if (!m || !host_grad || !host_x || !host_t) return fail(SV_ERR_ARG, "NULL argument");
    if (count == 0 || count > (size_t)1 << 30) return fail(SV_ERR_ARG, "count must be in 1..2^30");
    SV_TRY(ensure_rows(m, count));
    SV_CUDA(cudaMemcpyAsync(m->X, host_x, count * NF * sizeof(float), cudaMemcpyHostToDevice, m->stream));
    SV_CUDA(cudaMemcpyAsync(m->T, host_t, count * sizeof(float), cudaMemcpyHostToDevice, m->stream));
    SV_CUDA(cudaMemsetAsync(m->loss, 0, sizeof(double), m->stream));
    SV_TRY(grad_step(m, nullptr, (long long)count, 0.f, 0.f, 0.f, 0.f, m->gout, 1.0));
    double l = 0.0;
    SV_CUDA(cudaMemcpyAsync(host_grad, m->gout, NP * sizeof(float), cudaMemcpyDeviceToHost, m->stream));
    SV_CUDA(cudaMemcpyAsync(&l, m->loss, sizeof(double), cudaMemcpyDeviceToHost, m->stream));
    SV_CUDA(cudaStreamSynchronize(m->stream));
    if (host_loss) *host_loss = l;
    return SV_OK;
}

sv_status sv_cost_model_train(sv_cost_model m, const float *host_x, const float *host_t,
                              size_t count, const sv_train_config *cfg, float *host_epoch_loss) {
    clear_error();
    if (!m || !host_x || !host_t) return fail(SV_ERR_ARG, "NULL argument");
    if (count == 0 || count > (size_t)1 << 30) return fail(SV_ERR_ARG, "count must be in 1..2^30");
    sv_train_config c{};
    if (cfg) c = *cfg;
    const int epochs = c.epochs > 0 ? c.epochs : 100;
    const long long batch = c.batch > 0 ? c.batch : 4096;
    const float lr = c.lr > 0.f ? c.lr : 1e-3f;
    const float b1 = c.beta1 > 0.f ? c.beta1 : 0.9f;
    const float b2 = c.beta2 > 0.f ? c.beta2 : 0.999f;
    const float eps = c.eps > 0.f ? c.eps : 1e-8f;
    if (!(b1 < 1.f && b2 < 1.f)) return fail(SV_ERR_ARG, "beta1 and beta2 must be below 1");
    SV_TRY(ensure_rows(m, count));
    SV_CUDA(cudaMemcpyAsync(m->X, host_x, count * NF * sizeof(float), cudaMemcpyHostToDevice, m->stream));
    SV_CUDA(cudaMemcpyAsync(m->T, host_t, count * sizeof(float), cudaMemcpyHostToDevice, m->stream));
    std::vector<int> perm(count);
    for (size_t i = 0; i < count; i++) perm[i] = (int)i;
    uint64_t s = c.seed;
    for (int ep = 0; ep < epochs; ep++) {
        // Fisher-Yates with SplitMix64: j = next() mod (i + 1)
        for (size_t i = count - 1; i > 0; i--) {
            const size_t j = (size_t)(splitmix_next(s) % (uint64_t)(i + 1));
            std::swap(perm[i], perm[j]);
        }
        // the copy must finish before perm is shuffled again
        SV_CUDA(cudaMemcpyAsync(m->idx, perm.data(), count * sizeof(int), cudaMemcpyHostToDevice,
                                m->stream));
        SV_CUDA(cudaMemsetAsync(m->loss, 0, sizeof(double), m->stream));
        for (long long first = 0; first < (long long)count; first += batch) {
            const long long nb = std::min<long long>(batch, (long long)count - first);
            SV_TRY(grad_step(m, m->idx + first, nb, lr, b1, b2, eps, nullptr,
                             (double)nb / (double)count));
        }
        double l = 0.0;
        SV_CUDA(cudaMemcpyAsync(&l, m->loss, sizeof(double), cudaMemcpyDeviceToHost, m->stream));
        SV_CUDA(cudaStreamSynchronize(m->stream));
        if (host_epoch_loss) host_epoch_loss[ep] = (float)l;
        if (!std::isfinite(l)) return fail(SV_ERR_STATE, "cost model: training diverged at epoch %d", ep);
    }
    return SV_OK;
}

sv_status sv_cost_model_save(sv_cost_model m, const char *path) {
    clear_error();
    if (!m || !path) return fail(SV_ERR_ARG, "NULL argument");
    std::vector<float> p(NP);
    SV_TRY(sv_cost_model_get_params(m, p.data()));
    FILE *f = fopen(path, "wb");
    if (!f) return fail(SV_ERR_ARG, "cannot open %s for writing", path);
    const int32_t hdr[4] = {1, NF, HD, NP};
    bool ok = fwrite("SVCM", 1, 4, f) == 4 && fwrite(hdr, sizeof hdr, 1, f) == 1 &&
              fwrite(p.data(), sizeof(float), NP, f) == (size_t)NP;
    ok = (fclose(f) == 0) && ok;
    if (!ok) return fail(SV_ERR_ARG, "cannot write %s", path);
    return SV_OK;
}

sv_status sv_cost_model_load(const char *path, sv_cost_model *out) {
    clear_error();
    if (!path || !out) return fail(SV_ERR_ARG, "NULL argument");
    *out = nullptr;
    FILE *f = fopen(path, "rb");
    if (!f) return fail(SV_ERR_ARG, "cannot open %s", path);
    char magic[4];
    int32_t hdr[4];
    std::vector<float> p(NP);
    bool ok = fread(magic, 1, 4, f) == 4 && std::memcmp(magic, "SVCM", 4) == 0 &&
              fread(hdr, sizeof hdr, 1, f) == 1 && hdr[0] == 1 && hdr[1] == NF && hdr[2] == HD &&
              hdr[3] == NP && fread(p.data(), sizeof(float), NP, f) == (size_t)NP;
    fclose(f);
    if (!ok) return fail(SV_ERR_ARG, "%s is not a cost model of this layout", path);
    sv_cost_model m = nullptr;
    SV_TRY(sv_cost_model_create(0, &m));
    sv_status st = sv_cost_model_set_params(m, p.data());
    if (st != SV_OK) {
        sv_cost_model_destroy(m);
        return st;
    }
    *out = m;
    return SV_OK;
}

}  // extern "C"
