// Remap pass: exchange pairs of physical bit positions of the whole state.
//
// Sec. III-B brings a global target qubit into the block by a SWAP with a
// local qubit and then updates the logical-to-physical map; this kernel is
// that state permutation.  For disjoint pairs (a_i, b_i) the amplitude at
// index x moves to P(x), x with bits a_i and b_i exchanged for every i.  P is
// an involution, so the pass runs in place: the thread that owns x with
// P(x) > x swaps the two amplitudes.  Amplitudes are moved as raw bytes, so
// the permutation is exact.  Only indices with some pair of unequal bits move:
// the pass reads and writes (1 - 2^-pairs) of the state once.
//
// Amplitudes are handled in groups of 2^vb consecutive indices (up to 32
// bytes) when the vb lowest bits belong to no pair; a group then moves as
// one unit with 16-byte vector accesses.
#include <algorithm>
#include <cmath>
#include <utility>

#include "common.h"

namespace sv {
namespace {

constexpr int kRemapThreads = 256;
constexpr int kMaxPairs = 32;

struct RemapPairs {
    int np;
    uint64_t mask[kMaxPairs];  // (1 << a_i) | (1 << b_i)
};

template <int GB>
struct Group;
template <>
struct Group<8> {
    uint2 v;
    __device__ void load(const char *p) { v = __ldcs(reinterpret_cast<const uint2 *>(p)); }
    __device__ void store(char *p) const { __stcs(reinterpret_cast<uint2 *>(p), v); }
};
template <>
struct Group<16> {
    uint4 v;
    __device__ void load(const char *p) { v = __ldcs(reinterpret_cast<const uint4 *>(p)); }
    __device__ void store(char *p) const { __stcs(reinterpret_cast<uint4 *>(p), v); }
};
template <>
struct Group<32> {
    uint4 v0, v1;
    __device__ void load(const char *p) {
        v0 = __ldcs(reinterpret_cast<const uint4 *>(p));
        v1 = __ldcs(reinterpret_cast<const uint4 *>(p) + 1);
    }
    __device__ void store(char *p) const {
        __stcs(reinterpret_cast<uint4 *>(p), v0);
        __stcs(reinterpret_cast<uint4 *>(p) + 1, v1);
    }
};

template <int GB>
__device__ __forceinline__ void swap_groups(char *s, uint64_t gx, uint64_t gy) {
    Group<GB> a, b;
    a.load(s + gx * GB);
    b.load(s + gy * GB);
    b.store(s + gx * GB);
    a.store(s + gy * GB);
}

__device__ __forceinline__ uint64_t insert_zero(uint64_t x, int p) {
    const uint64_t low = x & ((UINT64_C(1) << p) - 1);
    return ((x >> p) << (p + 1)) | low;
}

// One pair (lo < hi): every work item is a group whose index has bit lo set
// and bit hi clear; its partner has them the other way round.  Group indices
// count in units of 2^vb amplitudes, so the bit positions arrive shifted.
template <int GB>
__global__ void __launch_bounds__(kRemapThreads)
k_remap_one(char *s, uint64_t items, int lo, int hi) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    const uint64_t d = (UINT64_C(1) << hi) - (UINT64_C(1) << lo);
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < items; i += stride) {
        const uint64_t gx = insert_zero(insert_zero(i, lo), hi) | (UINT64_C(1) << lo);
        swap_groups<GB>(s, gx, gx + d);
    }
}

// Several disjoint pairs: one thread per group, the smaller index of each
// exchanged pair does the move.
template <int GB>
__global__ void __launch_bounds__(kRemapThreads)
k_remap_many(char *s, uint64_t groups, RemapPairs p) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t gx = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; gx < groups; gx += stride) {
        uint64_t gy = gx;
        for (int j = 0; j < p.np; j++) {
            const uint64_t t = gx & p.mask[j];
            if (t != 0 && t != p.mask[j]) gy ^= p.mask[j];
        }
        if (gy > gx) swap_groups<GB>(s, gx, gy);
    }
}

unsigned grid_for(const sv_state *h, uint64_t work) {
    const uint64_t want = (work + kRemapThreads - 1) / kRemapThreads;
    const uint64_t cap = (uint64_t)std::max(1, h->sm_count) * 8;
    return (unsigned)std::max<uint64_t>(1, std::min(want, cap));
}

template <int GB>
void launch(sv_state *h, int np, const int *lo, const int *hi, int vb) {
    char *s = reinterpret_cast<char *>(h->amps);
    const uint64_t groups = UINT64_C(1) << (h->n - vb);
    if (np == 1) {
        const uint64_t items = groups >> 2;
        k_remap_one<GB><<<grid_for(h, items), kRemapThreads, 0, h->stream>>>(s, items, lo[0] - vb,
                                                                             hi[0] - vb);
    } else {
        RemapPairs p{};
        p.np = np;
        for (int j = 0; j < np; j++)
            p.mask[j] = (UINT64_C(1) << (lo[j] - vb)) | (UINT64_C(1) << (hi[j] - vb));
        k_remap_many<GB><<<grid_for(h, groups), kRemapThreads, 0, h->stream>>>(s, groups, p);
    }
}

}  // namespace

sv_status remap_apply(sv_state *h, const std::vector<std::pair<int, int>> &pairs) {
    SV_TRY(materialize(h));
    SV_TRY(launch_check());
    int lo[kMaxPairs], hi[kMaxPairs];
    int np = 0;
    uint64_t used = 0;
    for (const auto &pr : pairs) {
        const int a = std::min(pr.first, pr.second), b = std::max(pr.first, pr.second);
        if (a == b) continue;
        if (a < 0 || b >= h->n) return fail(SV_ERR_ARG, "internal: remap bit outside the state");
        const uint64_t m = (UINT64_C(1) << a) | (UINT64_C(1) << b);
        if (used & m) return fail(SV_ERR_ARG, "internal: remap pairs are not disjoint");
        used |= m;
        lo[np] = a;
        hi[np] = b;
        np++;
    }
    if (np == 0) return SV_OK;
    int low = 64;
    for (int j = 0; j < np; j++) low = std::min(low, lo[j]);
    const bool dbl = h->dt == SV_C128;
    const int vb_max = dbl ? 1 : 2;  // groups of at most 32 bytes
    const int vb = std::min(low, vb_max);
    const int gb = (int)h->amp_bytes << vb;

    sv_launch_record meta = describe_remap(h->n, h->dt, pairs);
    meta.pass = h->launch_index++;
    const int slot = prof_begin(h);
    switch (gb) {
        case 8: launch<8>(h, np, lo, hi, vb); break;
        case 16: launch<16>(h, np, lo, hi, vb); break;
        case 32: launch<32>(h, np, lo, hi, vb); break;
        default: return fail(SV_ERR_ARG, "internal: remap group of %d bytes", gb);
    }
    SV_CUDA(cudaGetLastError());
    note_launch();
    prof_end(h, slot, meta);
    h->stats.kernels++;
    h->stats.remaps++;
    h->stats.passes++;
    h->stats.touched_bytes += meta.bytes;
    return SV_OK;
}

// Physically reorder the state so that logical qubit q sits at bit q.  The
// bit permutation (physical phys[q] -> q) is split, cycle by cycle, into two
// reflections, each a set of disjoint pairs: at most two remap passes.
sv_status remap_to_identity(sv_state *h) {
    const int n = h->n;
    int dest[64];  // physical bit p moves to dest[p]
    for (int q = 0; q < n; q++) dest[h->phys[q]] = q;
    std::vector<std::pair<int, int>> r1, r2;
    bool seen[64] = {};
    for (int s = 0; s < n; s++) {
        if (seen[s]) continue;
        std::vector<int> cyc;  // c_0 = s, c_{i+1} = dest[c_i]
        for (int p = s; !seen[p]; p = dest[p]) {
            seen[p] = true;
            cyc.push_back(p);
        }
        const int m = (int)cyc.size();
        if (m < 2) continue;
        // dest = r2 o r1 with r1: c_i -> c_{-i}, r2: c_i -> c_{1-i}
        for (int i = 1; i < m - i; i++) r1.push_back({cyc[i], cyc[m - i]});
        for (int i = 0; i < m; i++) {
            const int j = ((1 - i) % m + m) % m;
            if (i < j) r2.push_back({cyc[i], cyc[j]});
        }
    }
    // a read-out step: the counters keep describing the last circuit
    const sv_stats keep = h->stats;
    sv_status st = remap_apply(h, r1);
    if (st == SV_OK) st = remap_apply(h, r2);
    h->stats = keep;
    if (st != SV_OK) return st;
    for (int q = 0; q < 64; q++) h->phys[q] = q;
    return SV_OK;
}

}  // namespace sv
