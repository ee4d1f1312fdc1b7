// Grouping of register-stage passes into L2 blocks (see l2group.h).
#include "l2group.h"

#include <algorithm>

namespace sv {

int l2_default_qubits(size_t l2_bytes, size_t amp_bytes) {
    int l = 0;
    while (l < 40 && ((size_t)1 << (l + 1)) * amp_bytes <= l2_bytes / 8) l++;
    return l;
}

int lag_for(int npass, int tiles_per_block, int grid, int chunk) {
    const long long per_step = (long long)npass * tiles_per_block;
    const long long want = (5LL * grid * chunk) / 2 + 1;
    return (int)std::max<long long>(1, (want + per_step - 1) / per_step);
}

std::string form_l2_groups(const Plan &plan, const std::vector<char> &eligible, int n, int k,
                           int l_cap, int grid, int chunk, std::vector<L2Group> *out) {
    out->clear();
    if (l_cap < k + 1 || l_cap > 40) return "block qubits outside k+1..40";
    if (grid < 1) return "grid must be positive";
    if (chunk < 1 || (chunk & (chunk - 1))) return "tiles per claim must be a power of two";
    const int P = (int)plan.passes.size();
    if ((int)eligible.size() != P) return "eligibility vector does not match the plan";
    const int l = std::min(l_cap, n);
    auto tile_mask = [&](int i) {
        uint64_t m = 0;
        for (int s = 0; s < plan.passes[i].k; s++) m |= UINT64_C(1) << plan.passes[i].slot_phys[s];
        return m;
    };
    for (int i = 0; i < P;) {
        if (!eligible[i] || plan.passes[i].k != k) {
            i++;
            continue;
        }
        uint64_t U = tile_mask(i);
        int j = i + 1;
        while (j < P && j - i < kMaxGroupPasses && eligible[j] && plan.passes[j].k == k &&
               plan.passes[j].remap_before.empty() && plan.passes[j].general.empty()) {
            const uint64_t U2 = U | tile_mask(j);
            if (__builtin_popcountll(U2) > l) break;
            U = U2;
            j++;
        }
        if (j - i >= 2) {
            L2Group g;
            g.first = i;
            g.count = j - i;
            g.l = l;
            g.bmask = U;
            for (int q = 0; q < n && __builtin_popcountll(g.bmask) < l; q++)
                g.bmask |= UINT64_C(1) << q;
            const uint64_t nblocks = UINT64_C(1) << (n - l);
            if (nblocks > (UINT64_C(1) << 20)) {  // the claim-order table would be too large
                i = j;
                continue;
            }
            const int tpb = 1 << (l - k);
            while ((1 << g.chunk_log) < std::min(chunk, tpb)) g.chunk_log++;
            g.lag = lag_for(g.count, tpb, grid, 1 << g.chunk_log);
            const uint64_t steps = nblocks + (uint64_t)(g.count - 1) * g.lag;
            g.segs.reserve(nblocks * g.count);
            for (uint64_t s = 0; s < steps; s++)
                for (int p = 0; p < g.count; p++) {
                    const long long b = (long long)s - (long long)p * g.lag;
                    if (b >= 0 && (uint64_t)b < nblocks) g.segs.push_back(((uint32_t)b << 3) | (uint32_t)p);
                }
            out->push_back(std::move(g));
        }
        i = j;
    }
    return "";
}

}  // namespace sv
