// Timing recorder: CUDA events around every kernel launch of
// sv_apply_circuit, and a process-wide launch counter.  The records feed the
// benchmark's roofline figure and the learned cost model's training set.
#include <atomic>

#include "common.h"

namespace sv {

static std::atomic<uint64_t> g_launches{0};

void note_launch(int count) { g_launches.fetch_add(count, std::memory_order_relaxed); }

static constexpr size_t kMaxPending = (size_t)1 << 20;

static cudaEvent_t take_event(sv_state *h) {
    if (!h->event_pool.empty()) {
        cudaEvent_t e = h->event_pool.back();
        h->event_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return e;
}

int prof_begin(sv_state *h) {
    if (!h->profiling || h->pending.size() >= kMaxPending) return -1;
    sv_state::Pending p{};
    p.e0 = take_event(h);
    p.e1 = take_event(h);
    if (!p.e0 || !p.e1) return -1;
    cudaEventRecord(p.e0, h->stream);
    h->pending.push_back(p);
    return (int)h->pending.size() - 1;
}

void prof_end(sv_state *h, int slot, const sv_launch_record &meta) {
    if (slot < 0) return;
    sv_state::Pending &p = h->pending[slot];
    cudaEventRecord(p.e1, h->stream);
    p.rec = meta;
}

}  // namespace sv

using namespace sv;

extern "C" {

sv_status sv_profile(sv_handle h, int enable) {
    clear_error();
    if (!h) return fail(SV_ERR_ARG, "handle is NULL");
    if (enable) {
        SV_CUDA(cudaStreamSynchronize(h->stream));
        for (auto &p : h->pending) {
            h->event_pool.push_back(p.e0);
            h->event_pool.push_back(p.e1);
        }
        h->pending.clear();
    }
    h->profiling = enable != 0;
    return SV_OK;
}

sv_status sv_profile_read(sv_handle h, sv_launch_record *host_out, size_t cap, size_t *count) {
    clear_error();
    if (!h || !count || (cap && !host_out)) return fail(SV_ERR_ARG, "NULL argument");
    SV_CUDA(cudaStreamSynchronize(h->stream));
    *count = h->pending.size();
    size_t take = cap < h->pending.size() ? cap : h->pending.size();
    for (size_t i = 0; i < take; i++) {
        sv_state::Pending &p = h->pending[i];
        float ms = 0.f;
        SV_CUDA(cudaEventElapsedTime(&ms, p.e0, p.e1));
        host_out[i] = p.rec;
        host_out[i].ms = ms;
        h->event_pool.push_back(p.e0);
        h->event_pool.push_back(p.e1);
    }
    h->pending.erase(h->pending.begin(), h->pending.begin() + take);
    return SV_OK;
}

uint64_t sv_launch_count(void) { return g_launches.load(); }

}  // extern "C"
