// Timing recorder: CUDA events around every kernel launch of
// sv_apply_circuit, and a process-wide launch counter.  The records feed the
// benchmark's roofline figure and the learned cost model's training set.
#include <atomic>

#include "common.h"

namespace sv {

static std::atomic<uint64_t> g_launches{0};

void note_launch(int count) { g_launches.fetch_add(count, std::memory_order_relaxed); }

namespace {
// Countdown per fault site: the call that takes it from 0 to -1 fails; < 0: off.
std::atomic<int> g_fault[kFaultSites] = {{-1}, {-1}, {-1}};
}  // namespace

void g_fault_set(int site, int after) { g_fault[site].store(after < 0 ? -1 : after); }

bool fault_fire(int site) {
    int v = g_fault[site].load(std::memory_order_relaxed);
    while (v >= 0)
        if (g_fault[site].compare_exchange_weak(v, v - 1, std::memory_order_relaxed)) return v == 0;
    return false;
}

sv_status launch_check() {
    if (fault_fire(kFaultLaunch)) return fail(SV_ERR_CUDA, "kernel launch failed (injected fault)");
    return SV_OK;
}

sv_status finish_sync(sv_state *h) {
    if (h->t2_err && h->flag_host)
        SV_CUDA(cudaMemcpyAsync(h->flag_host, h->t2_err, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    SV_CUDA(cudaStreamSynchronize(h->stream));
    if (h->t2_err && h->flag_host && *h->flag_host) {
        *h->flag_host = 0;
        SV_CUDA(cudaMemsetAsync(h->t2_err, 0, sizeof(int), h->stream));
        SV_CUDA(cudaStreamSynchronize(h->stream));
        return fail(SV_ERR_TIMEOUT, "a tile kernel gave up waiting (bounded device wait); the state is undefined");
    }
    return SV_OK;
}

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
