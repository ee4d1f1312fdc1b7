// C ABI entry points (include/sv.h): handle lifetime, validation, dispatch.
#include <algorithm>
#include <cstring>
#include <new>

#include "common.h"

using namespace sv;

namespace {

constexpr int kMaxQubits = 34;

sv_status make_handle(int n, sv_dtype dt, void *buf, size_t bytes, void *stream, bool own,
                      sv_handle *out) {
    clear_error();
    if (!out) return fail(SV_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (n < 1 || n > kMaxQubits) return fail(SV_ERR_ARG, "n=%d outside 1..%d", n, kMaxQubits);
    if (dt != SV_C64 && dt != SV_C128) return fail(SV_ERR_ARG, "unknown dtype %d", (int)dt);
    const size_t need = ((size_t)1 << n) * (dt == SV_C128 ? 16 : 8);
    if (!own) {
        if (!buf) return fail(SV_ERR_ARG, "dev_buf is NULL");
        if (bytes < need) return fail(SV_ERR_ARG, "buffer of %zu bytes < %zu needed", bytes, need);
        if ((uintptr_t)buf % 256) return fail(SV_ERR_ARG, "dev_buf not 256-byte aligned");
    }
    sv_state *h = new (std::nothrow) sv_state();
    if (!h) return fail(SV_ERR_OOM, "host allocation failed");
    h->n = n;
    h->dt = dt;
    h->amp_bytes = dt == SV_C128 ? 16 : 8;
    for (int q = 0; q < 64; q++) h->phys[q] = q;
    auto bail = [&](sv_status st) {
        if (h->owned && h->amps) cudaFree(h->amps);
        if (h->small) cudaFree(h->small);
        if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
        delete h;
        return st;
    };
    if (cudaGetDevice(&h->device) != cudaSuccess ||
        cudaDeviceGetAttribute(&h->sm_count, cudaDevAttrMultiProcessorCount, h->device) !=
            cudaSuccess ||
        cudaDeviceGetAttribute(&h->l2_bytes, cudaDevAttrL2CacheSize, h->device) != cudaSuccess) {
        cudaError_t e = cudaGetLastError();
        return bail(fail(SV_ERR_CUDA, "no usable CUDA device: %s", cudaGetErrorString(e)));
    }
    if (own) {
        if (cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            return bail(fail(SV_ERR_CUDA, "cudaStreamCreate failed"));
        }
        h->own_stream = true;
        if (dev_malloc(&h->amps, need) != cudaSuccess) {
            cudaGetLastError();
            return bail(fail(SV_ERR_OOM, "cannot allocate %zu bytes for the state", need));
        }
        h->owned = true;
    } else {
        h->amps = buf;
        h->stream = reinterpret_cast<cudaStream_t>(stream);
    }
    if (dev_malloc(&h->small, 65536) != cudaSuccess) {
        cudaGetLastError();
        return bail(fail(SV_ERR_OOM, "cannot allocate reduction buffer"));
    }
    sv_status st = init_zero_state(h);
    if (st != SV_OK) return bail(st);
    *out = h;
    return SV_OK;
}

int popcount64(uint64_t x) { return __builtin_popcountll(x); }

sv_status check_mask(sv_state *h, uint64_t mask) {
    if (!mask) return fail(SV_ERR_ARG, "qubit_mask is empty");
    if (h->n < 64 && (mask >> h->n)) return fail(SV_ERR_ARG, "qubit_mask has bits beyond n=%d", h->n);
    if (popcount64(mask) > 30) return fail(SV_ERR_ARG, "qubit_mask selects more than 30 qubits");
    return SV_OK;
}

// physical positions of the mask's logical qubits, in increasing logical order
int mask_positions(const sv_state *h, uint64_t mask, int *pos) {
    int m = 0;
    for (int q = 0; q < h->n; q++)
        if ((mask >> q) & 1) pos[m++] = h->phys[q];
    return m;
}

sv_status read_marginal(sv_state *h, uint64_t mask, uint64_t *len) {
    int pos[64];
    int m = mask_positions(h, mask, pos);
    *len = UINT64_C(1) << m;
    SV_TRY(ensure_probs(h, *len * sizeof(double)));
    return marginal_device(h, pos, m, h->probs);
}

}  // namespace

// While the state is a recorded product state H^{hq}|b> (H on the qubits of
// the mask hq, applied to the basis state |b>), a gate whose qubit no earlier
// gate of the list touches commutes to the front of the list.  An X on a
// qubit outside hq only flips a bit of b; an H toggles the qubit in hq (H H
// is the identity).  Drop such gates and update the record.  An X on a qubit
// in hq would add a sign that depends on b; it is kept, and so is every
// later gate on its qubit.
void sv::fold_basis_prefix(sv_state *h, std::vector<sv_gate> &g) {
    if (h->basis < 0) return;
    bool touched[64] = {};
    std::vector<sv_gate> out;
    out.reserve(g.size());
    for (const sv_gate &a : g) {
        const uint64_t bit = UINT64_C(1) << h->phys[a.target];
        if (!touched[a.target] && a.kind == SV_X && !(h->basis_h & bit)) {
            h->basis ^= (int64_t)bit;
            continue;
        }
        if (!touched[a.target] && a.kind == SV_H) {
            h->basis_h ^= bit;
            continue;
        }
        touched[a.target] = true;
        if (is_controlled_kind(a.kind) || a.kind == SV_SWAP || a.kind == SV_U2Q || a.kind == SV_MAT)
            touched[a.control] = true;
        if (a.kind == SV_MCU)
            for (int q = 0; q < 64; q++)
                if (((uint64_t)a.num >> q) & 1) touched[q] = true;
        out.push_back(a);
    }
    g.swap(out);
}

extern "C" {

sv_status sv_create(int n, sv_dtype dt, sv_handle *out) {
    return make_handle(n, dt, nullptr, 0, nullptr, true, out);
}

sv_status sv_create_on(int n, sv_dtype dt, void *dev_buf, size_t bytes, void *cuda_stream,
                       sv_handle *out) {
    return make_handle(n, dt, dev_buf, bytes, cuda_stream, false, out);
}

sv_status sv_destroy(sv_handle h) {
    clear_error();
    if (!h) return SV_OK;
    if (h->stream) cudaStreamSynchronize(h->stream);
    if (h->owned && h->amps) cudaFree(h->amps);
    if (h->scratch) cudaFree(h->scratch);
    if (h->probs) cudaFree(h->probs);
    if (h->small) cudaFree(h->small);
    if (h->grp) cudaFree(h->grp);
    if (h->slotv) cudaFree(h->slotv);
    h->plan_cache.clear();  // frees each entry's device copy
    if (h->plan_dev) cudaFree(h->plan_dev);
    if (h->plan_host) cudaFreeHost(h->plan_host);
    if (h->flag_host) cudaFreeHost(h->flag_host);
    if (h->t2_tables) cudaFree(h->t2_tables);
    if (h->t3_tables) cudaFree(h->t3_tables);
    if (h->tab64) cudaFree(h->tab64);
    if (h->norm_buf) cudaFree(h->norm_buf);
    for (auto &p : h->pending) {
        cudaEventDestroy(p.e0);
        cudaEventDestroy(p.e1);
    }
    for (cudaEvent_t e : h->event_pool) cudaEventDestroy(e);
    if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
    delete h;
    return SV_OK;
}

sv_status sv_reset(sv_handle h) {
    clear_error();
    if (!h) return fail(SV_ERR_ARG, "handle is NULL");
    h->norm_pending = false;
    return init_zero_state(h);
}

sv_status sv_info(sv_handle h, int *n, sv_dtype *dt, void **dev_amps) {
    clear_error();
    if (!h) return fail(SV_ERR_ARG, "handle is NULL");
    if (n) *n = h->n;
    if (dt) *dt = h->dt;
    if (dev_amps) {  // the caller may read the buffer: it must hold the state
        SV_TRY(materialize(h));
        *dev_amps = h->amps;
    }
    return SV_OK;
}

sv_status sv_qubit_map(sv_handle h, int *host_phys_of_logical) {
    clear_error();
    if (!h || !host_phys_of_logical) return fail(SV_ERR_ARG, "NULL argument");
    for (int q = 0; q < h->n; q++) host_phys_of_logical[q] = h->phys[q];
    return SV_OK;
}

sv_status sv_apply_circuit(sv_handle h, const sv_gate *host_gates, size_t m, const sv_config *cfg) {
    clear_error();
    if (!h) return fail(SV_ERR_ARG, "handle is NULL");
    if (m && !host_gates) return fail(SV_ERR_ARG, "gate list is NULL");
    sv_config c{};
    if (cfg) c = *cfg;
    for (int i = 0; i < 7; i++)
        if (c.reserved[i]) return fail(SV_ERR_ARG, "sv_config.reserved must be 0");
    if (c.l2_qubits != 0 && (c.l2_qubits < 14 || c.l2_qubits > 30))
        return fail(SV_ERR_ARG, "l2_qubits must be 0 or 14..30");
    if (c.l2_chunk < 0 || c.l2_chunk > 16 || (c.l2_chunk & (c.l2_chunk - 1)))
        return fail(SV_ERR_ARG, "l2_chunk must be 0 or a power of two up to 16");
    if (c.mode < SV_MODE_AUTO || c.mode > SV_MODE_FUSED)
        return fail(SV_ERR_ARG, "unknown mode %d", c.mode);
    if (c.planner < SV_PLANNER_GREEDY || c.planner > SV_PLANNER_LEARNED)
        return fail(SV_ERR_ARG, "unknown planner %d", c.planner);
    if (c.tile_qubits < 0 || c.tile_qubits > 14 || c.chunk_qubits < 0 || c.chunk_qubits > 14)
        return fail(SV_ERR_ARG, "tile_qubits / chunk_qubits outside 0..14");
    if (c.fuse_qubits != 0 && c.fuse_qubits != 5)
        return fail(SV_ERR_ARG, "fuse_qubits must be 0 or 5");
    {
        const std::string why = check_list(h->n, host_gates, m);
        if (!why.empty()) return fail(SV_ERR_ARG, "%s", why.c_str());
    }
    h->stats = sv_stats{};
    h->stats.gates = (int32_t)m;
    h->launch_index = 0;
    h->nmeas = 0;
    int mode = c.mode;
    if (mode == SV_MODE_AUTO) mode = h->n >= 16 ? SV_MODE_PARTITIONED : SV_MODE_PERGATE;
    sv_status st = SV_OK;
    if (mode == SV_MODE_PERGATE) {
        st = resolve_norm(h);
        for (size_t i = 0; i < m && st == SV_OK; i++) {
            if (is_general_kind(host_gates[i].kind)) {  // the general gate set, physical qubits
                const int nr = general_records(host_gates[i].kind);
                sv_gate g4[4];
                for (int r = 0; r < nr; r++) {
                    g4[r] = host_gates[i + r];
                    g4[r].target = h->phys[g4[r].target];
                    if (g4[r].control >= 0) g4[r].control = h->phys[g4[r].control];
                }
                if (g4[0].kind == SV_MCU) {
                    uint64_t pm = 0;
                    for (int q = 0; q < h->n; q++)
                        if (((uint64_t)g4[0].num >> q) & 1) pm |= UINT64_C(1) << h->phys[q];
                    g4[0].num = (int64_t)pm;
                }
                st = general_apply(h, g4);
                i += nr - 1;
                continue;
            }
            sv_gate g = host_gates[i];
            g.target = h->phys[g.target];
            if (is_controlled_kind(g.kind) || g.kind == SV_SWAP) g.control = h->phys[g.control];
            st = pergate_apply(h, g);
        }
    } else {
        std::vector<sv_gate> gl(host_gates, host_gates + m);
        const int64_t basis0 = h->basis;
        const uint64_t basis_h0 = h->basis_h;
        fold_basis_prefix(h, gl);
        c.mode = mode;
        sv_state::Learned *L = nullptr;
        if (c.planner == SV_PLANNER_LEARNED && h->cost_model) {
            sv_config key_cfg = c;
            key_cfg.planner = SV_PLANNER_GREEDY;
            st = learned_entry(h, gl, key_cfg, &L);
        }
        if (st == SV_OK && L && L->verdict != SV_PLANNER_GREEDY) {
            st = partitioned_apply(h, gl, c, &L->ov);
            h->stats.planner = SV_PLANNER_LEARNED;
            h->stats.predicted_ms = L->info.predicted_ms;
            h->stats.candidates = L->info.candidates;
        } else if (st == SV_OK) {
            st = partitioned_apply(h, gl, c);
        }
        // a call that fails before any kernel wrote the state leaves it as it
        // was, the recorded state included (materialising it changes nothing)
        if (st != SV_OK && h->stats.kernels == 0 && basis0 >= 0) {
            h->basis = basis0;
            h->basis_h = basis_h0;
        }
    }
    // per-gate: full-sweep convention (2 x passes x state); partitioned: the
    // bytes each pass moves (a pass that generates the initial state only writes)
    h->stats.sweep_bytes = mode == SV_MODE_PERGATE ? 2.0 * h->stats.passes * (double)state_bytes(h)
                                                   : h->stats.touched_bytes;
    return st;
}

sv_status sv_last_stats(sv_handle h, sv_stats *out) {
    clear_error();
    if (!h || !out) return fail(SV_ERR_ARG, "NULL argument");
    *out = h->stats;
    return SV_OK;
}

sv_status sv_probabilities(sv_handle h, uint64_t qubit_mask, double *host_out) {
    clear_error();
    if (!h || !host_out) return fail(SV_ERR_ARG, "NULL argument");
    SV_TRY(check_mask(h, qubit_mask));
    uint64_t len;
    SV_TRY(read_marginal(h, qubit_mask, &len));
    SV_CUDA(cudaMemcpyAsync(host_out, h->probs, len * sizeof(double), cudaMemcpyDeviceToHost,
                            h->stream));
    return finish_sync(h);
}

sv_status sv_probabilities_device(sv_handle h, uint64_t qubit_mask, double *dev_out) {
    clear_error();
    if (!h || !dev_out) return fail(SV_ERR_ARG, "NULL argument");
    SV_TRY(check_mask(h, qubit_mask));
    int pos[64];
    int m = mask_positions(h, qubit_mask, pos);
    return marginal_device(h, pos, m, dev_out);
}

sv_status sv_argmax(sv_handle h, uint64_t qubit_mask, uint64_t *host_idx, double *host_p) {
    clear_error();
    if (!h || !host_idx) return fail(SV_ERR_ARG, "NULL argument");
    SV_TRY(check_mask(h, qubit_mask));
    // the argmax does not need the normalised vector: only max / total
    int pos[64];
    const int m = mask_positions(h, qubit_mask, pos);
    const uint64_t len = UINT64_C(1) << m;
    SV_TRY(ensure_probs(h, len * sizeof(double)));
    const double *sums = nullptr;
    int nsums = 0;
    // the marginal stays in physical order (coalesced stores whatever the qubit map)
    OutPerm perm{};
    SV_TRY(marginal_device(h, pos, m, h->probs, false, &sums, &nsums, &perm));
    return argmax_device(h, h->probs, len, host_idx, host_p, sums, nsums, &perm);
}

sv_status sv_sample(sv_handle h, uint64_t qubit_mask, const double *host_u, size_t shots,
                    uint64_t *host_out) {
    clear_error();
    if (!h || (shots && (!host_u || !host_out))) return fail(SV_ERR_ARG, "NULL argument");
    SV_TRY(check_mask(h, qubit_mask));
    for (size_t s = 0; s < shots; s++)
        if (!(host_u[s] >= 0.0 && host_u[s] < 1.0))
            return fail(SV_ERR_ARG, "u[%zu] = %g is not in [0, 1)", s, host_u[s]);
    uint64_t len;
    SV_TRY(read_marginal(h, qubit_mask, &len));
    return sample_device(h, h->probs, len, host_u, shots, host_out);
}

sv_status sv_copy_out(sv_handle h, void *host_amps) {
    clear_error();
    if (!h || !host_amps) return fail(SV_ERR_ARG, "NULL argument");
    SV_TRY(materialize(h));
    SV_TRY(resolve_norm(h));
    SV_TRY(remap_to_identity(h));
    SV_CUDA(cudaMemcpyAsync(host_amps, h->amps, state_bytes(h), cudaMemcpyDeviceToHost, h->stream));
    return finish_sync(h);
}

sv_status sv_copy_in(sv_handle h, const void *host_amps) {
    clear_error();
    if (!h || !host_amps) return fail(SV_ERR_ARG, "NULL argument");
    SV_CUDA(cudaMemcpyAsync(h->amps, host_amps, state_bytes(h), cudaMemcpyHostToDevice, h->stream));
    SV_CUDA(cudaStreamSynchronize(h->stream));
    for (int q = 0; q < 64; q++) h->phys[q] = q;
    h->norm_pending = false;
    h->basis = -1;
    h->basis_h = 0;
    return SV_OK;
}

sv_status sv_last_measurements(sv_handle h, uint8_t *host_out, size_t cap, size_t *count) {
    clear_error();
    if (!h || !count || (cap && !host_out)) return fail(SV_ERR_ARG, "NULL argument");
    *count = h->nmeas;
    const size_t k = std::min(cap, h->nmeas);
    if (k) SV_CUDA(cudaMemcpyAsync(host_out, h->meas_dev, k, cudaMemcpyDeviceToHost, h->stream));
    return finish_sync(h);
}

sv_status sv_fault_inject(int site, int after) {
    clear_error();
    if (site < 0 || site >= kFaultSites) return fail(SV_ERR_ARG, "unknown fault site %d", site);
    g_fault_set(site, after);
    return SV_OK;
}

sv_status sv_fault_raise_device_flag(sv_handle h) {
    clear_error();
    if (!h) return fail(SV_ERR_ARG, "handle is NULL");
    SV_TRY(t2_prepare(h));  // the error word lives with the register-stage tables
    SV_CUDA(cudaMemsetAsync(h->t2_err, 0xff, sizeof(int), h->stream));
    return SV_OK;
}

const char *sv_last_error(void) { return last_error_cstr(); }

const char *sv_version(void) { return "libsv 0.1 (sm_103a)"; }

}  // extern "C"
