// Internal declarations shared by the translation units of libsv.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <map>
#include <memory>
#include <string>
#include <utility>
#include <vector>

#include "plan.h"
#include "sv.h"

namespace sv {
struct CompiledPlan;  // a planned, compiled and uploaded gate list (tile.cu)
}

namespace sv {

// ---- errors ---------------------------------------------------------------
sv_status fail(sv_status code, const char *fmt, ...);
void clear_error();

#define SV_CUDA(call)                                                          \
    do {                                                                       \
        cudaError_t e_ = (call);                                               \
        if (e_ != cudaSuccess)                                                 \
            return ::sv::fail(SV_ERR_CUDA, "%s failed: %s (%s:%d)", #call,     \
                              cudaGetErrorString(e_), __FILE__, __LINE__);     \
    } while (0)

#define SV_TRY(expr)                                                           \
    do {                                                                       \
        sv_status s_ = (expr);                                                 \
        if (s_ != SV_OK) return s_;                                            \
    } while (0)

// ---- gate matrices (host, FP64) --------------------------------------------
struct Mat2 {
    double re[4], im[4];  // row-major: U11, U12, U21, U22
};

bool is_diagonal_kind(int kind);
bool is_controlled_kind(int kind);
// Validate one gate for an n-qubit state; empty string when valid.
std::string check_gate(int n, const sv_gate &g);
// 2x2 matrix of a non-SWAP gate (controls excluded: the matrix on the target).
Mat2 gate_matrix(const sv_gate &g);
// Phase of a diagonal gate on |1> (or |11>) as a fraction of a full turn in
// units of 2^-64, exact for the dyadic kinds.  `exact` tells whether the
// value is exact (dyadic kinds, CZ) or rounded (P/CP in radians).
uint64_t diag_turns64(const sv_gate &g, bool *exact);

// ---- handle ---------------------------------------------------------------
}  // namespace sv

struct sv_state {
    int n = 0;
    sv_dtype dt = SV_C64;
    size_t amp_bytes = 8;
    void *amps = nullptr;
    bool owned = false;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int device = 0;
    int sm_count = 0;
    int l2_bytes = 0;
    int phys[64];                 // physical bit of each logical qubit
    // >= 0: the state is H on the physical qubits of basis_h applied to the
    // basis state |basis> (physical index), recorded only: the buffer may
    // still hold old data; -1: the buffer holds the state
    int64_t basis = -1;
    uint64_t basis_h = 0;
    void *scratch = nullptr;      // device scratch, grown on demand
    size_t scratch_cap = 0;
    double *probs = nullptr;      // device marginal of the last read-out
    size_t probs_cap = 0;
    void *small = nullptr;        // 64 KiB device area for reduction partials
    void *grp = nullptr;          // L2 block groups: done counters and claim queue
    size_t grp_cap = 0;
    void *slotv = nullptr;        // per-tile slot values of the register-stage passes
    size_t slotv_cap = 0;
    uint8_t *meas_dev = nullptr;  // outcomes of the last call's measurements
    size_t meas_cap = 0;
    size_t nmeas = 0;
    void *plan_host = nullptr;    // pinned host staging for programme uploads
    size_t plan_host_cap = 0;
    // compiled programmes of the last few distinct (gate list, configuration,
    // qubit map) keys, most recent first, each with its own device copy
    std::vector<std::shared_ptr<sv::CompiledPlan>> plan_cache;
    void *plan_dev = nullptr;     // device programme of a call that bypasses the cache
    size_t plan_cap = 0;
    sv_stats stats{};
    void *t2_tables = nullptr;    // FP64-generated phase tables (register-stage kernel)
    int *t2_err = nullptr;        // device flag: a bounded wait gave up
    int *flag_host = nullptr;     // pinned host copy of t2_err, read by finish_sync
    void *t3_tables = nullptr;    // FP64-generated 8-bit phase tables (fused kernel)
    void *tab64 = nullptr;        // FP64 phase tables of the complex128 tile kernel (12 MiB)
    double *norm_buf = nullptr;   // per-CTA squared norms of fused passes (2 x 256)
    bool norm_pending = false;    // the state still needs the last fused pass's norm correction
    int norm_idx = 0, norm_cnt = 0;
    // timing recorder
    bool profiling = false;
    struct Pending {
        sv_launch_record rec;
        cudaEvent_t e0, e1;
    };
    std::vector<Pending> pending;
    std::vector<cudaEvent_t> event_pool;
    int launch_index = 0;  // within the current sv_apply_circuit
    // learned planner
    sv_cost_model_s *cost_model = nullptr;  // attached, not owned
    struct Learned {
        sv::PlanOverride ov;
        std::vector<int8_t> rule_kernel;  // the greedy rule's kernel per pass of ov's plan
        sv_plan_choice info{};
        int verdict = -1;  // planner sv_planner_judge kept; -1 = not judged
    };
    std::map<uint64_t, Learned> learned;  // by circuit structure and start layout
};

namespace sv {

sv_status ensure_scratch(sv_state *h, size_t bytes);
sv_status ensure_probs(sv_state *h, size_t bytes);
const char *last_error_cstr();
inline uint64_t state_bytes(const sv_state *h) { return ((uint64_t)1 << h->n) * h->amp_bytes; }

// ---- timing recorder (prof.cpp) ---------------------------------------------
void note_launch(int count = 1);

// Host-side fault injection (sv_fault_inject): the sites a test can make
// fail, and the check each site makes before it acts.
enum FaultSite { kFaultAlloc = 0, kFaultUpload = 1, kFaultLaunch = 2, kFaultSites = 3 };
bool fault_fire(int site);
void g_fault_set(int site, int after);
// cudaMalloc, or cudaErrorMemoryAllocation when an injected fault fires.
template <typename T>
cudaError_t dev_malloc(T **p, size_t bytes) {
    if (fault_fire(kFaultAlloc)) return cudaErrorMemoryAllocation;
    return cudaMalloc(reinterpret_cast<void **>(p), bytes);
}
// The launch-site check: SV_ERR_CUDA, before the launch, when a fault fires.
sv_status launch_check();
// End of a call that returns data to the host: synchronise the stream and
// report (and clear) the handle's device error word, which a bounded device
// wait sets when it gives up, as SV_ERR_TIMEOUT.
sv_status finish_sync(sv_state *h);
// Record the start event of a launch; returns a record slot or -1.
int prof_begin(sv_state *h);
// Record the end event and the launch's description.
void prof_end(sv_state *h, int slot, const sv_launch_record &meta);

// ---- per-gate path (pergate.cu) ---------------------------------------------
// Apply one gate whose qubits are already PHYSICAL positions.
sv_status pergate_apply(sv_state *h, const sv_gate &g_phys);
// Set the state to |0...0> (recorded only; see sv_state::basis).
sv_status init_zero_state(sv_state *h);
// Write a recorded basis state into the buffer (no-op when it holds the state).
sv_status materialize(sv_state *h);
// The general gate set (general.cu): SV_MCU, SV_U2Q (with its three SV_MAT
// rows) and SV_MEASURE, run by their own per-gate kernels with physical qubit
// positions; `g` points at the gate's first record.
bool is_general_kind(int kind);
int general_records(int kind);
sv_status general_apply(sv_state *h, const sv_gate *g);
sv_status ensure_meas(sv_state *h, size_t count);
// Whole-list validation: every gate (check_gate), a U2Q followed by exactly
// three MAT rows, no MAT elsewhere; "" or the reason with the gate index.
std::string check_list(int n, const sv_gate *g, size_t m);
// Drop the X and H gates that only change a recorded basis state (see api.cu).
void fold_basis_prefix(sv_state *h, std::vector<sv_gate> &gates);

// ---- remap passes (remap.cu) --------------------------------------------------
// Exchange the disjoint physical bit pairs of the whole state, in place.
sv_status remap_apply(sv_state *h, const std::vector<std::pair<int, int>> &pairs);
// Move every logical qubit q to physical bit q (at most two remap passes).
sv_status remap_to_identity(sv_state *h);

// ---- cost model (costmodel.cu) -------------------------------------------------
void cost_features(const sv_launch_record &rec, float *out);
sv_status cost_predict(sv_cost_model_s *m, const float *host_x, size_t count, float *host_y);

// ---- read-out (measure.cu) ----------------------------------------------------
// Order of a marginal held in physical order: bit k of an entry's position
// is output bit bit[k] (m = 0: the entries are in output order).
struct OutPerm {
    int m;
    int8_t bit[34];
};

// Marginal over physical positions pos[0..m-1] (output bit j <-> pos[j]),
// renormalised, into device buffer dev_out (2^m doubles), on h->stream.
// normalise = false leaves the sums unnormalised and returns the block sums
// whose ordered total is the normaliser (sums_out / nsums_out may be NULL).
// With perm_out given, the entries stay in physical order (coalesced stores
// whatever the qubit map) and *perm_out says how to read them.
sv_status marginal_device(sv_state *h, const int *pos, int m, double *dev_out,
                          bool normalise = true, const double **sums_out = nullptr,
                          int *nsums_out = nullptr, OutPerm *perm_out = nullptr);
// Lowest output index of the maximum of dev_p (entries ordered as `perm`
// says); with sums given, dev_p is unnormalised and *host_p is max / total.
sv_status argmax_device(sv_state *h, const double *dev_p, uint64_t len,
                        uint64_t *host_idx, double *host_p, const double *sums = nullptr,
                        int nsums = 0, const OutPerm *perm = nullptr);
sv_status sample_device(sv_state *h, const double *dev_p, uint64_t len,
                        const double *host_u, size_t shots, uint64_t *host_out);

// ---- partitioned path (planner.cpp, tile.cu, tile2.cu) -------------------------
struct T2Pass;
struct T2Device;
struct T2Args;
struct GroupArgs;
size_t t2_smem_bytes();
// Gate kinds (X, real, general 2x2) a register-stage programme uses: picks the
// kernel instantiation.
int t2_gate_kinds(const T2Pass &p);
sv_status t2_prepare(sv_state *h);
// gen_basis >= 0: the state is that basis state and the pass generates it
// instead of reading the buffer.
sv_status t2_launch(sv_state *h, const T2Pass &p, const T2Device &d, const sv_launch_record &meta,
                    int64_t gen_basis = -1);
// The generated-state fields of a first pass that starts from the product
// state H^{basis_h}|gen_basis> (physical qubit masks).
void t2_set_gen(const T2Pass &p, int64_t gen_basis, uint64_t basis_h, T2Args *a);
// The complex128 register-stage kernel (tile2d.cu): a pass compiled by
// compile_t2v2_c128; gen_basis as for t2_launch.  Needs h->tab64.
sv_status t2d_launch(sv_state *h, const T2Pass &p, const T2Device &d, const sv_launch_record &meta,
                     int64_t gen_basis = -1);
// One launch running the passes of an L2 block group (complex64, 2^13 tiles);
// `need`: the gate kinds (t2_gate_kinds) of all its passes.
sv_status t2_group_launch(sv_state *h, const GroupArgs &g, int need, const sv_launch_record &meta);
sv_status t3_prepare(sv_state *h);
sv_status t3_launch(sv_state *h, const T2Pass &p, const T2Device &d, const sv_launch_record &meta);
// Multiply the state by the pending norm correction of the last fused pass.
sv_status resolve_norm(sv_state *h);
struct BatchArgs;
sv_status t2_build_tables(void **tables, int **err, cudaStream_t stream);
sv_status t2_batch_launch(float *states, const BatchArgs &b, int sm_count, cudaStream_t stream);
// SV_ERR_TIMEOUT if a kernel of this handle reported a bounded wait that gave up.
sv_status check_device_flag(sv_state *h);
sv_status partitioned_apply(sv_state *h, const std::vector<sv_gate> &gates_logical,
                            const sv_config &cfg, const PlanOverride *ov = nullptr);
// Learned planner (learned.cpp): the cached decision for this gate list,
// configuration and the handle's current qubit map (computed on first use).
sv_status learned_entry(sv_state *h, const std::vector<sv_gate> &gates, const sv_config &cfg,
                        sv_state::Learned **out);
// Launch descriptors (the cost model's input) of a tile pass on kernel
// family PK_* (t2 = its compiled programme, may be NULL for the generic
// kernel) and of a remap pass.
sv_launch_record describe_pass(int n, sv_dtype dt, const TilePass &p, const T2Pass *t2, int family);
sv_launch_record describe_remap(int n, sv_dtype dt, const std::vector<std::pair<int, int>> &pairs);

}  // namespace sv
