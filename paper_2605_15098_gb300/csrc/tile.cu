// Partitioned execution: tile kernels and the pass driver.
//
// One launch per pass.  A persistent grid walks the 2^(n-k) tiles of the
// pass; each CTA gathers its tile (2^(k-c) chunks of 2^c contiguous
// amplitudes) into shared memory, applies the pass's whole programme there
// (the deferred block-by-block execution of Sec. III-B, arxiv 2605.15098),
// and writes the tile back.  Out-of-tile bits are constants of the tile, so
// a control on a global qubit is a per-tile branch and every diagonal run
// reduces to a per-tile phase polynomial over the local bits.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <type_traits>

#include "common.h"
#include "plan.h"
#include "stagecomp.h"

namespace sv {
namespace {

constexpr int kTileThreads = 256;

struct PassArgs {
    int k, c, nops;
    int slot_phys[kMaxTileQubits];
    uint64_t gmask;
    uint64_t ntiles;
    const TileOp *ops;
    const PhaseTerm *terms;
    const double2 *tab64;  // complex128: phase tables (see k_phase_tables64)
    double hscale;         // complex128: 2^(-h/2) for the pass's h unnormalised Hadamards
};

// complex128 phases: e^{2 pi i phi / 2^64} = T0[phi >> 46] T1[(phi >> 28) & m] T2[(phi >> 10) & m]
// with T0[j] = e^{2 pi i j / 2^18}, T1[j] = e^{2 pi i j / 2^36}, T2[j] = e^{2 pi i j / 2^54}
// (the 10 lowest bits, under 2^-54 of a turn, are dropped), each entry from FP64 sincospi.
constexpr int kTab64Bits = 18;
constexpr int kTab64 = 1 << kTab64Bits;

__device__ __forceinline__ uint64_t pdep64(uint64_t v, uint64_t mask) {
    uint64_t r = 0;
    for (uint64_t b = 1; mask; b <<= 1) {
        const uint64_t low = mask & (~mask + 1);
        if (v & b) r |= low;
        mask &= mask - 1;
    }
    return r;
}

__device__ __forceinline__ uint32_t insert_bit(uint32_t x, int p, uint32_t v) {
    return ((x >> p) << (p + 1)) | (v << p) | (x & ((1u << p) - 1));
}

template <typename R>
struct Cx {
    R re, im;
};

template <typename R>
__device__ __forceinline__ void phase_cs(uint64_t phi, R *c, R *s);

template <>
__device__ __forceinline__ void phase_cs<double>(uint64_t phi, double *c, double *s) {
    // e^{2 pi i phi / 2^64} = cos/sin(pi x) with x = phi / 2^63 in [-1, 1)
    const double x = (double)(int64_t)phi * 0x1p-63;
    sincospi(x, s, c);
}

__device__ __forceinline__ double2 phase_tab64(const double2 *__restrict__ t, uint64_t phi) {
    constexpr uint64_t m = kTab64 - 1;
    const double2 a = __ldg(t + (phi >> 46));
    const double2 b = __ldg(t + kTab64 + ((phi >> 28) & m));
    const double2 c = __ldg(t + 2 * kTab64 + ((phi >> 10) & m));
    const double2 ab = make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
    return make_double2(ab.x * c.x - ab.y * c.y, ab.x * c.y + ab.y * c.x);
}

__global__ void k_phase_tables64(double2 *t) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= 3 * kTab64) return;
    const int lvl = i / kTab64, j = i % kTab64;
    const double x = (double)j * (lvl == 0 ? 0x1p-18 : lvl == 1 ? 0x1p-36 : 0x1p-54);
    double s, c;
    sincospi(2.0 * x, &s, &c);
    t[i] = make_double2(c, s);
}

template <>
__device__ __forceinline__ void phase_cs<float>(uint64_t phi, float *c, float *s) {
    const float x = (float)(int32_t)(uint32_t)(phi >> 32) * 0x1p-31f;
    sincospif(x, s, c);
}

// x / sqrt(2); in single precision 1/sqrt(2) is split into two floats so
// that the product is rounded once (a rounded constant would shrink the norm
// by the same factor at every H).
template <typename R>
__device__ __forceinline__ R hscale(R x) {
    if constexpr (sizeof(R) == 4)
        return fmaf(x, 0.70710677f, x * 1.21016175e-08f);
    else
        return x * 0.70710678118654752440084436210485;
}

// Offset (in amplitudes) of local chunk j of the tile.
__device__ __forceinline__ uint64_t chunk_offset(const PassArgs &a, uint32_t j) {
    uint64_t off = 0;
    for (int b = 0; b < a.k - a.c; b++)
        if ((j >> b) & 1) off |= UINT64_C(1) << a.slot_phys[a.c + b];
    return off;
}

template <typename R>
__global__ void __launch_bounds__(kTileThreads)
k_tile(R *__restrict__ state, const PassArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    R *sm = reinterpret_cast<R *>(smem_raw);
    __shared__ uint64_t lin[kMaxTileQubits];
    __shared__ uint64_t cst;
    using V = typename std::conditional<sizeof(R) == 4, float4, double2>::type;
    constexpr int APV = 16 / (2 * sizeof(R));  // amplitudes per 16-byte vector
    const uint32_t tile_amps = 1u << a.k;
    const uint32_t nvec = tile_amps / APV;
    const uint32_t cmask = (1u << a.c) - 1;
    V *gv = reinterpret_cast<V *>(state);
    V *svec = reinterpret_cast<V *>(sm);

    for (uint64_t tile = blockIdx.x; tile < a.ntiles; tile += gridDim.x) {
        const uint64_t base = pdep64(tile, a.gmask);
        for (uint32_t v = threadIdx.x; v < nvec; v += blockDim.x) {
            const uint32_t i = v * APV;
            const uint64_t g = base + chunk_offset(a, i >> a.c) + (i & cmask);
            svec[v] = gv[g / APV];
        }
        __syncthreads();

        for (int o = 0; o < a.nops; o++) {
            const TileOp &op = a.ops[o];
            const int type = op.type;
            if (type == TOP_DIAG) {
                if ((int)threadIdx.x < a.k) {
                    uint64_t acc = 0;
                    for (int t = op.tb; t < op.te; t++) {
                        const PhaseTerm &pt = a.terms[t];
                        if (pt.a != (int)threadIdx.x) continue;
                        if (pt.kind == TERM_L) acc += pt.theta;
                        if (pt.kind == TERM_LG && ((base >> pt.b) & 1)) acc += pt.theta;
                    }
                    lin[threadIdx.x] = acc;
                } else if ((int)threadIdx.x == a.k) {
                    uint64_t acc = 0;
                    for (int t = op.tb; t < op.te; t++) {
                        const PhaseTerm &pt = a.terms[t];
                        if (pt.kind == TERM_G && ((base >> pt.a) & 1)) acc += pt.theta;
                        if (pt.kind == TERM_GG && ((base >> pt.a) & 1) && ((base >> pt.b) & 1))
                            acc += pt.theta;
                    }
                    cst = acc;
                }
                __syncthreads();
                for (uint32_t i = threadIdx.x; i < tile_amps; i += blockDim.x) {
                    uint64_t phi = cst;
                    for (int b = 0; b < a.k; b++)
                        if ((i >> b) & 1) phi += lin[b];
                    for (int t = op.tb; t < op.te; t++) {
                        const PhaseTerm &pt = a.terms[t];
                        if (pt.kind == TERM_LL && ((i >> pt.a) & 1) && ((i >> pt.b) & 1))
                            phi += pt.theta;
                    }
                    if (phi) {
                        R c, s;
                        if constexpr (sizeof(R) == 8) {
                            const double2 f = phase_tab64(a.tab64, phi);
                            c = f.x;
                            s = f.y;
                        } else {
                            phase_cs<R>(phi, &c, &s);
                        }
                        const R re = sm[2 * i], im = sm[2 * i + 1];
                        sm[2 * i] = re * c - im * s;
                        sm[2 * i + 1] = re * s + im * c;
                    }
                }
            } else if (type == TOP_SWAP) {
                const int sa = op.slot, sb = op.cslot;
                const int lo = sa < sb ? sa : sb, hi = sa < sb ? sb : sa;
                for (uint32_t p = threadIdx.x; p < tile_amps / 4; p += blockDim.x) {
                    uint32_t i = insert_bit(p, lo, lo == sa ? 1u : 0u);
                    i = insert_bit(i, hi, hi == sa ? 1u : 0u);
                    const uint32_t j = i ^ (1u << sa) ^ (1u << sb);
                    const R r0 = sm[2 * i], i0 = sm[2 * i + 1];
                    sm[2 * i] = sm[2 * j];
                    sm[2 * i + 1] = sm[2 * j + 1];
                    sm[2 * j] = r0;
                    sm[2 * j + 1] = i0;
                }
            } else {
                if (type == TOP_GATE_CG && !((base >> op.cbit) & 1)) continue;  // uniform
                const int t = op.slot;
                const bool lctl = type == TOP_GATE_CL;
                const uint32_t npairs = lctl ? tile_amps / 4 : tile_amps / 2;
                const R m0r = (R)op.m[0], m0i = (R)op.m[1], m1r = (R)op.m[2], m1i = (R)op.m[3];
                const R m2r = (R)op.m[4], m2i = (R)op.m[5], m3r = (R)op.m[6], m3i = (R)op.m[7];
                for (uint32_t p = threadIdx.x; p < npairs; p += blockDim.x) {
                    uint32_t i;
                    if (lctl) {
                        const int cs = op.cslot;
                        if (cs < t)
                            i = insert_bit(insert_bit(p, cs, 1u), t, 0u);
                        else
                            i = insert_bit(insert_bit(p, t, 0u), cs, 1u);
                    } else {
                        i = insert_bit(p, t, 0u);
                    }
                    const uint32_t j = i | (1u << t);
                    const R ar = sm[2 * i], ai = sm[2 * i + 1];
                    const R br = sm[2 * j], bi = sm[2 * j + 1];
                    R xr, xi, yr, yi;
                    if (type == TOP_X) {
                        xr = br; xi = bi; yr = ar; yi = ai;
                    } else if (type == TOP_H) {
                        if constexpr (sizeof(R) == 8) {  // unnormalised; scaled once at the end
                            xr = ar + br; xi = ai + bi;
                            yr = ar - br; yi = ai - bi;
                        } else {
                            xr = hscale<R>(ar + br); xi = hscale<R>(ai + bi);
                            yr = hscale<R>(ar - br); yi = hscale<R>(ai - bi);
                        }
                    } else {
                        xr = m0r * ar - m0i * ai + m1r * br - m1i * bi;
                        xi = m0r * ai + m0i * ar + m1r * bi + m1i * br;
                        yr = m2r * ar - m2i * ai + m3r * br - m3i * bi;
                        yi = m2r * ai + m2i * ar + m3r * bi + m3i * br;
                    }
                    sm[2 * i] = xr; sm[2 * i + 1] = xi;
                    sm[2 * j] = yr; sm[2 * j + 1] = yi;
                }
            }
            __syncthreads();
        }

        for (uint32_t v = threadIdx.x; v < nvec; v += blockDim.x) {
            const uint32_t i = v * APV;
            const uint64_t g = base + chunk_offset(a, i >> a.c) + (i & cmask);
            V val = svec[v];
            if constexpr (sizeof(R) == 8) {
                if (a.hscale != 1.0) {
                    val.x *= a.hscale;
                    val.y *= a.hscale;
                }
            }
            gv[g / APV] = val;
        }
        __syncthreads();
    }
}

template <typename R>
sv_status launch_pass(sv_state *h, const PassArgs &a, const sv_launch_record &meta) {
    SV_TRY(launch_check());
    const size_t smem = ((size_t)1 << a.k) * 2 * sizeof(R);
    static bool configured[2] = {false, false};
    auto kern = k_tile<R>;
    const int idx = sizeof(R) == 8;
    if (!configured[idx]) {
        SV_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
        configured[idx] = true;
    }
    int per_sm = 0;
    SV_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kTileThreads, smem));
    if (per_sm < 1) return fail(SV_ERR_UNSUPPORTED, "tile of %zu bytes does not fit on an SM", smem);
    const uint64_t grid = std::min<uint64_t>(a.ntiles, (uint64_t)per_sm * h->sm_count);
    const int slot = prof_begin(h);
    kern<<<(unsigned)grid, kTileThreads, smem, h->stream>>>(reinterpret_cast<R *>(h->amps), a);
    SV_CUDA(cudaGetLastError());
    note_launch();
    prof_end(h, slot, meta);
    h->stats.kernels++;
    return SV_OK;
}

}  // namespace

namespace {

// Host staging of everything a call uploads, 256-byte aligned sections.
struct Blob {
    std::vector<char> b;
    size_t put(const void *p, size_t n) {
        const size_t off = (b.size() + 255) & ~(size_t)255;
        b.resize(off + n);  // zero-filled
        if (n && p) std::memcpy(b.data() + off, p, n);
        return off;
    }
    template <typename T>
    size_t put_vec(const std::vector<T> &v) {
        return put(v.data(), v.size() * sizeof(T));
    }
};

// Blob offsets of one compiled register-stage programme.
struct T2Off {
    size_t ins = 0, stages = 0, mats = 0, fac = 0, stat = 0, statc = 0, slots = 0, tterms = 0;
    size_t soff = 0, sterms = 0;
    size_t layx = 0, epi = 0;
};

T2Off put_t2(Blob &blob, const T2Pass &t) {
    T2Off o;
    o.ins = blob.put_vec(t.ins);
    o.stages = blob.put_vec(t.stages);
    o.layx = blob.put_vec(t.layx);
    o.epi = blob.put(&t.epi, sizeof(T2Epilogue));
    // a complex128 programme's FP64 records take the places of the FP32 ones
    o.mats = t.wide ? blob.put_vec(t.mats64) : blob.put_vec(t.mats);
    o.fac = t.format == 2 ? blob.put_vec(t.fac2) : blob.put_vec(t.factors);
    o.stat = blob.put_vec(t.stat);
    o.statc = t.wide ? blob.put_vec(t.statc64) : blob.put_vec(t.statc);
    o.slots = blob.put_vec(t.slots);
    o.tterms = blob.put_vec(t.tterms);
    o.soff = blob.put_vec(t.soff);
    o.sterms = t.wide ? blob.put_vec(t.sterms64) : blob.put_vec(t.sterms);
    return o;
}

T2Device t2_device(const char *dev, const T2Off &o) {
    T2Device d{};
    d.ins = reinterpret_cast<const T2Ins *>(dev + o.ins);
    d.stages = reinterpret_cast<const T2Stage *>(dev + o.stages);
    d.layx = reinterpret_cast<const T2LayoutX *>(dev + o.layx);
    d.epi = reinterpret_cast<const T2Epilogue *>(dev + o.epi);
    d.mats = reinterpret_cast<const T2Mat *>(dev + o.mats);
    d.fac = dev + o.fac;
    d.stat = reinterpret_cast<const uint32_t *>(dev + o.stat);
    d.statc = reinterpret_cast<const float *>(dev + o.statc);
    d.slots = reinterpret_cast<const T2Slot *>(dev + o.slots);
    d.tterms = reinterpret_cast<const T2TileTerm *>(dev + o.tterms);
    d.soff = reinterpret_cast<const int32_t *>(dev + o.soff);
    d.sterms = reinterpret_cast<const T2SlotTerm *>(dev + o.sterms);
    return d;
}

struct PassUpload {
    bool t2 = false;
    bool t3 = false;
    bool has_gen = false;  // a format-2 variant for a generated basis state
    size_t blocks = 0;
    size_t ops = 0, terms = 0;  // generic kernel
    T2Off main, gen;            // register-stage kernels
};

constexpr size_t kPlanCacheEntries = 8;

// 64-bit FNV-1a
uint64_t fnv1a(const void *p, size_t n, uint64_t h = 0xcbf29ce484222325ull) {
    const unsigned char *b = static_cast<const unsigned char *>(p);
    for (size_t i = 0; i < n; i++) h = (h ^ b[i]) * 0x100000001b3ull;
    return h;
}

}  // namespace

// A gate list planned and compiled for one configuration and starting qubit
// map, with its programme uploaded to its own device buffer.  The key holds
// every input the plan and the programmes depend on.
struct CompiledPlan {
    std::string key;
    uint64_t hash = 0;
    Plan plan;
    std::vector<T2Pass> t2;
    std::vector<PassUpload> up;
    std::vector<L2Group> groups;       // L2 block groups (SV_FLAG_L2_BLOCKS)
    std::vector<size_t> group_segs;    // blob offset of each group's claim order
    std::vector<int> group_at;         // per pass: the group it starts, or -1
    int phys_out[64];
    void *dev = nullptr;
    size_t bytes = 0;
    bool owns_dev = false;  // false: the handle's buffer for uncached calls
    ~CompiledPlan() {
        if (owns_dev && dev) cudaFree(dev);  // synchronises with work that may still read it
    }
};

static sv_status tab64_prepare(sv_state *h) {
    if (h->tab64) return SV_OK;
    void *p = nullptr;
    if (dev_malloc(&p, (size_t)3 * kTab64 * sizeof(double2)) != cudaSuccess) {
        cudaGetLastError();
        return fail(SV_ERR_OOM, "cannot allocate complex128 phase tables");
    }
    h->tab64 = p;
    k_phase_tables64<<<(3 * kTab64 + 255) / 256, 256, 0, h->stream>>>(reinterpret_cast<double2 *>(p));
    SV_CUDA(cudaGetLastError());
    note_launch();
    return SV_OK;
}

sv_status check_device_flag(sv_state *h) {
    if (!h->t2_err) return SV_OK;
    int flag = 0;
    SV_CUDA(cudaMemcpyAsync(&flag, h->t2_err, sizeof flag, cudaMemcpyDeviceToHost, h->stream));
    SV_CUDA(cudaStreamSynchronize(h->stream));
    if (flag) {
        SV_CUDA(cudaMemsetAsync(h->t2_err, 0, sizeof(int), h->stream));
        return fail(SV_ERR_TIMEOUT, "a tile kernel gave up waiting for its bulk copies");
    }
    return SV_OK;
}

sv_launch_record describe_pass(int n, sv_dtype dt, const TilePass &p, const T2Pass *t2, int family) {
    sv_launch_record r{};
    r.kind = family == PK_T3 ? SV_KERNEL_FUSED : SV_KERNEL_TILE;
    r.n = n;
    r.k = p.k;
    r.c = p.c;
    r.nops = (int)p.ops.size();
    r.ngates = p.ngates;
    r.dtype = (int32_t)dt;
    r.gate_kind = family == PK_T3 ? -3 : family == PK_T2 ? -2 : -1;
    r.bytes = 2.0 * (double)(UINT64_C(1) << n) * (dt == SV_C128 ? 16.0 : 8.0);
    r.feat = ~p.gmask & ((UINT64_C(1) << n) - 1);
    if (t2 && family != PK_GENERIC) {
        r.stages = (int)t2->stages.size();
        r.blocks = family == PK_T3 ? t2->nblocks : 0;
        r.nins = (int)t2->ins.size();
        r.nfactors = (int)(t2->format == 2 ? t2->fac2.size() : t2->factors.size());
    }
    return r;
}

sv_launch_record describe_remap(int n, sv_dtype dt, const std::vector<std::pair<int, int>> &pairs) {
    sv_launch_record r{};
    r.kind = SV_KERNEL_REMAP;
    r.n = n;
    r.dtype = (int32_t)dt;
    r.gate_kind = -4;
    r.ngates = (int)pairs.size();
    for (const auto &pr : pairs) r.feat |= (UINT64_C(1) << pr.first) | (UINT64_C(1) << pr.second);
    const double sb = (double)(UINT64_C(1) << n) * (dt == SV_C128 ? 16.0 : 8.0);
    r.bytes = 2.0 * (1.0 - std::ldexp(1.0, -(int)pairs.size())) * sb;
    return r;
}

// The cache key: every input of planning and compilation.
static int l2_cap(const sv_state *h, const sv_config &cfg) {
    if (cfg.l2_qubits) return cfg.l2_qubits;
    return l2_default_qubits(h->l2_bytes > 0 ? (size_t)h->l2_bytes : ((size_t)126 << 20), h->amp_bytes);
}

static std::string plan_key(const sv_state *h, const std::vector<sv_gate> &gates, const sv_config &cfg,
                            const PlanOptions &opt, const PlanOverride *ov) {
    std::string k;
    auto put = [&](const void *p, size_t n) { k.append(static_cast<const char *>(p), n); };
    const int head[] = {h->n, (int)h->dt, cfg.mode, (int)cfg.flags, opt.n, opt.k, opt.c,
                        opt.merge_diag, opt.relabel, opt.paper, opt.split_u3, opt.late_diag,
                        opt.search, ov ? 1 : 0, l2_cap(h, cfg), cfg.l2_chunk, h->sm_count};
    put(head, sizeof head);
    put(h->phys, sizeof h->phys);
    if (ov) {
        const int n = (int)ov->kernel.size();
        put(&n, sizeof n);
        put(ov->kernel.data(), ov->kernel.size());
    }
    put(gates.data(), gates.size() * sizeof(sv_gate));
    return k;
}

// Plan, compile and upload (or find in the handle's cache) the gate list.
static sv_status compiled_plan(sv_state *h, const std::vector<sv_gate> &gates, const sv_config &cfg,
                               const PlanOverride *ov, std::shared_ptr<CompiledPlan> *out) {
    const bool dbl = h->dt == SV_C128;
    PlanOptions opt = ov ? ov->opt : plan_options(h->n, h->dt, cfg);
    if (dbl && opt.k > 13) return fail(SV_ERR_ARG, "complex128 tiles hold at most 2^13 amplitudes");
    std::string key = plan_key(h, gates, cfg, opt, ov);
    const uint64_t hash = fnv1a(key.data(), key.size());
    const bool use_cache = !(cfg.flags & SV_FLAG_NO_PLAN_CACHE);
    for (size_t i = 0; use_cache && i < h->plan_cache.size(); i++) {
        const auto &e = h->plan_cache[i];
        if (e->hash == hash && e->key == key) {
            std::shared_ptr<CompiledPlan> hit = e;
            h->plan_cache.erase(h->plan_cache.begin() + (long)i);
            h->plan_cache.insert(h->plan_cache.begin(), hit);
            *out = hit;
            return SV_OK;
        }
    }
    auto cp = std::make_shared<CompiledPlan>();
    cp->key = std::move(key);
    cp->hash = hash;
    Plan &plan = cp->plan;
    int *phys = cp->phys_out;
    std::copy(h->phys, h->phys + 64, phys);
    std::string err = build_plan(gates, opt, phys, &plan);
    if (!err.empty()) return fail(SV_ERR_ARG, "planner: %s", err.c_str());

    // compile every pass; register-stage kernel where it applies (complex128:
    // the FP64 variant on 2^13-amplitude tiles)
    const bool allow_t2 = !(cfg.flags & SV_FLAG_GENERIC_TILE) && (!dbl || opt.k == kT2Qubits);
    const bool fused = cfg.mode == SV_MODE_FUSED;
    std::vector<T2Pass> &t2 = cp->t2;
    std::vector<PassUpload> &up = cp->up;
    t2.resize(plan.passes.size());
    up.resize(plan.passes.size());
    Blob blob;
    if (ov && ov->kernel.size() != plan.passes.size())
        return fail(SV_ERR_STATE, "internal: learned plan does not match the planner's passes");
    bool first_pass = true;  // the pass that may start from a recorded basis state
    for (size_t i = 0; i < plan.passes.size(); i++) {
        const TilePass &p = plan.passes[i];
        if (!p.general.empty()) first_pass = false;  // the step writes the state first
        if (p.ops.empty()) continue;
        const bool first_ops = first_pass && p.remap_before.empty();
        first_pass = false;
        const int want = ov ? ov->kernel[i] : (!allow_t2 ? PK_GENERIC : fused && !dbl ? PK_T3 : PK_T2);
        bool ok = false;
        if (dbl) {
            if (want != PK_GENERIC && allow_t2 && compile_t2v2_c128(p, &t2[i], false).empty()) {
                ok = true;
                if (first_ops) {
                    auto g = std::make_shared<T2Pass>();
                    if (compile_t2v2_c128(p, g.get(), true).empty()) {
                        t2[i].genv = g;
                        up[i].has_gen = true;
                        up[i].gen = put_t2(blob, *g);
                    }
                }
            }
        } else if (want == PK_T3 && compile_t2(p, &t2[i], true).empty()) {
            ok = true;
            up[i].t3 = true;
            up[i].blocks = blob.put_vec(t2[i].blocks_dev);
        } else if ((want == PK_T3 || want == PK_T2) && compile_t2(p, &t2[i], false).empty()) {
            ok = true;
            if (first_ops) {
                auto g = std::make_shared<T2Pass>();
                if (compile_t2v2(p, g.get(), true).empty()) {
                    t2[i].genv = g;
                    up[i].has_gen = true;
                    up[i].gen = put_t2(blob, *g);
                }
            }
        }
        if (ok) {
            up[i].t2 = true;
            up[i].main = put_t2(blob, t2[i]);
        } else {
            up[i].ops = blob.put_vec(p.ops);
            up[i].terms = blob.put_vec(p.terms);
        }
    }
    cp->group_at.assign(plan.passes.size(), -1);
    if ((cfg.flags & SV_FLAG_L2_BLOCKS) && !dbl) {
        // two-level blocking: consecutive register-stage passes that fit one L2 block
        std::vector<char> eligible(plan.passes.size(), 0);
        for (size_t i = 0; i < plan.passes.size(); i++)
            eligible[i] = up[i].t2 && !up[i].t3 && t2[i].format == 2 && plan.passes[i].k == kT2Qubits &&
                          !plan.passes[i].ops.empty();
        const std::string why =
            form_l2_groups(plan, eligible, h->n, kT2Qubits, l2_cap(h, cfg), 2 * std::max(1, h->sm_count),
                           cfg.l2_chunk ? cfg.l2_chunk : 2, &cp->groups);
        if (!why.empty()) return fail(SV_ERR_ARG, "L2 blocks: %s", why.c_str());
        for (size_t g = 0; g < cp->groups.size(); g++) {
            cp->group_segs.push_back(blob.put_vec(cp->groups[g].segs));
            cp->group_at[cp->groups[g].first] = (int)g;
        }
    }
    blob.put(nullptr, 0);
    const size_t total = blob.b.size();
    if (total > h->plan_host_cap) {
        SV_CUDA(cudaStreamSynchronize(h->stream));
        if (h->plan_host) cudaFreeHost(h->plan_host);
        h->plan_host = nullptr;
        h->plan_host_cap = 0;
        const size_t cap = std::max<size_t>(total * 2, (size_t)1 << 16);
        if (cudaMallocHost(&h->plan_host, cap) != cudaSuccess) {
            cudaGetLastError();
            return fail(SV_ERR_OOM, "cannot allocate the programme staging (%zu bytes)", cap);
        }
        h->plan_host_cap = cap;
    } else {
        // the previous upload must have finished before the staging is reused
        SV_CUDA(cudaStreamSynchronize(h->stream));
    }
    if (use_cache) {
        if (dev_malloc(&cp->dev, total + 256) != cudaSuccess) {
            cudaGetLastError();
            cp->dev = nullptr;
            return fail(SV_ERR_OOM, "cannot allocate the pass programme (%zu bytes)", total);
        }
        cp->owns_dev = true;
    } else {  // one buffer per handle, reused (the stream was synchronised above)
        if (total + 256 > h->plan_cap) {
            if (h->plan_dev) cudaFree(h->plan_dev);
            h->plan_dev = nullptr;
            h->plan_cap = 0;
            const size_t cap = std::max<size_t>(2 * (total + 256), (size_t)1 << 16);
            if (dev_malloc(&h->plan_dev, cap) != cudaSuccess) {
                cudaGetLastError();
                h->plan_dev = nullptr;
                return fail(SV_ERR_OOM, "cannot allocate the pass programme (%zu bytes)", cap);
            }
            h->plan_cap = cap;
        }
        cp->dev = h->plan_dev;
    }
    cp->bytes = total;
    if (fault_fire(kFaultUpload)) return fail(SV_ERR_CUDA, "programme upload failed (injected fault)");
    std::memcpy(h->plan_host, blob.b.data(), total);
    SV_CUDA(cudaMemcpyAsync(cp->dev, h->plan_host, total, cudaMemcpyHostToDevice, h->stream));
    h->stats.h2d_bytes += (double)total;
    if (use_cache) {
        h->plan_cache.insert(h->plan_cache.begin(), cp);
        if (h->plan_cache.size() > kPlanCacheEntries) h->plan_cache.pop_back();
    }
    *out = cp;
    return SV_OK;
}

// Run L2 block group gi of the plan (its first pass's remap already done).
static sv_status group_apply(sv_state *h, const CompiledPlan &cp, int gi) {
    const L2Group &g = cp.groups[gi];
    const char *dev = reinterpret_cast<const char *>(cp.dev);
    SV_TRY(resolve_norm(h));
    // a recorded basis state: generated by the first pass, or written out first
    int64_t gen = -1;
    if (h->basis >= 0) {
        if (cp.up[g.first].has_gen)
            gen = h->basis;
        else
            SV_TRY(materialize(h));
    }
    GroupArgs ga{};
    int need = 0, ngates = 0, nins = 0, nfac = 0, nstages = 0;
    uint64_t feat = 0;
    for (int j = 0; j < g.count; j++) {
        const int i = g.first + j;
        const bool gj = j == 0 && gen >= 0;
        const T2Pass &tp = gj ? *cp.t2[i].genv : cp.t2[i];
        T2Args &a = ga.pass[j];
        t2_fill_args(tp, t2_device(dev, gj ? cp.up[i].gen : cp.up[i].main), h->n, &a);
        if (!t2_block_runs(&a, tp.gmask, g.bmask, h->n))
            return fail(SV_ERR_STATE, "internal: tile index runs of an L2 block do not fit");
        if (gj) t2_set_gen(tp, gen, h->basis_h, &a);
        a.tables = reinterpret_cast<const float2 *>(h->t2_tables);
        a.err = h->t2_err;
        a.keep = j + 1 < g.count;
        need |= t2_gate_kinds(tp);
        ngates += cp.plan.passes[i].ngates;
        nins += (int)tp.ins.size();
        nfac += (int)tp.fac2.size();
        nstages += (int)tp.stages.size();
        feat |= ~cp.plan.passes[i].gmask;
    }
    const uint64_t nblocks = UINT64_C(1) << (h->n - g.l);
    const size_t ncnt = (size_t)nblocks * g.count;
    const size_t need_bytes = 256 + ncnt * sizeof(unsigned);
    if (need_bytes > h->grp_cap) {
        if (h->grp) {
            SV_CUDA(cudaStreamSynchronize(h->stream));
            cudaFree(h->grp);
        }
        h->grp = nullptr;
        h->grp_cap = 0;
        const size_t cap = std::max<size_t>(2 * need_bytes, (size_t)1 << 16);
        if (dev_malloc(&h->grp, cap) != cudaSuccess) {
            cudaGetLastError();
            h->grp = nullptr;
            return fail(SV_ERR_OOM, "cannot allocate the L2 block counters (%zu bytes)", cap);
        }
        h->grp_cap = cap;
    }
    SV_CUDA(cudaMemsetAsync(h->grp, 0, need_bytes, h->stream));
    ga.queue = reinterpret_cast<unsigned long long *>(h->grp);
    ga.done = reinterpret_cast<unsigned *>(reinterpret_cast<char *>(h->grp) + 256);
    ga.segs = reinterpret_cast<const uint32_t *>(dev + cp.group_segs[gi]);
    ga.npass = g.count;
    ga.tpb_log = g.l - kT2Qubits;
    ga.chunk_log = g.chunk_log;
    ga.nitems = (uint64_t)g.segs.size() << ga.tpb_log;
    ga.err = h->t2_err;

    sv_launch_record meta{};
    meta.kind = SV_KERNEL_L2BLOCK;
    meta.pass = h->launch_index++;
    meta.n = h->n;
    meta.k = g.l;
    meta.c = cp.plan.passes[g.first].c;
    meta.nops = g.count;
    meta.ngates = ngates;
    meta.dtype = (int32_t)h->dt;
    meta.gate_kind = -5;
    // HBM: the group's first read (none for a generated state) and last write
    meta.bytes = (gen >= 0 ? 1.0 : 2.0) * (double)state_bytes(h);
    meta.feat = feat & ((h->n >= 64) ? ~UINT64_C(0) : ((UINT64_C(1) << h->n) - 1));
    meta.stages = nstages;
    meta.nins = nins;
    meta.nfactors = nfac;
    SV_TRY(t2_group_launch(h, ga, need, meta));
    if (gen >= 0) {
        h->basis = -1;
        h->basis_h = 0;
    }
    h->stats.passes += g.count;
    h->stats.touched_bytes += meta.bytes;
    return SV_OK;
}

sv_status partitioned_apply(sv_state *h, const std::vector<sv_gate> &gates, const sv_config &cfg,
                            const PlanOverride *ov) {
    const bool dbl = h->dt == SV_C128;
    std::shared_ptr<CompiledPlan> cp;
    SV_TRY(compiled_plan(h, gates, cfg, ov, &cp));
    const Plan &plan = cp->plan;
    const std::vector<T2Pass> &t2 = cp->t2;
    const std::vector<PassUpload> &up = cp->up;
    const char *dev = reinterpret_cast<const char *>(cp->dev);
    bool any_t2 = false, any_t3 = false;
    for (auto &u : up) {
        any_t2 |= u.t2;
        any_t3 |= u.t3;
    }
    if (any_t2) SV_TRY(t2_prepare(h));
    if (any_t2 && dbl) SV_TRY(tab64_prepare(h));
    if (any_t2 && !dbl) {  // the per-tile slot values of the one-level register-stage passes
        size_t need = 0;
        for (size_t i = 0; i < up.size(); i++) {
            if (!up[i].t2 || up[i].t3 || cp->group_at[i] >= 0) continue;
            need = std::max(need, t2_slotv_bytes(t2[i], h->n));
            if (t2[i].genv) need = std::max(need, t2_slotv_bytes(*t2[i].genv, h->n));
        }
        if (need > h->slotv_cap) {
            if (h->slotv) {
                SV_CUDA(cudaStreamSynchronize(h->stream));
                cudaFree(h->slotv);
            }
            h->slotv = nullptr;
            h->slotv_cap = 0;
            if (dev_malloc(&h->slotv, need) != cudaSuccess) {
                cudaGetLastError();
                h->slotv = nullptr;
                return fail(SV_ERR_OOM, "cannot allocate the per-tile slot values (%zu bytes)", need);
            }
            h->slotv_cap = need;
        }
    }
    if (any_t3) SV_TRY(t3_prepare(h));

    for (size_t i = 0; i < plan.passes.size(); i++) {
        const TilePass &p = plan.passes[i];
        if (!p.general.empty()) {  // a gate of the general set, on the per-gate path
            SV_TRY(general_apply(h, p.general.data()));
            continue;
        }
        if (!p.remap_before.empty()) SV_TRY(remap_apply(h, p.remap_before));
        if (p.ops.empty()) continue;
        if (cp->group_at[i] >= 0) {  // an L2 block group: its passes in one launch
            const int gi = cp->group_at[i];
            SV_TRY(group_apply(h, *cp, gi));
            i += (size_t)cp->groups[gi].count - 1;
            continue;
        }
        sv_launch_record meta = describe_pass(h->n, h->dt, p, up[i].t2 ? &t2[i] : nullptr,
                                              up[i].t3 ? PK_T3 : up[i].t2 ? PK_T2 : PK_GENERIC);
        meta.pass = h->launch_index++;
        sv_status st;
        if (!up[i].t3) SV_TRY(resolve_norm(h));
        // a recorded basis state: the register-stage kernel generates it in
        // its first pass; every other kernel needs it written out first
        int64_t gen = -1;
        if (h->basis >= 0) {
            if (up[i].t2 && !up[i].t3 && up[i].has_gen) {
                gen = h->basis;
                meta.bytes = (double)state_bytes(h);  // written, not read
                meta.generated = 1;
            } else {
                SV_TRY(materialize(h));
            }
        }
        if (up[i].t2) {
            const bool g = gen >= 0;
            T2Device d = t2_device(dev, g ? up[i].gen : up[i].main);
            d.blocks = up[i].t3 ? reinterpret_cast<const float *>(dev + up[i].blocks) : nullptr;
            st = up[i].t3 ? t3_launch(h, t2[i], d, meta)
                 : dbl    ? t2d_launch(h, g ? *t2[i].genv : t2[i], d, meta, gen)
                          : t2_launch(h, g ? *t2[i].genv : t2[i], d, meta, gen);
            if (st == SV_OK && gen >= 0) {
                h->basis = -1;
                h->basis_h = 0;
            }
        } else {
            PassArgs a{};
            a.k = p.k;
            a.c = p.c;
            a.nops = (int)p.ops.size();
            for (int s = 0; s < p.k; s++) a.slot_phys[s] = p.slot_phys[s];
            a.gmask = p.gmask;
            a.ntiles = UINT64_C(1) << (h->n - p.k);
            a.ops = reinterpret_cast<const TileOp *>(dev + up[i].ops);
            a.terms = reinterpret_cast<const PhaseTerm *>(dev + up[i].terms);
            a.hscale = 1.0;
            if (dbl) {
                int nh = 0;
                for (const TileOp &op : p.ops) nh += op.type == TOP_H;
                a.hscale = std::pow(2.0, -0.5 * nh);
                SV_TRY(tab64_prepare(h));
                a.tab64 = reinterpret_cast<const double2 *>(h->tab64);
            }
            st = dbl ? launch_pass<double>(h, a, meta) : launch_pass<float>(h, a, meta);
        }
        if (st != SV_OK) return st;
        h->stats.passes++;
        h->stats.touched_bytes += meta.bytes;
    }
    std::copy(cp->phys_out, cp->phys_out + 64, h->phys);
    h->stats.relabels = plan.relabels;
    return SV_OK;
}

}  // namespace sv
