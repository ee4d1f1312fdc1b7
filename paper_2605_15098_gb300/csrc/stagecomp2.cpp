// Stage compiler, format 2: tile pass (plan.h) -> register-stage programme
// of the complex64 CUDA-core kernels (k_tile2, k_batch; tileprog.h).
//
// Every gate target is a register bit of its stage.  A stage covers the
// longest run of steps whose targets fit four register bits besides tile
// bit 0 (which is always register bit 0): the register bits of a new stage
// are the next four distinct targets, so no shorter segmentation exists.
// Gates therefore never exchange amplitudes between threads; a stage change
// moves the tile through shared memory in a swizzled order (tileprog.h).
// Lane bits 0..2 take tile bits whose float4 bits differ mod 3 (conflict-free
// under the swizzle), preferring tile bits 1..3, which the first stage of a
// pass that reads its tile (the bulk copies' linear order) and the last stage
// (coalesced write-back) need; a pass whose last stage cannot have them gets
// one more stage change before the write-back.
//
// Diagonal runs (Sec. III-B's rule that global qubits are constants of a
// block, applied to every diagonal gate) compile against the layout of the
// stage that executes them:
//   * phases constant across threads (register-bit terms, and constants
//     predicated on one thread bit) become 32-entry tables over the register
//     index, each entry formed in FP64 from its summed 32-bit phase;
//   * what depends on the thread's own bits becomes a static complex row,
//     one FP32 value per thread formed in FP64 here;
//   * what depends on the tile (terms with a global qubit) becomes a slot,
//     evaluated once per tile by the kernel from its integer phase words.
// A run that is the identity where bit j is 0, directly followed by a
// Hadamard on register bit j (an inverse-QFT step), becomes one phased
// butterfly (T2_HPH).
#include <cmath>
#include <cstring>
#include <map>
#include <string>
#include <tuple>
#include <vector>

#include "common.h"
#include "plan.h"
#include "stagecomp.h"

namespace sv {
namespace {

struct Lay {
    int k = kT2Qubits, nw = kT2WarpBits;
    int reg[kT2RegBits];
    int lane[5];
    int warp[4];
    int cls[kT2MaxQubits];
    int pos[kT2MaxQubits];  // register bit, or thread bit (lane l -> l, warp w -> 5 + w)

    void index() {
        for (int j = 0; j < kT2RegBits; j++) {
            cls[reg[j]] = T2C_REG;
            pos[reg[j]] = j;
        }
        for (int l = 0; l < 5; l++) {
            cls[lane[l]] = T2C_THREAD;
            pos[lane[l]] = l;
        }
        for (int w = 0; w < nw; w++) {
            cls[warp[w]] = T2C_THREAD;
            pos[warp[w]] = 5 + w;
        }
    }
    int tbits() const { return 5 + nw; }
    int ttb(int t) const { return t < 5 ? lane[t] : warp[t - 5]; }
    bool canonical() const { return lane[0] == 1 && lane[1] == 2 && lane[2] == 3; }
};

bool is_gate(int type) {
    return type == TOP_GATE || type == TOP_GATE_CL || type == TOP_GATE_CG || type == TOP_H ||
           type == TOP_X;
}

// Layout with register bits 0, r[0..3]; lane bits 0..2 conflict-free under
// the swizzle (tile bits 1..3 when `canon`, which the caller keeps free).
Lay make_layout(int k, const int r[4], bool canon) {
    Lay L;
    L.k = k;
    L.nw = k - kT2RegBits - 5;
    bool used[kT2MaxQubits] = {};
    L.reg[0] = 0;
    used[0] = true;
    for (int j = 0; j < 4; j++) {
        L.reg[1 + j] = r[j];
        used[r[j]] = true;
    }
    for (int l = 0; l < 3; l++) {
        int pick = -1;
        if (canon) {
            pick = 1 + l;
        } else {
            for (int tb = 1 + l; tb < k && pick < 0; tb += 3)
                if (!used[tb]) pick = tb;
            for (int tb = 1; tb < k && pick < 0; tb++)  // no bit of this residue is free
                if (!used[tb]) pick = tb;
        }
        L.lane[l] = pick;
        used[pick] = true;
    }
    int nl = 3, nwp = 0;
    for (int tb = 1; tb < k; tb++) {
        if (used[tb]) continue;
        if (nl < 5)
            L.lane[nl++] = tb;
        else
            L.warp[nwp++] = tb;
        used[tb] = true;
    }
    L.index();
    return L;
}

// The next register bits from step `from`: the first four distinct targets
// (tile bit 0 aside); with `no123` the segment stops at a target among tile
// bits 1..3 (the first stage of a pass that reads its tile).  Padded with
// tile bits that keep 1..3 free, highest first.
void pick_regs(const TilePass &tp, size_t from, bool no123, int out[4]) {
    int n = 0;
    for (size_t i = from; i < tp.ops.size() && n < 4; i++) {
        const TileOp &op = tp.ops[i];
        if (!is_gate(op.type)) continue;
        const int t = op.slot;
        if (t == 0) continue;
        bool seen = false;
        for (int j = 0; j < n; j++) seen |= out[j] == t;
        if (seen) continue;
        if (no123 && t <= 3) break;
        out[n++] = t;
    }
    for (int tb = tp.k - 1; tb >= 4 && n < 4; tb--) {
        bool seen = false;
        for (int j = 0; j < n; j++) seen |= out[j] == tb;
        if (!seen) out[n++] = tb;
    }
}

uint32_t turns32(uint64_t t64) { return (uint32_t)((t64 + (UINT64_C(1) << 31)) >> 32); }

// cos and sin of 2 pi u / 2^32, evaluated in FP64 and rounded to FP32.  A
// pass's static rows repeat the same phases across threads and rows, so a
// small direct-mapped memo per host thread hands back values it has already
// evaluated; a value is the same whichever way it is obtained.
void expi(uint32_t u, float *re, float *im) {
    struct Memo {
        uint32_t u;
        bool ok;
        float re, im;
    };
    static thread_local Memo memo[4096];
    Memo &e = memo[(u * 2654435761u) >> 20];
    if (!e.ok || e.u != u) {
        const double ang = 2.0 * M_PI * ((double)(int32_t)u * 0x1p-32);
        e.u = u;
        e.ok = true;
        e.re = (float)std::cos(ang);
        e.im = (float)std::sin(ang);
    }
    *re = e.re;
    *im = e.im;
}

// Precision policies of the compiler.  P32 (complex64 kernels): phases as
// 32-bit fractions of a turn, values rounded to FP32 (T2Pass::mats, statc,
// sterms).  P64 (complex128 kernel): phases as the planner's 64-bit
// fractions, values in FP64 (T2Pass::mats64, statc64, sterms64).  The
// programme structure (instructions, stages, factor records, slots) is the
// same for both.
struct P32 {
    using Ph = uint32_t;
    using V = float;
    static Ph ph(uint64_t t64) { return turns32(t64); }
    static void ex(Ph u, V *re, V *im) { expi(u, re, im); }
    static bool real(const double *m) {
        return (float)m[1] == 0.f && (float)m[3] == 0.f && (float)m[5] == 0.f && (float)m[7] == 0.f;
    }
    static int32_t push_mat(T2Pass *o, const double *m) {
        T2Mat t{};
        for (int e = 0; e < 8; e++) t.m[e] = (float)m[e];
        o->mats.push_back(t);
        return (int32_t)o->mats.size() - 1;
    }
    static size_t nmats(const T2Pass *o) { return o->mats.size(); }
    static size_t nrowvals(const T2Pass *o) { return o->statc.size(); }
    static void push_row(T2Pass *o, V re, V im) {
        o->statc.push_back(re);
        o->statc.push_back(im);
    }
    // 32-entry table: T[q] = (re[2q], re[2q+1], im[2q], im[2q+1]), eight records
    static int32_t push_table(T2Pass *o, const Ph *u) {
        const int32_t m0 = (int32_t)o->mats.size();
        float tab[64];
        for (int x = 0; x < 32; x++) {
            float re, im;
            expi(u[x], &re, &im);
            tab[4 * (x >> 1) + (x & 1)] = re;
            tab[4 * (x >> 1) + 2 + (x & 1)] = im;
        }
        for (int m = 0; m < 8; m++) {
            T2Mat tm{};
            for (int e = 0; e < 8; e++) tm.m[e] = tab[8 * m + e];
            o->mats.push_back(tm);
        }
        return m0;
    }
    static bool table_one(const T2Pass *o, int m0, int x) {
        const float *tf = o->mats[m0 + (x >> 2)].m;
        const int off = 4 * ((x >> 1) & 1) + (x & 1);
        return tf[off] == 1.f && tf[off + 2] == 0.f;
    }
    // the packed entries q1 of a phased butterfly on register bit j (q1 over
    // register bits 1..4, bit j - 1 of q1 set) depend only on register bits
    // below j: every entry equals the one with the same low j - 1 bits
    static constexpr bool kSharedTwiddles = true;
    static constexpr int kSharedMinJ = 1, kSharedMaxJ = 3;  // bit 0 is the packed element
    static bool table_low_only(const T2Pass *o, int m0, int j) {
        auto entry = [&](int q) { return o->mats[m0 + (q >> 1)].m + 4 * (q & 1); };
        const int hb = 1 << (j - 1);
        for (int q1 = 0; q1 < 16; q1++) {
            if (!(q1 & hb)) continue;
            const float *a = entry(q1), *b = entry((q1 & (hb - 1)) | hb);
            if (std::memcmp(a, b, 4 * sizeof(float)) != 0) return false;
        }
        return true;
    }
    // s as an unevaluated FP32 sum hi + lo
    static int32_t push_scale(T2Pass *o, double s) {
        const float hi = (float)s;
        double m[8] = {};
        m[0] = hi;
        m[1] = (float)(s - (double)hi);
        return push_mat(o, m);
    }
    static void push_sterm(T2Pass *o, int g0, int g1, Ph th) {
        o->sterms.push_back({(int16_t)g0, (int16_t)g1, th});
    }
};

struct P64 {
    using Ph = uint64_t;
    using V = double;
    static Ph ph(uint64_t t64) { return t64; }
    static void ex(Ph u, V *re, V *im) {
        const double ang = 2.0 * M_PI * ((double)(int64_t)u * 0x1p-64);
        *re = std::cos(ang);
        *im = std::sin(ang);
    }
    static bool real(const double *m) { return m[1] == 0.0 && m[3] == 0.0 && m[5] == 0.0 && m[7] == 0.0; }
    // entries x of a phased butterfly on register bit j (bit j of x set)
    // depend only on register bits below j
    static constexpr bool kSharedTwiddles = true;
    static constexpr int kSharedMinJ = 0, kSharedMaxJ = 3;
    static bool table_low_only(const T2Pass *o, int m0, int j) {
        auto entry = [&](int x) { return &o->mats64[8 * (size_t)m0 + 2 * x]; };
        const int hb = 1 << j;
        for (int x = 0; x < 32; x++) {
            if (!(x & hb)) continue;
            if (std::memcmp(entry(x), entry((x & (hb - 1)) | hb), 2 * sizeof(double)) != 0) return false;
        }
        return true;
    }
    static int32_t push_mat(T2Pass *o, const double *m) {
        o->mats64.insert(o->mats64.end(), m, m + 8);
        return (int32_t)(o->mats64.size() / 8) - 1;
    }
    static size_t nmats(const T2Pass *o) { return o->mats64.size() / 8; }
    static size_t nrowvals(const T2Pass *o) { return o->statc64.size(); }
    static void push_row(T2Pass *o, V re, V im) {
        o->statc64.push_back(re);
        o->statc64.push_back(im);
    }
    // 32-entry table: entry x = (re, im) at doubles 2x, 2x + 1, eight records
    static int32_t push_table(T2Pass *o, const Ph *u) {
        const int32_t m0 = (int32_t)nmats(o);
        for (int x = 0; x < 32; x++) {
            double re, im;
            ex(u[x], &re, &im);
            o->mats64.push_back(re);
            o->mats64.push_back(im);
        }
        return m0;
    }
    static bool table_one(const T2Pass *o, int m0, int x) {
        const double *t = &o->mats64[8 * (size_t)m0 + 2 * x];
        return t[0] == 1.0 && t[1] == 0.0;
    }
    static int32_t push_scale(T2Pass *o, double s) {
        double m[8] = {};
        m[0] = s;
        return push_mat(o, m);
    }
    static void push_sterm(T2Pass *o, int g0, int g1, Ph th) {
        o->sterms64.push_back({(int16_t)g0, (int16_t)g1, 0, th});
    }
};

template <class P>
std::string compile_fmt2(const TilePass &tp, T2Pass *out, bool gen) {
    using Ph = typename P::Ph;
    using V = typename P::V;
    // a tile term with its phase in the policy's width
    struct TT {
        int32_t run, tb, g0, g1;
        Ph theta;
    };
    std::vector<TT> tts;
    *out = T2Pass{};
    out->wide = sizeof(Ph) == 8;
    if (tp.k != kT2Qubits && tp.k != kT2WideQubits) return "tile is not 2^13 or 2^14 amplitudes";
    if (tp.c < 4) return "chunk smaller than 16 amplitudes";
    for (const TileOp &op : tp.ops)
        if (op.type == TOP_SWAP) return "in-tile SWAP";
    int nruns = 0;
    for (const TileOp &op : tp.ops) nruns += op.type == TOP_DIAG;
    if (nruns > kT2MaxRuns) return "too many diagonal runs";
    out->format = 2;
    out->k = tp.k;
    out->c = tp.c;
    for (int s = 0; s < tp.k; s++) out->slot_phys[s] = tp.slot_phys[s];
    out->gmask = tp.gmask;
    out->ngates = tp.ngates;
    out->nruns = nruns;
    const int K = tp.k;
    const int NW = K - kT2RegBits - 5;
    const int NT = 1 << (K - kT2RegBits);
    const int TB = 5 + NW;
    out->rb = kT2RegBits;
    out->threads = NT;

    // the leading Hadamards (uncontrolled, distinct tile bits, before any
    // other step): part of the generated state in the variant for a pass
    // that starts from a recorded basis state
    size_t first = 0;
    if (gen) {
        for (; first < tp.ops.size(); first++) {
            const TileOp &op = tp.ops[first];
            if (op.type != TOP_H || ((out->gen_hmask >> op.slot) & 1u)) break;
            out->gen_hmask |= 1u << op.slot;
            out->n_h++;
        }
    }

    std::map<std::pair<int, int>, int> slot_of;
    std::map<std::vector<Ph>, int32_t> table_of;  // table phases -> first matrix record
    auto slot = [&](int i0, int i1) -> int {
        auto key = std::make_pair(i0, i1);
        auto it = slot_of.find(key);
        if (it != slot_of.end()) return it->second;
        const int s = (int)out->slots.size();
        out->slots.push_back({(int16_t)i0, (int16_t)i1});
        slot_of[key] = s;
        return s;
    };

    Lay L;
    auto emit_stage = [&](const Lay &l) {
        T2Stage st{};
        for (int j = 0; j < kT2RegBits; j++) st.tb[j] = (int8_t)l.reg[j];
        for (int t = 0; t < 5; t++) st.tb[5 + t] = (int8_t)l.lane[t];
        for (int w = 0; w < NW; w++) st.tb[10 + w] = (int8_t)l.warp[w];
        T2Ins in{};
        in.op = T2_STAGE;
        in.hd = kT2HdStage;
        in.aux = (int32_t)out->stages.size();
        out->stages.push_back(st);
        out->ins.push_back(in);
        L = l;
    };
    {
        int r[4];
        pick_regs(tp, first, !gen, r);
        emit_stage(make_layout(K, r, !gen));
    }
    int run = 0;
    for (size_t i = first; i < tp.ops.size(); i++) {
        const TileOp &op = tp.ops[i];
        // a stage change moves data only, so it commutes with diagonal runs:
        // the layout of the next gate is taken before the runs that precede
        // it, which then compile in the stage of the gate they feed (and can
        // become phased butterflies with it)
        size_t g = i;
        while (g < tp.ops.size() && !is_gate(tp.ops[g].type)) g++;
        if (g < tp.ops.size() && L.cls[tp.ops[g].slot] != T2C_REG) {
            int r[4];
            pick_regs(tp, g, false, r);
            emit_stage(make_layout(K, r, false));
        }
        if (is_gate(op.type)) {
            T2Ins in{};
            in.op = (int8_t)(op.type == TOP_H ? T2_H : op.type == TOP_X ? T2_X : T2_GATE);
            if (in.op == T2_GATE && P::real(op.m)) in.op = T2_RGATE;  // a real matrix (a rotation RY, for one)
            // an uncontrolled rotation [[c, -s], [s, c]] runs as three shears;
            // with c < 0 it is -1 times the rotation by c' = -c, s' = -s, and
            // the sign joins the pass's closing scale
            double rot_t = 0.0, rot_s = 0.0;
            if (in.op == T2_RGATE && op.type == TOP_GATE) {
                const double c = op.m[0], s = op.m[4];
                if (op.m[6] == c && op.m[2] == -s && std::fabs(c * c + s * s - 1.0) <= 1e-12) {
                    const bool flip = c < 0.0;
                    const double cc = flip ? -c : c, ss = flip ? -s : s;
                    rot_t = -ss / (1.0 + cc);
                    rot_s = ss;
                    if (flip) out->sign_flips++;
                    in.op = T2_ROT;
                }
            }
            in.cls = (int8_t)T2C_REG;
            in.idx = (int8_t)L.pos[op.slot];
            in.ccls = T2C_NONE;
            if (op.type == TOP_GATE_CL) {
                const int c = op.cslot;
                if (L.cls[c] == T2C_REG) {
                    in.ccls = (int8_t)T2C_REG;
                    in.cidx = (int16_t)L.pos[c];
                    // packed pairs q (register bits 1..4 = bits 0..3 of q) that
                    // hold the control; control on register bit 0: odd elements
                    uint32_t pm = 0;
                    for (int q = 0; q < 16; q++)
                        if (L.pos[c] == 0 || ((q >> (L.pos[c] - 1)) & 1)) pm |= 1u << q;
                    in.e0 = (int16_t)(uint16_t)pm;
                    in.e1 = (int16_t)(L.pos[c] == 0 ? 1 : 0);
                } else {
                    in.ccls = (int8_t)T2C_THREAD;
                    in.cidx = (int16_t)L.pos[c];
                }
            } else if (op.type == TOP_GATE_CG) {
                in.ccls = T2C_GLOBAL;
                in.cidx = (int16_t)op.cbit;
            }
            if (in.op == T2_ROT) {
                double m[8] = {};
                m[0] = rot_t;
                m[1] = rot_s;
                in.aux = P::push_mat(out, m);
            } else if (in.op == T2_GATE || in.op == T2_RGATE) {
                in.aux = P::push_mat(out, op.m);
            }
            const int kind = in.op == T2_H ? 0 : in.op == T2_X ? 1 : in.op == T2_RGATE ? 2
                           : in.op == T2_ROT ? 3 : 4;
            const int hslot = in.ccls == T2C_NONE ? in.idx : 7;
            in.hd = (int16_t)(kT2Handler + 8 * kind + hslot);
            if (op.type == TOP_H) out->n_h++;
            out->ins.push_back(in);
            continue;
        }
        // ---- diagonal run against layout L
        const int r = run++;
        Ph sl[kT2MaxQubits] = {};  // static linear coefficient of each tile bit
        bool dyn[kT2MaxQubits] = {};     // tile bit with a per-tile (global) coefficient
        bool use_cst = false;
        Ph rt[kT2RegBits][kMaxThreadBits] = {};  // register x thread pairs
        Ph tt[kMaxThreadBits][kMaxThreadBits] = {};
        std::map<int, Ph> rr;  // register-bit mask -> theta
        for (int t = op.tb; t < op.te; t++) {
            const PhaseTerm &pt = tp.terms[t];
            const Ph th = P::ph(pt.theta);
            if (!th) continue;
            switch (pt.kind) {
                case TERM_L:
                    sl[pt.a] += th;
                    break;
                case TERM_G:
                    tts.push_back({r, -1, pt.a, -1, th});
                    use_cst = true;
                    break;
                case TERM_GG:
                    tts.push_back({r, -1, pt.a, pt.b, th});
                    use_cst = true;
                    break;
                case TERM_LG:
                    tts.push_back({r, pt.a, pt.b, -1, th});
                    dyn[pt.a] = true;
                    break;
                case TERM_LL: {
                    const int a = pt.a, b = pt.b;
                    const bool ra = L.cls[a] == T2C_REG, rb = L.cls[b] == T2C_REG;
                    if (ra && rb) {
                        rr[(1 << L.pos[a]) | (1 << L.pos[b])] += th;
                    } else if (ra || rb) {
                        rt[ra ? L.pos[a] : L.pos[b]][ra ? L.pos[b] : L.pos[a]] += th;
                    } else {
                        tt[L.pos[a]][L.pos[b]] += th;
                        tt[L.pos[b]][L.pos[a]] += th;
                    }
                    break;
                }
                default:
                    return "unknown phase term";
            }
        }
        // constants: (register mask, thread predicate 0 = all / t + 1) -> phase
        std::map<std::pair<int, int>, Ph> cst;
        std::vector<T2Fac> facs;
        // a static row over the thread index: a constant, a constant on the
        // threads with one bit set (thread factors only: a register-bit
        // factor keeps such a row, so that the run can still become a phased
        // butterfly), or a complex row
        auto add_factor = [&](int mask, const Ph *row, int sl0, int dmask) {
            bool any = false;
            for (int tau = 0; tau < NT; tau++) any |= row[tau] != 0;
            int rowi = -1;
            if (any) {
                bool uniform = true;
                for (int tau = 1; tau < NT && uniform; tau++) uniform = row[tau] == row[0];
                int single = -1;
                if (!uniform && mask == 0)
                    for (int t = 0; t < TB && single < 0; t++) {
                        const Ph th = row[1 << t];
                        if (!th) continue;
                        bool ok = true;
                        for (int tau = 0; tau < NT && ok; tau++)
                            ok = row[tau] == (((tau >> t) & 1) ? th : 0u);
                        if (ok) single = t;
                        else break;
                    }
                if (uniform) {
                    cst[{mask, 0}] += row[0];
                } else if (single >= 0) {
                    cst[{mask, single + 1}] += row[1 << single];
                } else {
                    rowi = (int)(P::nrowvals(out) / (2 * (size_t)NT));
                    for (int tau = 0; tau < NT; tau++) {
                        V re, im;
                        P::ex(row[tau], &re, &im);
                        P::push_row(out, re, im);
                    }
                }
            }
            if (rowi < 0 && sl0 < 0 && dmask == 0) return;
            T2Fac f{};
            f.w0 = (uint32_t)mask | (1u << 8) | ((uint32_t)dmask << kFacDynShift);
            f.slot = (int16_t)sl0;
            f.dslot = -1;
            f.row = rowi;
            if (dmask) {  // one slot per dynamic thread bit, consecutive
                f.dslot = (int16_t)out->slots.size();
                for (int t = 0; t < TB; t++)
                    if ((dmask >> t) & 1) out->slots.push_back({(int16_t)(r * 16 + L.ttb(t)), -1});
            }
            facs.push_back(f);
        };
        {  // thread factor (every amplitude of the thread)
            Ph row[1 << (kT2MaxQubits - kT2RegBits)];
            row[0] = 0;
            for (int tau = 1; tau < NT; tau++) {
                const int b = __builtin_ctz((unsigned)tau);
                const int prev = tau & (tau - 1);
                Ph u = row[prev] + sl[L.ttb(b)];
                for (int rest = prev; rest; rest &= rest - 1) u += tt[b][__builtin_ctz((unsigned)rest)];
                row[tau] = u;
            }
            int dmask = 0;
            for (int t = 0; t < TB; t++)
                if (dyn[L.ttb(t)]) dmask |= 1 << t;
            const int s0 = use_cst ? slot(r * 16 + 15, -1) : -1;
            add_factor(0, row, s0, dmask);
        }
        for (int j = 0; j < kT2RegBits; j++) {  // one factor per register bit with a coefficient
            const int tb = L.reg[j];
            Ph row[1 << (kT2MaxQubits - kT2RegBits)];
            row[0] = sl[tb];
            for (int tau = 1; tau < NT; tau++)
                row[tau] = row[tau & (tau - 1)] + rt[j][__builtin_ctz((unsigned)tau)];
            add_factor(1 << j, row, dyn[tb] ? slot(r * 16 + tb, -1) : -1, 0);
        }
        for (auto &kv : rr)
            if (kv.second) cst[{kv.first, 0}] += kv.second;
        // constants with the same thread predicate merge into one 32-entry table
        std::map<int, std::vector<std::pair<int, Ph>>> group;
        for (auto &kv : cst)
            if (kv.second) group[kv.first.second].push_back({kv.first.first, kv.second});
        T2Ins in{};
        in.op = T2_DIAG;
        in.hd = kT2HdDiag;
        in.e0 = (int16_t)out->fac2.size();
        for (auto &g : group) {
            Ph u[32] = {};
            for (auto &mc : g.second)
                for (int x = 0; x < 32; x++)
                    if ((x & mc.first) == mc.first) u[x] += mc.second;
            // identical tables share their matrix records
            std::vector<Ph> key(u, u + 32);
            auto hit = table_of.find(key);
            int32_t m0;
            if (hit != table_of.end()) {
                m0 = hit->second;
            } else {
                m0 = P::push_table(out, u);
                table_of[key] = m0;
            }
            T2Fac f{};
            f.w0 = kFacTable | ((uint32_t)g.first << 10);
            f.slot = f.dslot = -1;
            f.row = m0;
            out->fac2.push_back(f);
        }
        out->fac2.insert(out->fac2.end(), facs.begin(), facs.end());
        in.e1 = (int16_t)out->fac2.size();
        if (out->fac2.size() > 32000) return "too many factor applications";
        if (in.e1 > in.e0) out->ins.push_back(in);
    }
    if (out->slots.size() > (size_t)kT2MaxSlots) return "too many per-tile phase slots";
    // each slot's terms (those of its two phase words), for the kernel
    out->soff.push_back(0);
    for (const T2Slot &sl : out->slots) {
        int nterm = 0;
        for (const TT &t : tts) {
            const int li = t.run * 16 + (t.tb >= 0 ? t.tb : 15);
            if (li == sl.i0 || (sl.i1 >= 0 && li == sl.i1)) {
                P::push_sterm(out, t.g0, t.g1, t.theta);
                nterm++;
            }
        }
        out->soff.push_back(out->soff.back() + nterm);
    }
    if (!out->wide)  // the 32-bit tile terms, as the format-1 compiler records them
        for (const TT &t : tts) out->tterms.push_back({t.run, t.tb, t.g0, t.g1, (uint32_t)t.theta, 0});
    // the phased butterfly: a run that is the identity where register bit j
    // is 0 (at most one unpredicated table, one per-thread factor on bit j)
    // directly followed by an uncontrolled H on register bit j
    auto phased_ok = [&](const T2Ins &d, int j) {
        int ntab = 0, nthr = 0;
        for (int e = d.e0; e < d.e1; e++) {
            const T2Fac &f = out->fac2[e];
            if (f.w0 & kFacTable) {
                if (((f.w0 >> 10) & 0xfu) || ++ntab > 1) return false;
                for (int x = 0; x < 32; x++) {
                    if ((x >> j) & 1) continue;
                    if (!P::table_one(out, f.row, x)) return false;
                }
            } else {
                if ((f.w0 & 0xffu) != (1u << j) || ((f.w0 >> kFacDynShift) & 0x1ffu) || ++nthr > 1)
                    return false;
            }
        }
        return d.e1 > d.e0;
    };
    {
        std::vector<T2Ins> merged;
        for (size_t i = 0; i < out->ins.size(); i++) {
            const T2Ins &d = out->ins[i];
            if (d.op == T2_DIAG && i + 1 < out->ins.size()) {
                const T2Ins &hh = out->ins[i + 1];
                if (hh.op == T2_H && hh.ccls == T2C_NONE && phased_ok(d, hh.idx)) {
                    T2Ins f = hh;
                    f.op = T2_HPH;
                    f.e0 = d.e0;
                    f.e1 = d.e1;
                    f.hd = (int16_t)(kT2Handler + 8 * 5 + hh.idx);
                    // the run's table, static row and slot, also in the step
                    // itself (tileprog.h: T2_HPH), so that the register-stage
                    // kernels read them without the factor records
                    int trec = -1, row = -1, sl = -1;
                    for (int e = d.e0; e < d.e1; e++) {
                        const T2Fac &fc = out->fac2[e];
                        if (fc.w0 & kFacTable) {
                            trec = fc.row;
                        } else {
                            row = fc.row;
                            sl = fc.slot;
                        }
                    }
                    f.ccls = kT2HphDirect;
                    if (P::kSharedTwiddles && trec >= 0 && hh.idx >= P::kSharedMinJ &&
                        hh.idx <= P::kSharedMaxJ && P::table_low_only(out, trec, hh.idx))
                        f.ccls = kT2HphShared;
                    f.cidx = (int16_t)sl;
                    f.aux = (int32_t)(((uint32_t)(row + 1) << 16) | (uint32_t)(trec + 1));
                    merged.push_back(f);
                    i++;
                    continue;
                }
            }
            merged.push_back(d);
        }
        out->ins.swap(merged);
    }
    // coalesced write-back: the last stage has lane bits 0..2 = tile bits 1..3
    if (!L.canonical()) {
        int r[4], n = 0;
        for (int j = 1; j < kT2RegBits; j++)
            if (L.reg[j] > 3) r[n++] = L.reg[j];
        for (int tb = K - 1; tb >= 4 && n < 4; tb--) {
            bool seen = false;
            for (int j = 0; j < n; j++) seen |= r[j] == tb;
            if (!seen) r[n++] = tb;
        }
        emit_stage(make_layout(K, r, true));
    }
    if (out->ins.size() > (size_t)kT2SmemIns || out->fac2.size() > (size_t)kT2SmemFactors)
        return "programme longer than the kernel's shared-memory copy";
    if (P::nmats(out) > (size_t)kT2SmemMats) return "more matrix records than the kernel's shared-memory copy";
    for (size_t i = 0; i < out->ins.size(); i++)
        if (out->ins[i].op == T2_STAGE) out->last_stage = (int)i;
    // kernel-side layouts (linear and swizzled) and the write-back offsets
    out->layx.resize(out->stages.size());
    for (size_t si = 0; si < out->stages.size(); si++) {
        const T2Stage &st = out->stages[si];
        T2LayoutX &x = out->layx[si];
        for (int v = 0; v < 32; v++) {
            int lo = 0;
            for (int t = 0; t < 5; t++)
                if ((v >> t) & 1) lo += 1 << st.tb[5 + t];
            x.lo[v] = (uint16_t)lo;
            x.plo[v] = (uint16_t)swz(lo >> 1);
        }
        for (int v = 0; v < 16; v++) {
            int hi = 0;
            for (int t = 0; t < NW; t++)
                if ((v >> t) & 1) hi += 1 << st.tb[10 + t];
            x.hi[v] = (uint16_t)hi;
            x.phi[v] = (uint16_t)swz(hi >> 1);
        }
        for (int j = 0; j < 4; j++) {
            x.s[j] = 1 << st.tb[1 + j];
            x.ps[j] = swz(x.s[j] >> 1);
        }
    }
    {
        const T2Stage &st = out->stages[out->ins[out->last_stage].aux];
        auto w = [&](int tb) { return UINT64_C(1) << tp.slot_phys[tb]; };
        for (int v = 0; v < 32; v++) {
            uint64_t lo = 0;
            for (int t = 0; t < 5; t++)
                if ((v >> t) & 1) lo += w(st.tb[5 + t]);
            out->epi.glo[v] = lo;
        }
        for (int v = 0; v < 16; v++) {
            uint64_t hi = 0;
            for (int t = 0; t < NW; t++)
                if ((v >> t) & 1) hi += w(st.tb[10 + t]);
            out->epi.ghi[v] = hi;
        }
        for (int j = 0; j < 4; j++) out->epi.g[j] = w(st.tb[1 + j]);
    }
    if (out->n_h || (out->sign_flips & 1)) {
        const double s = std::pow(2.0, -0.5 * out->n_h) * ((out->sign_flips & 1) ? -1.0 : 1.0);
        if (gen) {
            // every step is linear: the pass that generates its starting
            // state generates it times the closing scale instead
            out->gen_scale = s;
            return "";
        }
        T2Ins in{};
        in.op = T2_SCALE;
        in.hd = kT2HdScale;
        in.aux = P::push_scale(out, s);
        out->ins.push_back(in);
    }
    if (P::nmats(out) > (size_t)kT2SmemMats) return "more matrix records than the kernel's shared-memory copy";
    return "";
}

}  // namespace

std::string compile_t2v2(const TilePass &tp, T2Pass *out, bool gen) { return compile_fmt2<P32>(tp, out, gen); }

std::string compile_t2v2_c128(const TilePass &tp, T2Pass *out, bool gen) {
    if (tp.k != kT2Qubits) return "complex128 register-stage tiles hold 2^13 amplitudes";
    return compile_fmt2<P64>(tp, out, gen);
}

}  // namespace sv
