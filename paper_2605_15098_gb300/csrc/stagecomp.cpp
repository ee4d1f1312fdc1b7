// Stage compiler, format 1: tile pass (plan.h) -> register-stage programme of
// the fused tensor-core kernel (k_tile3; tileprog.h).  Passes without fused
// blocks compile to format 2 (stagecomp2.cpp).
//
// Layouts are chosen greedily: a stage starts at the first gate that the
// previous layout cannot execute and takes as register bits the first four
// new target bits that the following non-diagonal gates need.  Tile bit 0 is
// always register bit 0 and tile bits 1..3 are always lane bits 0..2 (gates
// on them use shuffles); every other target must be a register bit.  The
// remaining tile bits fill lane bits 3..4 and the warp bits.  Diagonal runs
// are compiled against the layout of the stage that executes them; register-
// bit gates between two shuffle gates or stage changes fold into one 32x32
// block.
#include <cmath>
#include <complex>
#include <cstring>
#include <tuple>
#include <map>
#include <string>

#include "common.h"
#include "plan.h"
#include "stagecomp.h"

namespace sv {
namespace {

uint32_t turns32(uint64_t t64) { return (uint32_t)((t64 + (UINT64_C(1) << 31)) >> 32); }

struct Layout {
    int rb = kT2RegBits, nwarp = kT2WarpBits;  // geometry
    int reg[kMaxRegBits];  // tile bit of register bit j
    int lane[5];           // tile bit of lane bit l
    int warp[4];           // tile bit of warp bit w
    int cls[kT2MaxQubits];  // T2C_REG / T2C_LANE / T2C_THREAD (warp)
    int pos[kT2MaxQubits];  // register bit, or thread bit (lane l -> l, warp w -> 5 + w)

    void index() {
        for (int j = 0; j < rb; j++) {
            cls[reg[j]] = T2C_REG;
            pos[reg[j]] = j;
        }
        for (int l = 0; l < 5; l++) {
            cls[lane[l]] = T2C_LANE;
            pos[lane[l]] = l;
        }
        for (int w = 0; w < nwarp; w++) {
            cls[warp[w]] = T2C_THREAD;
            pos[warp[w]] = 5 + w;
        }
    }
    int tbits() const { return 5 + nwarp; }
    int thread_tile_bit(int t) const { return t < 5 ? lane[t] : warp[t - 5]; }
};

bool is_gate_op(int type) {
    return type == TOP_GATE || type == TOP_GATE_CL || type == TOP_GATE_CG || type == TOP_H ||
           type == TOP_X;
}

Layout choose_layout(const TilePass &tp, int from, int rb, int nwarp) {
    Layout L{};
    L.rb = rb;
    L.nwarp = nwarp;
    bool used[kT2MaxQubits] = {};
    L.reg[0] = 0;
    used[0] = true;
    for (int l = 0; l < 3; l++) {
        L.lane[l] = 1 + l;
        used[1 + l] = true;
    }
    int nreg = 1, nlane = 3, nw = 0;
    // the next gate targets become register bits, then lane bits 3 and 4
    // (gates there are warp shuffles, cheaper than another stage change)
    for (size_t i = from; i < tp.ops.size() && (nreg < rb || nlane < 5); i++) {
        const TileOp &op = tp.ops[i];
        if (!is_gate_op(op.type)) continue;
        const int t = op.slot;
        if (used[t]) continue;
        if (nreg < rb)
            L.reg[nreg++] = t;
        else
            L.lane[nlane++] = t;
        used[t] = true;
    }
    for (int t = 0; t < tp.k; t++) {
        if (used[t]) continue;
        if (nreg < rb)
            L.reg[nreg++] = t;
        else if (nlane < 5)
            L.lane[nlane++] = t;
        else
            L.warp[nw++] = t;
        used[t] = true;
    }
    L.index();
    return L;
}

using cplx = std::complex<double>;

struct Block {
    cplx m[32][32];
    void identity() {
        for (int r = 0; r < 32; r++)
            for (int c = 0; c < 32; c++) m[r][c] = r == c ? 1.0 : 0.0;
    }
    // m <- G m, G = u on register bit j (controlled on register bit c when c >= 0)
    void gate(int j, const cplx u[4], int c) {
        for (int k = 0; k < 32; k++)
            for (int r = 0; r < 32; r++) {
                if ((r >> j) & 1) continue;
                if (c >= 0 && !((r >> c) & 1)) continue;
                const int r1 = r | (1 << j);
                const cplx a = m[r][k], b = m[r1][k];
                m[r][k] = u[0] * a + u[1] * b;
                m[r1][k] = u[2] * a + u[3] * b;
            }
    }
    // m <- diag(e^{2 pi i ph[r] / 2^64}) m
    void phase(const uint64_t ph[32]) {
        for (int r = 0; r < 32; r++) {
            if (!ph[r]) continue;
            const double ang = 2.0 * M_PI * ((double)(int64_t)ph[r] * 0x1p-64);
            const cplx f(std::cos(ang), std::sin(ang));
            for (int k = 0; k < 32; k++) m[r][k] *= f;
        }
    }
};

float tf32_round(float x) {
    uint32_t b;
    std::memcpy(&b, &x, 4);
    b = (b + 0x1000u) & ~0x1FFFu;  // nearest, ties away from zero (magnitude)
    float r;
    std::memcpy(&r, &b, 4);
    return r;
}

void block_device_layout(const Block &B, float *dst) {
    for (int part = 0; part < 2; part++)  // 0: hi, 1: lo
        for (int ri = 0; ri < 2; ri++)    // 0: re, 1: im
            for (int n = 0; n < 32; n++)
                for (int k = 0; k < 32; k++) {
                    const double v = ri ? B.m[n][k].imag() : B.m[n][k].real();
                    const float hi = tf32_round((float)v);
                    const float val = part ? (float)(v - (double)hi) : hi;
                    const int off = (n / 8) * 256 + (k / 4) * 32 + (n % 8) * 4 + (k % 4);
                    dst[(part * 2 + ri) * 1024 + off] = val;
                }
}

bool executable(const Layout &L, const TileOp &op) {
    if (!is_gate_op(op.type)) return true;
    return L.cls[op.slot] == T2C_REG || L.cls[op.slot] == T2C_LANE;
}

}  // namespace

bool unitary2(const double *m) {
    const cplx a(m[0], m[1]), b(m[2], m[3]), c(m[4], m[5]), d(m[6], m[7]);
    const cplx p00 = std::conj(a) * a + std::conj(c) * c, p11 = std::conj(b) * b + std::conj(d) * d;
    const cplx p01 = std::conj(a) * b + std::conj(c) * d;
    return std::abs(p00 - 1.0) < 1e-9 && std::abs(p11 - 1.0) < 1e-9 && std::abs(p01) < 1e-9;
}

std::string compile_t2(const TilePass &tp, T2Pass *out, bool fused) {
    if (!fused) return compile_t2v2(tp, out, false);
    *out = T2Pass{};
    if (fused)
        for (const TileOp &op : tp.ops)
            if ((op.type == TOP_GATE || op.type == TOP_GATE_CL || op.type == TOP_GATE_CG) &&
                !unitary2(op.m))
                return "non-unitary gate matrix (fused passes renormalise)";
    if (tp.k != kT2Qubits) return "tile is not 2^13 amplitudes";
    if (tp.c < 4) return "chunk smaller than 16 amplitudes";
    for (const TileOp &op : tp.ops)
        if (op.type == TOP_SWAP) return "in-tile SWAP";
    int nruns = 0;
    for (const TileOp &op : tp.ops) nruns += op.type == TOP_DIAG;
    if (nruns > kT2MaxRuns) return "too many diagonal runs";
    out->k = tp.k;
    out->c = tp.c;
    for (int s = 0; s < tp.k; s++) out->slot_phys[s] = tp.slot_phys[s];
    out->gmask = tp.gmask;
    out->ngates = tp.ngates;
    out->nruns = nruns;
    // geometry: the fused kernel needs 5 register bits (32x32 blocks)
    const int RB = fused ? kT3RegBits : kT2RegBits;
    const int NW = tp.k - RB - 5;                    // warp bits: 3, or 4 for a 2^14 tile
    const int NT = 1 << (tp.k - RB);                 // threads = rows of a static phase table
    const int TB = 5 + NW;                           // thread bits
    out->rb = RB;
    out->threads = NT;

    auto emit_stage = [&](const Layout &L) {
        T2Stage st{};
        for (int j = 0; j < RB; j++) st.tb[j] = (int8_t)L.reg[j];
        for (int l = 0; l < 5; l++) st.tb[5 + l] = (int8_t)L.lane[l];
        for (int w = 0; w < NW; w++) st.tb[10 + w] = (int8_t)L.warp[w];
        T2Ins in{};
        in.op = T2_STAGE;
        in.aux = (int32_t)out->stages.size();
        out->stages.push_back(st);
        out->ins.push_back(in);
    };

    Layout L = choose_layout(tp, 0, RB, NW);
    emit_stage(L);
    int run = 0;
    // fused mode: register-bit gates accumulate into a block; thread-dependent
    // diagonal factors that commute with it wait in `pre` (applied before it)
    Block blk;
    blk.identity();
    bool dirty = false;
    int nd = 0;  // register bits the block acts on non-diagonally
    std::vector<T2Factor> pre;
    auto flush = [&]() -> std::string {
        if (!pre.empty()) {
            T2Ins in{};
            in.op = T2_DIAG;
            in.e0 = (int16_t)out->factors.size();
            out->factors.insert(out->factors.end(), pre.begin(), pre.end());
            in.e1 = (int16_t)out->factors.size();
            out->ins.push_back(in);
            pre.clear();
        }
        if (dirty) {
            if (out->nblocks >= 256) return "more than 256 fused blocks in one pass";
            T2Ins in{};
            in.op = T2_BLOCK;
            in.aux = out->nblocks++;
            for (int r = 0; r < 32; r++)
                for (int c = 0; c < 32; c++) out->blocks64.push_back(blk.m[r][c].real());
            for (int r = 0; r < 32; r++)
                for (int c = 0; c < 32; c++) out->blocks64.push_back(blk.m[r][c].imag());
            const size_t off = out->blocks_dev.size();
            out->blocks_dev.resize(off + kBlockFloats);
            block_device_layout(blk, out->blocks_dev.data() + off);
            out->ins.push_back(in);
            blk.identity();
            dirty = false;
            nd = 0;
        }
        return "";
    };
    for (size_t i = 0; i < tp.ops.size(); i++) {
        const TileOp &op = tp.ops[i];
        if (!executable(L, op)) {
            if (fused) {
                std::string e = flush();
                if (!e.empty()) return e;
            }
            L = choose_layout(tp, (int)i, RB, NW);
            emit_stage(L);
        }
        if (fused && is_gate_op(op.type) && L.cls[op.slot] == T2C_REG &&
            (op.type != TOP_GATE_CL || L.cls[op.cslot] == T2C_REG) && op.type != TOP_GATE_CG) {
            cplx u[4];
            if (op.type == TOP_H) {
                const double r = 0.70710678118654752440084436210485;
                u[0] = r; u[1] = r; u[2] = r; u[3] = -r;
            } else if (op.type == TOP_X) {
                u[0] = 0; u[1] = 1; u[2] = 1; u[3] = 0;
            } else {
                for (int e = 0; e < 4; e++) u[e] = cplx(op.m[2 * e], op.m[2 * e + 1]);
            }
            const int j = L.pos[op.slot];
            const int c = op.type == TOP_GATE_CL ? L.pos[op.cslot] : -1;
            blk.gate(j, u, c);
            nd |= 1 << j;
            dirty = true;
            continue;
        }
        if (fused && is_gate_op(op.type)) {  // shuffle gate, or a control the block cannot hold
            std::string e = flush();
            if (!e.empty()) return e;
        }
        if (is_gate_op(op.type)) {
            T2Ins in{};
            in.op = (int8_t)(op.type == TOP_H ? T2_H : op.type == TOP_X ? T2_X : T2_GATE);
            if (in.op == T2_GATE && (float)op.m[1] == 0.f && (float)op.m[3] == 0.f &&
                (float)op.m[5] == 0.f && (float)op.m[7] == 0.f)
                in.op = T2_RGATE;  // a real matrix (a rotation RY, for one)
            in.cls = (int8_t)L.cls[op.slot];
            in.idx = (int8_t)L.pos[op.slot];
            in.ccls = T2C_NONE;
            if (op.type == TOP_GATE_CL) {
                const int c = op.cslot;
                if (L.cls[c] == T2C_REG) return "gate controlled by a register bit";
                in.ccls = (int8_t)T2C_THREAD;
                in.cidx = (int16_t)L.pos[c];
            } else if (op.type == TOP_GATE_CG) {
                in.ccls = T2C_GLOBAL;
                in.cidx = (int16_t)op.cbit;
            }
            if (in.op == T2_GATE || in.op == T2_RGATE) {
                T2Mat m{};
                for (int e = 0; e < 8; e++) m.m[e] = (float)op.m[e];
                in.aux = (int32_t)out->mats.size();
                out->mats.push_back(m);
            }
            {  // dispatch code (tileprog.h)
                const int kind = in.op == T2_H ? 0 : in.op == T2_X ? 1 : in.op == T2_RGATE ? 2 : 4;
                int slot = 7;
                if (in.ccls == T2C_NONE && in.cls == T2C_REG) slot = in.idx;
                else if (in.ccls == T2C_NONE && in.cls == T2C_LANE) slot = 5;
                else if (in.ccls == T2C_THREAD && in.cls == T2C_LANE) slot = 6;
                in.hd = (int16_t)(kT2Handler + 8 * kind + slot);
            }
            if (op.type == TOP_H) out->n_h++;
            out->ins.push_back(in);
            continue;
        }
        // ---- diagonal run: compile its phase polynomial against layout L
        const int r = run++;
        uint32_t sl[kT2MaxQubits] = {};  // static linear coefficient of each tile bit
        bool dyn[kT2MaxQubits] = {};     // tile bit has global-dependent (per-tile) terms
        bool use_cst = false;
        uint32_t rt[kMaxRegBits][kMaxThreadBits] = {};
        std::vector<std::tuple<int, int, uint32_t>> tt;
        std::map<int, uint32_t> rr;     // register-bit mask -> theta
        for (int t = op.tb; t < op.te; t++) {
            const PhaseTerm &pt = tp.terms[t];
            const uint32_t th = turns32(pt.theta);
            if (!th) continue;
            switch (pt.kind) {
                case TERM_L:
                    sl[pt.a] += th;
                    break;
                case TERM_G:
                    out->tterms.push_back({r, -1, pt.a, -1, th, 0});
                    use_cst = true;
                    break;
                case TERM_GG:
                    out->tterms.push_back({r, -1, pt.a, pt.b, th, 0});
                    use_cst = true;
                    break;
                case TERM_LG:
                    out->tterms.push_back({r, pt.a, pt.b, -1, th, 0});
                    dyn[pt.a] = true;
                    break;
                case TERM_LL: {
                    const int a = pt.a, b = pt.b;
                    const bool ra = L.cls[a] == T2C_REG, rb = L.cls[b] == T2C_REG;
                    if (ra && rb) {
                        rr[(1 << L.pos[a]) | (1 << L.pos[b])] += th;
                    } else if (ra || rb) {
                        const int j = ra ? L.pos[a] : L.pos[b];
                        const int tbit = ra ? L.pos[b] : L.pos[a];
                        rt[j][tbit] += th;
                    } else {
                        tt.emplace_back(L.pos[a], L.pos[b], th);
                    }
                    break;
                }
                default:
                    return "unknown phase term";
            }
        }
        if (fused) {
            // register-only part (linear terms on register bits, pairs of register bits)
            // folds into the block at this position, in full 64-bit phase precision
            uint64_t ph[32] = {};
            for (int t = op.tb; t < op.te; t++) {
                const PhaseTerm &pt = tp.terms[t];
                if (pt.kind == TERM_L && L.cls[pt.a] == T2C_REG) {
                    for (int rr_ = 0; rr_ < 32; rr_++)
                        if ((rr_ >> L.pos[pt.a]) & 1) ph[rr_] += pt.theta;
                    sl[pt.a] = 0;
                } else if (pt.kind == TERM_LL && L.cls[pt.a] == T2C_REG && L.cls[pt.b] == T2C_REG) {
                    for (int rr_ = 0; rr_ < 32; rr_++)
                        if (((rr_ >> L.pos[pt.a]) & (rr_ >> L.pos[pt.b])) & 1) ph[rr_] += pt.theta;
                }
            }
            rr.clear();
            bool any_ph = false;
            for (int rr_ = 0; rr_ < 32; rr_++) any_ph |= ph[rr_] != 0;
            if (any_ph) {
                blk.phase(ph);
                dirty = true;
            }
        }
        T2Ins in{};
        in.op = T2_DIAG;
        in.e0 = (int16_t)out->factors.size();
        const size_t nfac0 = out->factors.size();
        std::map<size_t, uint32_t> cturn;  // phase (turns / 2^32) of each constant factor
        auto add_thread_factor = [&](int mask, bool cst, int lin_reg, int dmask,
                                     const uint32_t *row) {
            T2Factor f{};
            // a static row theta * (bit t of the thread) is a constant factor
            // that only the threads with bit t set apply: no table lookups
            if (!cst && lin_reg < 0 && dmask == 0) {
                bool uniform = true;  // the same phase in every thread: a constant
                for (int tau = 1; tau < NT && uniform; tau++) uniform = row[tau] == row[0];
                if (uniform) {
                    const uint32_t w0 = (uint32_t)mask;
                    std::memcpy(&f.w0, &w0, sizeof w0);
                    f.run = r;
                    const double ang = 2.0 * M_PI * ((double)(int32_t)row[0] * 0x1p-32);
                    f.c0 = (float)std::cos(ang);
                    f.c1 = (float)std::sin(ang);
                    cturn[out->factors.size()] = row[0];
                    out->factors.push_back(f);
                    return;
                }
                for (int t = 0; t < TB; t++) {
                    const uint32_t th = row[1 << t];
                    if (!th) continue;
                    bool single = true;
                    for (int tau = 0; tau < NT && single; tau++)
                        single = row[tau] == (((tau >> t) & 1) ? th : 0u);
                    if (!single) break;
                    const uint32_t w0 = (uint32_t)mask | ((uint32_t)(t + 1) << 10);
                    std::memcpy(&f.w0, &w0, sizeof w0);
                    f.run = r;
                    const double ang = 2.0 * M_PI * ((double)(int32_t)th * 0x1p-32);
                    f.c0 = (float)std::cos(ang);
                    f.c1 = (float)std::sin(ang);
                    cturn[out->factors.size()] = th;
                    out->factors.push_back(f);
                    return;
                }
            }
            const uint32_t w0 = (uint32_t)mask | (1u << 8) | (cst ? (1u << 9) : 0u) |
                                ((uint32_t)(lin_reg + 1) << kFacLinShift) |
                                ((uint32_t)dmask << kFacDynShift);
            std::memcpy(&f.w0, &w0, sizeof w0);
            f.run = r;
            const int32_t rowi = (int32_t)(out->stat.size() / NT);
            std::memcpy(&f.c0, &rowi, sizeof rowi);
            out->stat.insert(out->stat.end(), row, row + NT);
            out->factors.push_back(f);
        };
        // thread factor (all amplitudes of the thread)
        {
            uint32_t row[1 << (kT2MaxQubits - kT2RegBits)];
            bool any = false;
            int dmask = 0;
            for (int t = 0; t < TB; t++)
                if (dyn[L.thread_tile_bit(t)]) dmask |= 1 << t;
            // row[tau] = sum of the linear terms of tau's bits and of the pair
            // terms inside tau, built from tau without its lowest bit b: add
            // b's linear term and its pairs with the bits already there
            uint32_t lin_t[kMaxThreadBits] = {}, pair[kMaxThreadBits][kMaxThreadBits] = {};
            for (int t = 0; t < TB; t++) lin_t[t] = sl[L.thread_tile_bit(t)];
            for (auto &p : tt) {
                pair[std::get<0>(p)][std::get<1>(p)] += std::get<2>(p);
                pair[std::get<1>(p)][std::get<0>(p)] += std::get<2>(p);
            }
            row[0] = 0;
            for (int tau = 1; tau < NT; tau++) {
                const int b = __builtin_ctz((unsigned)tau);
                const int prev = tau & (tau - 1);
                uint32_t u = row[prev] + lin_t[b];
                for (int rest = prev; rest; rest &= rest - 1) u += pair[b][__builtin_ctz((unsigned)rest)];
                row[tau] = u;
                any |= u != 0;
            }
            if (any || use_cst || dmask) add_thread_factor(0, use_cst, -1, dmask, row);
        }
        // one factor per register bit with a coefficient
        for (int j = 0; j < RB; j++) {
            const int tb = L.reg[j];
            uint32_t row[1 << (kT2MaxQubits - kT2RegBits)];
            bool any = false;
            row[0] = sl[tb];  // then row[tau] = row[tau without its lowest bit b] + rt[j][b]
            any = row[0] != 0;
            for (int tau = 1; tau < NT; tau++) {
                row[tau] = row[tau & (tau - 1)] + rt[j][__builtin_ctz((unsigned)tau)];
                any |= row[tau] != 0;
            }
            if (any || dyn[tb]) add_thread_factor(1 << j, false, dyn[tb] ? tb : -1, 0, row);
        }
        for (auto &kv : rr) {
            if (!kv.second) continue;
            T2Factor f{};
            f.w0 = kv.first;
            f.run = r;
            const double ang = 2.0 * M_PI * ((double)(int32_t)kv.second * 0x1p-32);
            f.c0 = (float)std::cos(ang);
            f.c1 = (float)std::sin(ang);
            cturn[out->factors.size()] = kv.second;
            out->factors.push_back(f);
        }
        if (fused) {
            // move this run's thread-dependent factors into `pre` (before the
            // block) when they commute with it, else close the block first
            std::vector<T2Factor> fs(out->factors.begin() + nfac0, out->factors.end());
            out->factors.resize(nfac0);
            int jt = 0;
            for (const T2Factor &f : fs) jt |= f.w0 & 0xff;
            if (jt & nd) {
                std::string e = flush();
                if (!e.empty()) return e;
            }
            pre.insert(pre.end(), fs.begin(), fs.end());
            continue;
        }
        in.e1 = (int16_t)out->factors.size();
        if (out->factors.size() > 32000) return "too many factor applications";
        if (in.e1 > in.e0) out->ins.push_back(in);
    }
    if (fused) {
        std::string e = flush();
        if (!e.empty()) return e;
        if (out->factors.size() > 32000) return "too many factor applications";
    }
    for (size_t i = 0; i < out->ins.size(); i++)
        if (out->ins[i].op == T2_STAGE) out->last_stage = (int)i;
    // kernel-side layouts and the write-back offsets of the final layout
    out->layx.resize(out->stages.size());
    for (size_t si = 0; si < out->stages.size(); si++) {
        const T2Stage &st = out->stages[si];
        T2LayoutX &x = out->layx[si];
        for (int v = 0; v < 32; v++) {
            int lo = 0;
            for (int t = 0; t < 5; t++)
                if ((v >> t) & 1) lo += 1 << st.tb[5 + t];
            x.lo[v] = (uint16_t)lo;
        }
        for (int v = 0; v < 16; v++) {
            int hi = 0;
            for (int t = 0; t < NW; t++)
                if ((v >> t) & 1) hi += 1 << st.tb[10 + t];
            x.hi[v] = (uint16_t)hi;
        }
        for (int j = 0; j < 4; j++) x.s[j] = 1 + j < RB ? 1 << st.tb[1 + j] : 0;
    }
    if (out->last_stage >= 0) {
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
        for (int j = 0; j < 4; j++) out->epi.g[j] = 1 + j < RB ? w(st.tb[1 + j]) : 0;
    }
    if (out->n_h || fused || (out->sign_flips & 1)) {  // fused passes always end with a scale
        const double s = std::pow(2.0, -0.5 * out->n_h) * ((out->sign_flips & 1) ? -1.0 : 1.0);
        const float hi = (float)s;
        T2Mat m{};
        m.m[0] = hi;
        m.m[1] = (float)(s - (double)hi);
        T2Ins in{};
        in.op = T2_SCALE;
        in.aux = (int32_t)out->mats.size();
        out->mats.push_back(m);
        out->ins.push_back(in);
    }
    return "";
}

}  // namespace sv
