// Greedy partition planner (host).
//
// Follows Sec. III-B of arxiv 2605.15098:
//  * SWAP gates become relabels of the logical-to-physical qubit map ("the
//    simulator maintains a logical-to-physical qubit mapping that is updated
//    after each SWAP"), so they cost no data movement;
//  * gates are deferred and grouped into passes; every gate of a pass is
//    applied to one tile before the next tile is touched;
//  * only the target of a gate has to be local; a global control is decided
//    per tile from the tile's index;
//  * diagonal gates (P, CP, CZ and their dyadic forms) never need a local
//    qubit: every out-of-tile bit is a constant of the tile.
// Passes are built by list scheduling over the gate dependency graph: two
// gates depend on each other when they share a qubit that at least one of
// them acts on non-diagonally.  A pass takes, in program order, every ready
// gate whose non-diagonal qubits fit in the tile's k slots.
#include <algorithm>
#include <cmath>
#include <string>

#include "common.h"
#include "plan.h"

namespace sv {
namespace {

struct PGate {
    sv_gate g;       // physical qubits
    int nd[2], nnd;  // qubits acted on non-diagonally
    int dq[2], ndq;  // qubits acted on diagonally
    bool diag;
    bool counted;    // a circuit gate (false: a phase split off a U3)
};

void classify(PGate &p) {
    const sv_gate &g = p.g;
    p.nnd = p.ndq = 0;
    p.diag = is_diagonal_kind(g.kind);
    if (g.kind == SV_SWAP) {
        p.nd[p.nnd++] = g.target;
        p.nd[p.nnd++] = g.control;
    } else if (p.diag) {
        p.dq[p.ndq++] = g.target;
        if (is_controlled_kind(g.kind)) p.dq[p.ndq++] = g.control;
    } else {
        p.nd[p.nnd++] = g.target;
        if (is_controlled_kind(g.kind)) p.dq[p.ndq++] = g.control;
    }
}

bool commutes_with_gate(const PGate &d, const PGate &g) {
    // d diagonal; g non-diagonal: they commute unless g acts non-diagonally
    // on one of d's qubits.
    for (int i = 0; i < g.nnd; i++)
        for (int j = 0; j < d.ndq; j++)
            if (g.nd[i] == d.dq[j]) return false;
    return true;
}

// Build one tile pass: the gates pg[order] (dependency order) on the tile
// whose local qubits are the physical bits with in_l set (k of them, the c
// lowest first).  Diagonal gates merge into runs; see build_plan.
std::string emit_pass(const std::vector<PGate> &pg, const std::vector<int> &order,
                      const bool *in_l, int n, int k, int c, const PlanOptions &opt,
                      TilePass *out_pass) {
    TilePass tp;
    tp.k = k;
    tp.c = c;
    tp.ngates = 0;
    for (int i : order) tp.ngates += pg[i].counted ? 1 : 0;
    int slot_of[64];
    for (int q = 0; q < 64; q++) slot_of[q] = -1;
    int s = 0;
    for (int q = 0; q < n; q++)
        if (in_l[q]) {
            tp.slot_phys[s] = q;
            slot_of[q] = s++;
        }
    tp.gmask = 0;
    for (int q = 0; q < n; q++)
        if (!in_l[q]) tp.gmask |= UINT64_C(1) << q;

    // segments: gates in order, diagonal gates merged into runs
    struct Seg {
        bool diag;
        std::vector<int> g;
    };
    // A diagonal gate may move anywhere between the last earlier and the
    // first later non-diagonal gate it does not commute with (diagonal gates
    // commute with each other).  Gap j is the place just before the j-th
    // non-diagonal gate of the pass (gap N: the end).  The fewest runs that
    // hold every diagonal gate is a minimum stabbing of these gap intervals:
    // taken in order of their right ends, an interval not yet stabbed puts a
    // run at its right end, as late as possible, so that a run collects the
    // phases that feed one non-diagonal gate (as the inverse QFT writes them).
    std::vector<int> nd_gates;  // non-diagonal gates of the pass, in order
    struct Win {
        int lo, hi, gate;
    };
    std::vector<Win> wins;
    for (int i : order) {
        const PGate &p = pg[i];
        if (!p.diag) {
            nd_gates.push_back(i);
            continue;
        }
        const int here = (int)nd_gates.size();
        if (!opt.merge_diag) {
            wins.push_back({here, here, i});
            continue;
        }
        int lo = 0;
        for (int j = here - 1; j >= 0; j--)
            if (!commutes_with_gate(p, pg[nd_gates[j]])) {
                lo = j + 1;
                break;
            }
        wins.push_back({lo, -1, i});
    }
    const int N = (int)nd_gates.size();
    if (opt.merge_diag) {
        // right ends: the first later non-commuting non-diagonal gate
        size_t w = 0;
        int here = 0;
        for (int i : order) {
            if (!pg[i].diag) {
                here++;
                continue;
            }
            Win &wi = wins[w++];
            wi.hi = N;
            for (int j = here; j < N; j++)
                if (!commutes_with_gate(pg[i], pg[nd_gates[j]])) {
                    wi.hi = j;
                    break;
                }
        }
    }
    std::vector<std::vector<int>> run_at(N + 1);
    if (!opt.merge_diag) {
        for (const Win &wi : wins) run_at[wi.lo].push_back(wi.gate);
    } else {
        std::vector<int> idx(wins.size());
        for (size_t i = 0; i < idx.size(); i++) idx[i] = (int)i;
        std::stable_sort(idx.begin(), idx.end(),
                         [&](int a, int b) { return wins[a].hi < wins[b].hi; });
        std::vector<char> is_point(N + 1, 0);
        int point = -1;
        for (int i : idx)
            if (wins[i].lo > point) {
                point = wins[i].hi;
                is_point[point] = 1;
            }
        // each gate joins the latest run inside its window, next to the
        // gate it feeds, where its phase terms most often share a factor
        for (const Win &wi : wins) {
            int j = wi.hi;
            while (!is_point[j]) j--;
            run_at[j].push_back(wi.gate);
        }
    }
    std::vector<Seg> segs;
    for (int j = 0; j <= N; j++) {
        if (!run_at[j].empty()) {
            if (opt.merge_diag) {
                segs.push_back({true, run_at[j]});
            } else {
                for (int gi : run_at[j]) segs.push_back({true, {gi}});
            }
        }
        if (j < N) segs.push_back({false, {nd_gates[j]}});
    }

    struct Acc {
        int kind, a, b;
        uint64_t th;
    };
    std::vector<Acc> acc;
    for (const Seg &sg : segs) {
        TileOp op{};
        if (!sg.diag) {
            const sv_gate &g = pg[sg.g[0]].g;
            if (g.kind == SV_SWAP) {
                op.type = TOP_SWAP;
                op.slot = slot_of[g.target];
                op.cslot = slot_of[g.control];
            } else {
                op.slot = slot_of[g.target];
                Mat2 mm = gate_matrix(g);
                for (int e = 0; e < 4; e++) {
                    op.m[2 * e] = mm.re[e];
                    op.m[2 * e + 1] = mm.im[e];
                }
                if (g.kind == SV_CU) {
                    if (slot_of[g.control] >= 0) {
                        op.type = TOP_GATE_CL;
                        op.cslot = slot_of[g.control];
                    } else {
                        op.type = TOP_GATE_CG;
                        op.cbit = g.control;
                    }
                } else if (g.kind == SV_H) {
                    op.type = TOP_H;
                } else if (g.kind == SV_X) {
                    op.type = TOP_X;
                } else {
                    op.type = TOP_GATE;
                }
            }
            tp.ops.push_back(op);
            continue;
        }
        // merged diagonal run -> phase polynomial over local / global bits:
        // one term per (kind, a, b), in that order, its phases summed (exact
        // 64-bit fractions of a turn, so the order of the sum is immaterial)
        acc.clear();
        for (int gi : sg.g) {
            const sv_gate &g = pg[gi].g;
            bool exact;
            uint64_t th = diag_turns64(g, &exact);
            if (!is_controlled_kind(g.kind)) {
                int q = g.target;
                if (slot_of[q] >= 0)
                    acc.push_back({TERM_L, slot_of[q], 0, th});
                else
                    acc.push_back({TERM_G, q, 0, th});
            } else {
                int q1 = g.control, q2 = g.target;
                int s1 = slot_of[q1], s2 = slot_of[q2];
                if (s1 >= 0 && s2 >= 0)
                    acc.push_back({TERM_LL, std::min(s1, s2), std::max(s1, s2), th});
                else if (s1 >= 0)
                    acc.push_back({TERM_LG, s1, q2, th});
                else if (s2 >= 0)
                    acc.push_back({TERM_LG, s2, q1, th});
                else
                    acc.push_back({TERM_GG, std::min(q1, q2), std::max(q1, q2), th});
            }
        }
        std::sort(acc.begin(), acc.end(), [](const Acc &x, const Acc &y) {
            return x.kind != y.kind ? x.kind < y.kind : x.a != y.a ? x.a < y.a : x.b < y.b;
        });
        op.type = TOP_DIAG;
        op.tb = (int)tp.terms.size();
        for (size_t i = 0; i < acc.size();) {
            PhaseTerm t{};
            t.kind = acc[i].kind;
            t.a = acc[i].a;
            t.b = acc[i].b;
            t.theta = 0;
            for (; i < acc.size() && acc[i].kind == t.kind && acc[i].a == t.a && acc[i].b == t.b; i++)
                t.theta += acc[i].th;
            if (t.theta != 0) tp.terms.push_back(t);
        }
        op.te = (int)tp.terms.size();
        if (op.te > op.tb) tp.ops.push_back(op);
    }
    *out_pass = std::move(tp);
    return "";
}

// Sec. III-B as the paper states it.  The local qubits are the physical bits
// 0..k-1, so a tile is one contiguous block of 2^k amplitudes.  Gates are
// deferred in program order; a gate whose target (both qubits for a SWAP
// executed as data) is global ends the deferred batch, which becomes one
// pass, and a remap exchanges that global bit with the local bit that was
// used least recently (ties: the lowest bit), updating the logical-to-physical
// map.  A global control needs no remap: it is decided per tile.
std::string build_plan_paper(const std::vector<sv_gate> &gates, const std::vector<char> &counted,
                             const PlanOptions &opt, int *phys,
                             Plan *out) {
    const int n = opt.n;
    const int k = std::min(opt.k, n);
    int inv[64];
    for (int q = 0; q < 64; q++) inv[q] = -1;
    for (int q = 0; q < n; q++) inv[phys[q]] = q;
    std::vector<long> lru(k, -1);
    long clock = 0;
    bool in_l[64] = {};
    for (int q = 0; q < k; q++) in_l[q] = true;
    std::vector<PGate> pending;
    std::vector<std::pair<int, int>> remaps;
    auto flush = [&]() -> std::string {
        if (pending.empty()) return "";
        std::vector<int> order(pending.size());
        for (size_t i = 0; i < order.size(); i++) order[i] = (int)i;
        TilePass tp;
        std::string e = emit_pass(pending, order, in_l, n, k, k, opt, &tp);
        if (!e.empty()) return e;
        tp.remap_before.swap(remaps);
        remaps.clear();
        out->passes.push_back(std::move(tp));
        pending.clear();
        return "";
    };
    for (size_t gi = 0; gi < gates.size(); gi++) {
        const sv_gate &g = gates[gi];
        if (g.kind == SV_SWAP && opt.relabel) {
            std::swap(phys[g.target], phys[g.control]);
            inv[phys[g.target]] = g.target;
            inv[phys[g.control]] = g.control;
            out->relabels++;
            continue;
        }
        int need[2], nneed = 0;
        need[nneed++] = g.target;
        if (g.kind == SV_SWAP) need[nneed++] = g.control;
        for (int a = 0; a < nneed; a++) {
            const int t = phys[need[a]];
            if (t < k) continue;
            std::string e = flush();
            if (!e.empty()) return e;
            // victim: least recently used local bit the gate does not use
            int v = -1;
            for (int p = 0; p < k; p++) {
                bool used = false;
                for (int b = 0; b < nneed; b++) used |= phys[need[b]] == p;
                if (is_controlled_kind(g.kind) && phys[g.control] == p) used = true;
                if (used) continue;
                if (v < 0 || lru[p] < lru[v]) v = p;
            }
            if (v < 0) return "tile too small for a remap";
            const int lq = inv[v], gq = inv[t];
            phys[lq] = t;
            phys[gq] = v;
            inv[v] = gq;
            inv[t] = lq;
            remaps.push_back({v, t});
            out->remaps++;
        }
        PGate p{};
        p.counted = counted[gi] != 0;
        p.g = g;
        p.g.target = phys[g.target];
        if (is_controlled_kind(g.kind) || g.kind == SV_SWAP) p.g.control = phys[g.control];
        classify(p);
        pending.push_back(p);
        const long now = clock++;
        if (p.g.target < k) lru[p.g.target] = now;
        if ((is_controlled_kind(g.kind) || g.kind == SV_SWAP) && p.g.control < k)
            lru[p.g.control] = now;
    }
    return flush();
}

}  // namespace

PlanOptions plan_options(int n, sv_dtype dt, const sv_config &cfg) {
    PlanOptions opt;
    opt.n = n;
    const bool dbl = dt == SV_C128;
    // complex128 defaults to the FP64 register-stage kernel's 2^13 tiles
    opt.k = cfg.tile_qubits ? cfg.tile_qubits : 13;
    opt.c = cfg.chunk_qubits ? cfg.chunk_qubits : 5;
    if (!dbl && opt.c < 1) opt.c = 1;
    opt.merge_diag = !(cfg.flags & SV_FLAG_NO_DIAG_MERGE);
    opt.relabel = !(cfg.flags & SV_FLAG_NO_RELABEL);
    opt.paper = (cfg.flags & SV_FLAG_PAPER_SWAP) != 0;
    opt.late_diag = !(cfg.flags & SV_FLAG_EARLY_DIAG);
    opt.search = !(cfg.flags & SV_FLAG_GREEDY_ONLY);
    if (opt.paper) opt.c = opt.k;  // the block is contiguous
    if ((cfg.flags & SV_FLAG_NARROW_FIRST) && !opt.paper) opt.first_c = 4;
    opt.split_u3 = !dbl;
    return opt;
}

namespace {

// Local-qubit search of one pass: hill-climbing steps, and how many blocked
// outside qubits (those of the earliest gates only locality holds back) a
// step tries to bring in.
constexpr int kSearchSteps = 16;
constexpr int kSearchWant = 32;

// U3(theta, phi, lambda) = P(phi) RY(theta) P(lambda) exactly, with
// RY(theta) = [[cos(theta/2), -sin(theta/2)], [sin(theta/2), cos(theta/2)]]
// (multiply out the definition of U3 in sv.h).  The two phases are diagonal
// gates that merge into the neighbouring diagonal runs, and the rotation is
// a real matrix, half the arithmetic of a general complex 2x2.
// counted[i] is 0 for the phases, which are not gates of the circuit.
std::vector<sv_gate> split_u3(const std::vector<sv_gate> &gates, std::vector<char> *counted) {
    std::vector<sv_gate> out;
    out.reserve(gates.size() + gates.size() / 2);
    counted->clear();
    for (const sv_gate &g : gates) {
        if (g.kind != SV_U3) {
            out.push_back(g);
            counted->push_back(1);
            continue;
        }
        const double c = std::cos(0.5 * g.p[0]), s = std::sin(0.5 * g.p[0]);
        sv_gate p{};
        p.kind = SV_P;
        p.target = g.target;
        p.p[0] = g.p[2];
        if (p.p[0] != 0.0) {
            out.push_back(p);
            counted->push_back(0);
        }
        sv_gate ry{};
        ry.kind = SV_U;
        ry.target = g.target;
        ry.p[0] = c;
        ry.p[2] = -s;
        ry.p[4] = s;
        ry.p[6] = c;
        out.push_back(ry);
        counted->push_back(1);
        p.p[0] = g.p[1];
        if (p.p[0] != 0.0) {
            out.push_back(p);
            counted->push_back(0);
        }
    }
    return out;
}

}  // namespace

static std::string build_plan_once(const std::vector<sv_gate> &gates_in, const PlanOptions &opt,
                                   int *phys, Plan *out) {
    const int n = opt.n;
    out->passes.clear();
    out->relabels = 0;
    out->remaps = 0;
    std::vector<sv_gate> split;
    std::vector<char> counted(gates_in.size(), 1);
    if (opt.split_u3) split = split_u3(gates_in, &counted);
    const std::vector<sv_gate> &gates = opt.split_u3 ? split : gates_in;
    if (opt.paper && n > opt.k) return build_plan_paper(gates, counted, opt, phys, out);
    int k = std::min(opt.k, n);
    int c = std::min(opt.c, k);
    if (n > k && k - c < 2) return "tile must leave at least two free slots (k - c >= 2)";

    // 1. physical gate list, SWAPs absorbed into the map
    std::vector<PGate> pg;
    pg.reserve(gates.size());
    for (size_t gi = 0; gi < gates.size(); gi++) {
        const sv_gate &g = gates[gi];
        if (g.kind == SV_SWAP && opt.relabel) {
            std::swap(phys[g.target], phys[g.control]);
            out->relabels++;
            continue;
        }
        PGate p{};
        p.counted = counted[gi] != 0;
        p.g = g;
        p.g.target = phys[g.target];
        if (is_controlled_kind(g.kind) || g.kind == SV_SWAP) p.g.control = phys[g.control];
        classify(p);
        pg.push_back(p);
    }
    const int m = (int)pg.size();

    // 2. dependencies, gate i's in dep_idx[dep_off[i] .. dep_off[i + 1])
    std::vector<int> last_nd(64, -1);
    std::vector<std::vector<int>> diag_since(64);
    for (int q = 0; q < n; q++) diag_since[q].reserve(16);
    std::vector<int> dep_off(m + 1, 0), dep_idx;
    dep_idx.reserve(4 * (size_t)m);
    for (int i = 0; i < m; i++) {
        PGate &p = pg[i];
        dep_off[i] = (int)dep_idx.size();
        for (int a = 0; a < p.nnd; a++) {
            int q = p.nd[a];
            if (last_nd[q] >= 0) dep_idx.push_back(last_nd[q]);
            for (int d : diag_since[q]) dep_idx.push_back(d);
        }
        for (int a = 0; a < p.ndq; a++) {
            int q = p.dq[a];
            if (last_nd[q] >= 0) dep_idx.push_back(last_nd[q]);
        }
        for (int a = 0; a < p.nnd; a++) {
            last_nd[p.nd[a]] = i;
            diag_since[p.nd[a]].clear();
        }
        for (int a = 0; a < p.ndq; a++) diag_since[p.dq[a]].push_back(i);
    }
    dep_off[m] = (int)dep_idx.size();

    // 3. passes by list scheduling.  A gate left out of a pass blocks its
    // non-diagonal qubits: every later gate on one of them depends on it.
    // Once every qubit is blocked no later gate can run, and a scan stops.
    const uint64_t all_q = n >= 64 ? ~UINT64_C(0) : (UINT64_C(1) << n) - 1;
    auto nd_mask = [&](const PGate &p) {
        uint64_t b = 0;
        for (int a = 0; a < p.nnd; a++) b |= UINT64_C(1) << p.nd[a];
        return b;
    };
    std::vector<char> done(m, 0);
    auto deps_done = [&](int i) {
        for (int e = dep_off[i]; e < dep_off[i + 1]; e++)
            if (!done[dep_idx[e]]) return false;
        return true;
    };
    std::vector<int> pass_c;  // chunk qubits of each pass
    std::vector<std::vector<int>> orders;
    std::vector<std::vector<char>> locals;
    std::vector<int> taken, rem;
    taken.reserve((size_t)m);
    rem.reserve((size_t)m);
    int remaining = m;
    while (remaining > 0) {
        bool in_l[64] = {};
        int cnt = 0;
        if (n <= k) {
            for (int q = 0; q < n; q++) in_l[q] = true;
            cnt = n;
        }
        // the first pass may gather narrower chunks (SV_FLAG_NARROW_FIRST)
        const int cc = (orders.empty() && opt.first_c > 0) ? std::min(opt.first_c, c) : c;
        if (n > k) {
            for (int q = 0; q < cc; q++) in_l[q] = true;
            cnt = cc;
        }
        std::vector<int> order;
        order.reserve((size_t)remaining);
        uint64_t blocked = 0;
        for (int i = 0; i < m && blocked != all_q; i++) {
            if (done[i]) continue;
            const PGate &p = pg[i];
            if (!deps_done(i)) {
                blocked |= nd_mask(p);
                continue;
            }
            int need = 0;
            for (int a = 0; a < p.nnd; a++) need += !in_l[p.nd[a]];
            if (cnt + need > k) {
                blocked |= nd_mask(p);
                continue;
            }
            for (int a = 0; a < p.nnd; a++)
                if (!in_l[p.nd[a]]) {
                    in_l[p.nd[a]] = true;
                    cnt++;
                }
            order.push_back(i);
            done[i] = 1;
            remaining--;
        }
        if (order.empty()) return "internal: planner made no progress";
        if (opt.search && n > k) {
            // The greedy set is the qubits of the earliest ready gates.  Refine
            // it by hill climbing: swap one of its free qubits for an outside
            // one (or add one while a slot is free) when the pass then runs
            // more gates, with the set fixed and the gates taken in list order.
            for (int i : order) done[i] = 0;
            rem.clear();
            for (int i = 0; i < m; i++)
                if (!done[i]) rem.push_back(i);
            // Gates run in list order with the set fixed; `want` collects the
            // outside qubits of the earliest gates that only locality blocks.
            auto run_pass = [&](const bool *S, std::vector<int> *ord, std::vector<int> *want) {
                taken.clear();
                int cntg = 0;
                uint64_t blk = 0;
                for (size_t r = 0; r < rem.size() && blk != all_q; r++) {
                    const int i = rem[r];
                    const PGate &p = pg[i];
                    bool ok = deps_done(i);
                    if (!ok) {
                        blk |= nd_mask(p);
                        continue;
                    }
                    for (int a = 0; ok && a < p.nnd; a++) ok = S[p.nd[a]];
                    if (!ok) {
                        blk |= nd_mask(p);
                        if (want && (int)want->size() < kSearchWant)
                            for (int a = 0; a < p.nnd; a++)
                                if (!S[p.nd[a]] &&
                                    std::find(want->begin(), want->end(), p.nd[a]) == want->end())
                                    want->push_back(p.nd[a]);
                        continue;
                    }
                    done[i] = 1;
                    taken.push_back(i);
                    cntg++;
                }
                for (int i : taken) done[i] = 0;
                if (ord) *ord = taken;
                return cntg;
            };
            bool S[64];
            for (int q = 0; q < 64; q++) S[q] = in_l[q];
            std::vector<int> want;
            want.reserve(kSearchWant);
            int best = run_pass(S, nullptr, &want);
            for (int it = 0; it < kSearchSteps && !want.empty(); it++) {
                int bv = best, bin = -1, bout = -1;
                for (int qo : want) {
                    S[qo] = true;
                    if (cnt < k) {  // a free slot: try adding qo
                        const int v = run_pass(S, nullptr, nullptr);
                        if (v > bv) {
                            bv = v;
                            bin = -1;
                            bout = qo;
                        }
                    }
                    for (int qi = cc; qi < n; qi++) {
                        if (!S[qi] || qi == qo) continue;
                        S[qi] = false;
                        const int v = run_pass(S, nullptr, nullptr);
                        S[qi] = true;
                        if (v > bv) {
                            bv = v;
                            bin = qi;
                            bout = qo;
                        }
                    }
                    S[qo] = false;
                }
                if (bout < 0) break;
                S[bout] = true;
                if (bin >= 0)
                    S[bin] = false;
                else
                    cnt++;
                want.clear();
                best = run_pass(S, nullptr, &want);
            }
            order.clear();
            run_pass(S, &order, nullptr);
            for (int i : order) done[i] = 1;
            for (int q = 0; q < 64; q++) in_l[q] = S[q];
            remaining = 0;
            for (int i = 0; i < m; i++) remaining += !done[i];
        }
        // fill unused slots with the lowest free bits (longer contiguous runs)
        for (int q = 0; q < n && cnt < k; q++)
            if (!in_l[q]) {
                in_l[q] = true;
                cnt++;
            }

        pass_c.push_back(cc);
        orders.push_back(std::move(order));
        locals.emplace_back(in_l, in_l + 64);
    }

    // 4. A diagonal gate is ready as soon as the gates before it on its
    // qubits are done, but it only has to run before the next gate that acts
    // non-diagonally on one of them.  It moves to the pass of its first such
    // successor, at the front of that pass's order: there its phase terms
    // join the run that feeds that gate instead of forming a run at the end
    // of an earlier pass.  Gates without a successor stay where they are.
    std::vector<int> pass_of(m, 0);
    for (size_t p = 0; p < orders.size(); p++)
        for (int i : orders[p]) pass_of[i] = (int)p;
    std::vector<int> first_succ(m, -1);
    for (int j = 0; j < m; j++)
        for (int e = dep_off[j]; e < dep_off[j + 1]; e++) {
            const int d = dep_idx[e];
            if (first_succ[d] < 0 || pass_of[j] < first_succ[d]) first_succ[d] = pass_of[j];
        }
    if (opt.merge_diag && opt.late_diag) {
        std::vector<std::vector<int>> moved(orders.size());
        for (size_t p = 0; p < orders.size(); p++) {
            std::vector<int> keep;
            keep.reserve(orders[p].size());
            for (int i : orders[p]) {
                if (pg[i].diag && first_succ[i] > (int)p)
                    moved[first_succ[i]].push_back(i);
                else
                    keep.push_back(i);
            }
            orders[p].swap(keep);
        }
        for (size_t p = 0; p < orders.size(); p++)
            if (!moved[p].empty()) orders[p].insert(orders[p].begin(), moved[p].begin(), moved[p].end());
    }
    for (size_t p = 0; p < orders.size(); p++) {
        if (orders[p].empty()) continue;
        bool in_l[64];
        for (int q = 0; q < 64; q++) in_l[q] = locals[p][q] != 0;
        TilePass tp;
        std::string e = emit_pass(pg, orders[p], in_l, n, k, pass_c[p], opt, &tp);
        if (!e.empty()) return e;
        out->passes.push_back(std::move(tp));
    }
    return "";
}

// The local search makes each pass run at least the gates the greedy
// scheduling puts there, but a fuller pass can leave a remainder that needs
// more passes.  The greedy plan is built as well (a small fraction of the
// search's cost) and kept when it has strictly fewer passes.
static std::string build_plan_segment(const std::vector<sv_gate> &gates, const PlanOptions &opt, int *phys,
                                      Plan *out) {
    if (!opt.search || opt.paper || opt.n <= opt.k) return build_plan_once(gates, opt, phys, out);
    int phys_g[64];
    std::copy(phys, phys + 64, phys_g);
    std::string err = build_plan_once(gates, opt, phys, out);
    if (!err.empty()) return err;
    PlanOptions og = opt;
    og.search = false;
    Plan greedy;
    if (build_plan_once(gates, og, phys_g, &greedy).empty() &&
        greedy.passes.size() < out->passes.size()) {
        *out = std::move(greedy);
        std::copy(phys_g, phys_g + 64, phys);
    }
    return "";
}

std::string build_plan(const std::vector<sv_gate> &gates, const PlanOptions &opt, int *phys,
                       Plan *out) {
    bool general = false;
    for (const sv_gate &g : gates) general |= is_general_kind(g.kind);
    if (!general) return build_plan_segment(gates, opt, phys, out);
    out->passes.clear();
    out->relabels = 0;
    out->remaps = 0;
    size_t i = 0;
    for (;;) {
        size_t j = i;
        while (j < gates.size() && !is_general_kind(gates[j].kind)) j++;
        if (j > i) {
            std::vector<sv_gate> seg(gates.begin() + (long)i, gates.begin() + (long)j);
            Plan sp;
            PlanOptions os = opt;  // only the list's first pass may be narrow
            if (!out->passes.empty()) os.first_c = 0;
            const std::string err = build_plan_segment(seg, os, phys, &sp);
            if (!err.empty()) return err;
            for (TilePass &tp : sp.passes) out->passes.push_back(std::move(tp));
            out->relabels += sp.relabels;
            out->remaps += sp.remaps;
        }
        if (j == gates.size()) break;
        const int nr = general_records(gates[j].kind);
        TilePass step;
        step.ngates = nr;
        for (int r = 0; r < nr; r++) {
            sv_gate g = gates[j + r];
            g.target = phys[g.target];
            if (g.control >= 0) g.control = phys[g.control];
            if (g.kind == SV_MCU) {
                uint64_t pm = 0;
                for (int q = 0; q < opt.n; q++)
                    if (((uint64_t)g.num >> q) & 1) pm |= UINT64_C(1) << phys[q];
                g.num = (int64_t)pm;
            }
            step.general.push_back(g);
        }
        out->passes.push_back(std::move(step));
        i = j + nr;
    }
    return "";
}

}  // namespace sv
