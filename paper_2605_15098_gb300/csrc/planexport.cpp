// sv_plan_export: the programme the partitioned path would run, as JSON.
// Host only (no CUDA call), for inspection and for host-side tests that
// execute the exported programme and compare it with the oracle.
#include <cinttypes>
#include <cstdio>
#include <cstring>
#include <string>

#include "common.h"
#include "plan.h"
#include "stagecomp.h"

namespace sv {
namespace {

struct J {
    std::string s;
    void raw(const char *t) { s += t; }
    void num(long long v) { s += std::to_string(v); }
    void u64(uint64_t v) { s += std::to_string(v); }
    void dbl(double v) {
        char b[40];
        snprintf(b, sizeof b, "%.17g", v);
        s += b;
    }
    template <typename T>
    void arr(const T *p, int n) {
        s += "[";
        for (int i = 0; i < n; i++) {
            if (i) s += ",";
            s += std::to_string(p[i]);
        }
        s += "]";
    }
};

void put_t2(J &j, const T2Pass &t) {
    j.raw("{\"ins\":[");
    for (size_t i = 0; i < t.ins.size(); i++) {
        const T2Ins &in = t.ins[i];
        if (i) j.raw(",");
        j.raw("{\"op\":"); j.num(in.op);
        j.raw(",\"cls\":"); j.num(in.cls);
        j.raw(",\"idx\":"); j.num(in.idx);
        j.raw(",\"ccls\":"); j.num(in.ccls);
        j.raw(",\"cidx\":"); j.num(in.cidx);
        j.raw(",\"e0\":"); j.num(in.e0);
        j.raw(",\"e1\":"); j.num(in.e1);
        j.raw(",\"aux\":"); j.num(in.aux);
        j.raw("}");
    }
    j.raw("],\"rb\":"); j.num(t.rb);
    j.raw(",\"threads\":"); j.num(t.threads);
    j.raw(",\"stages\":[");
    for (size_t i = 0; i < t.stages.size(); i++) {
        if (i) j.raw(",");
        int tb[14];
        for (int e = 0; e < 14; e++) tb[e] = t.stages[i].tb[e];
        j.arr(tb, 14);
    }
    // matrix records: FP32 (complex64 programmes) or FP64 (complex128), 8 values each
    j.raw("],\"mats\":[");
    const size_t nm = t.mats.empty() ? t.mats64.size() / 8 : t.mats.size();
    for (size_t i = 0; i < nm; i++) {
        if (i) j.raw(",");
        j.raw("[");
        for (int e = 0; e < 8; e++) {
            if (e) j.raw(",");
            j.dbl(t.mats.empty() ? t.mats64[8 * i + e] : (double)t.mats[i].m[e]);
        }
        j.raw("]");
    }
    j.raw("],\"factors\":[");
    for (size_t i = 0; i < t.factors.size(); i++) {
        const T2Factor &f = t.factors[i];
        uint32_t w0;
        std::memcpy(&w0, &f.w0, sizeof w0);
        int32_t row;
        std::memcpy(&row, &f.c0, sizeof row);
        if (i) j.raw(",");
        j.raw("{\"w0\":"); j.u64(w0);
        j.raw(",\"run\":"); j.num(f.run);
        j.raw(",\"row\":"); j.num(row);
        j.raw(",\"c\":["); j.dbl(f.c0); j.raw(","); j.dbl(f.c1); j.raw("]}");
    }
    j.raw("],\"stat\":");
    j.arr(t.stat.data(), (int)t.stat.size());
    j.raw(",\"format\":"); j.num(t.format);
    j.raw(",\"gen_hmask\":"); j.num(t.gen_hmask);
    j.raw(",\"gen_scale\":"); j.dbl(t.gen_scale);
    j.raw(",\"fac2\":[");
    for (size_t i = 0; i < t.fac2.size(); i++) {
        const T2Fac &f = t.fac2[i];
        if (i) j.raw(",");
        j.raw("{\"w0\":"); j.u64(f.w0);
        j.raw(",\"slot\":"); j.num(f.slot);
        j.raw(",\"dslot\":"); j.num(f.dslot);
        j.raw(",\"row\":"); j.num(f.row);
        j.raw("}");
    }
    j.raw("],\"statc\":[");
    const size_t ns = t.statc.empty() ? t.statc64.size() : t.statc.size();
    for (size_t i = 0; i < ns; i++) {
        if (i) j.raw(",");
        j.dbl(t.statc.empty() ? t.statc64[i] : (double)t.statc[i]);
    }
    j.raw("],\"slots\":[");
    for (size_t i = 0; i < t.slots.size(); i++) {
        if (i) j.raw(",");
        j.raw("["); j.num(t.slots[i].i0); j.raw(","); j.num(t.slots[i].i1); j.raw("]");
    }
    j.raw("]");
    j.raw(",\"tterms\":[");
    for (size_t i = 0; i < t.tterms.size(); i++) {
        const T2TileTerm &tt = t.tterms[i];
        if (i) j.raw(",");
        j.raw("["); j.num(tt.run); j.raw(","); j.num(tt.tb); j.raw(","); j.num(tt.g0); j.raw(",");
        j.num(tt.g1); j.raw(","); j.u64(tt.theta); j.raw("]");
    }
    j.raw("],\"blocks\":[");
    for (int b = 0; b < t.nblocks; b++) {
        if (b) j.raw(",");
        j.raw("[");
        for (int e = 0; e < 2048; e++) {
            if (e) j.raw(",");
            j.dbl(t.blocks64[(size_t)b * 2048 + e]);
        }
        j.raw("]");
    }
    j.raw("],\"nruns\":"); j.num(t.nruns);
    j.raw(",\"n_h\":"); j.num(t.n_h);
    j.raw("}");
}

}  // namespace
}  // namespace sv

using namespace sv;

extern "C" sv_status sv_plan_export(int n, sv_dtype dt, const int *host_phys_of_logical,
                                    const sv_gate *host_gates, size_t m, const sv_config *cfg,
                                    char *host_buf, size_t cap, size_t *len) {
    clear_error();
    if (!len || (cap && !host_buf) || (m && !host_gates)) return fail(SV_ERR_ARG, "NULL argument");
    if (n < 1 || n > 34) return fail(SV_ERR_ARG, "n=%d outside 1..34", n);
    if (dt != SV_C64 && dt != SV_C128) return fail(SV_ERR_ARG, "unknown dtype %d", (int)dt);
    {
        const std::string why = check_list(n, host_gates, m);
        if (!why.empty()) return fail(SV_ERR_ARG, "%s", why.c_str());
    }
    sv_config c{};
    if (cfg) c = *cfg;
    const bool dbl = dt == SV_C128;
    PlanOptions opt = plan_options(n, dt, c);
    int phys[64];
    for (int q = 0; q < 64; q++) phys[q] = q;
    if (host_phys_of_logical)
        for (int q = 0; q < n; q++) phys[q] = host_phys_of_logical[q];
    Plan plan;
    std::vector<sv_gate> gl(host_gates, host_gates + m);
    std::string err = build_plan(gl, opt, phys, &plan);
    if (!err.empty()) return fail(SV_ERR_ARG, "planner: %s", err.c_str());
    const bool allow_t2 = !dbl && !(c.flags & SV_FLAG_GENERIC_TILE);
    J j;
    j.raw("{\"n\":"); j.num(n);
    j.raw(",\"relabels\":"); j.num(plan.relabels);
    j.raw(",\"remaps\":"); j.num(plan.remaps);
    j.raw(",\"phys\":"); j.arr(phys, n);
    j.raw(",\"passes\":[");
    bool first = true, first_pass = true;
    std::vector<char> eligible;  // register-stage, format 2, 2^13 tiles: may join an L2 block group
    for (const TilePass &p : plan.passes) {
        eligible.push_back(0);
        if (!first) j.raw(",");
        first = false;
        const bool first_ops = first_pass && !p.ops.empty() && p.remap_before.empty();
        if (!p.ops.empty() || !p.general.empty()) first_pass = false;
        j.raw("{\"k\":"); j.num(p.k);
        j.raw(",\"c\":"); j.num(p.c);
        j.raw(",\"ngates\":"); j.num(p.ngates);
        j.raw(",\"gmask\":"); j.u64(p.gmask);
        j.raw(",\"slot_phys\":"); j.arr(p.slot_phys, p.k);
        j.raw(",\"remap_before\":[");
        for (size_t i = 0; i < p.remap_before.size(); i++) {
            if (i) j.raw(",");
            j.raw("["); j.num(p.remap_before[i].first); j.raw(",");
            j.num(p.remap_before[i].second); j.raw("]");
        }
        j.raw("]");
        j.raw(",\"ops\":[");
        for (size_t i = 0; i < p.ops.size(); i++) {
            const TileOp &op = p.ops[i];
            if (i) j.raw(",");
            j.raw("{\"type\":"); j.num(op.type);
            j.raw(",\"slot\":"); j.num(op.slot);
            j.raw(",\"cslot\":"); j.num(op.cslot);
            j.raw(",\"cbit\":"); j.num(op.cbit);
            j.raw(",\"tb\":"); j.num(op.tb);
            j.raw(",\"te\":"); j.num(op.te);
            j.raw(",\"m\":[");
            for (int e = 0; e < 8; e++) {
                if (e) j.raw(",");
                j.dbl(op.m[e]);
            }
            j.raw("]}");
        }
        j.raw("],\"terms\":[");
        for (size_t i = 0; i < p.terms.size(); i++) {
            if (i) j.raw(",");
            j.raw("["); j.num(p.terms[i].kind); j.raw(","); j.num(p.terms[i].a); j.raw(",");
            j.num(p.terms[i].b); j.raw(","); j.u64(p.terms[i].theta); j.raw("]");
        }
        j.raw("]");
        if (!p.general.empty()) {  // a gate of the general set, run on the per-gate path
            j.raw(",\"kernel\":\"pergate\",\"general\":[");
            for (size_t r = 0; r < p.general.size(); r++) {
                const sv_gate &g = p.general[r];
                if (r) j.raw(",");
                j.raw("{\"kind\":"); j.num(g.kind);
                j.raw(",\"target\":"); j.num(g.target);
                j.raw(",\"control\":"); j.num(g.control);
                j.raw(",\"num\":"); j.u64((uint64_t)g.num);
                j.raw(",\"p\":[");
                for (int e = 0; e < 8; e++) {
                    if (e) j.raw(",");
                    j.dbl(g.p[e]);
                }
                j.raw("]}");
            }
            j.raw("]}");
            continue;
        }
        T2Pass t2;
        const bool fused = c.mode == SV_MODE_FUSED;
        std::string why = "disabled";
        const char *kname = "t2";
        if (allow_t2 && !p.ops.empty()) {
            why = fused ? compile_t2(p, &t2, true) : "not fused";
            kname = "t3";
            if (!why.empty()) {
                if (fused) {
                    j.raw(",\"fused_why\":\"");
                    j.raw(why.c_str());
                    j.raw("\"");
                }
                why = compile_t2(p, &t2, false);
                kname = "t2";
            }
        }
        if (dbl && !(c.flags & SV_FLAG_GENERIC_TILE) && p.k == kT2Qubits && !p.ops.empty()) {
            // complex128 on 2^13-amplitude tiles: the FP64 register-stage kernel
            // (its programme is the emulator's business only through the ops)
            why = compile_t2v2_c128(p, &t2, false);
            if (why.empty()) {
                j.raw(",\"kernel\":\"t2d\",\"t2d\":");
                put_t2(j, t2);
                if (first_ops) {
                    T2Pass g;
                    if (compile_t2v2_c128(p, &g, true).empty()) {
                        j.raw(",\"t2dgen\":");
                        put_t2(j, g);
                    }
                }
                j.raw("}");
                continue;
            }
        }
        if (why.empty()) {
            eligible.back() = t2.format == 2 && p.k == kT2Qubits;
            j.raw(",\"kernel\":\"");
            j.raw(kname);
            j.raw("\",\"t2\":");
            put_t2(j, t2);
            // the variant the first pass runs when it starts from a recorded basis state
            if (t2.format == 2 && first_ops) {
                T2Pass g;
                if (compile_t2v2(p, &g, true).empty()) {
                    j.raw(",\"t2gen\":");
                    put_t2(j, g);
                }
            }
        } else {
            j.raw(",\"kernel\":\"generic\",\"why\":\"");
            j.raw(why.c_str());
            j.raw("\"");
        }
        j.raw("}");
    }
    j.raw("]");
    if ((c.flags & SV_FLAG_L2_BLOCKS) && !dbl) {
        // the groups of two-level blocking, for GB300's defaults: a 126 MiB
        // L2 (unless l2_qubits is given) and 2 x 152 resident CTAs
        const int cap = c.l2_qubits ? c.l2_qubits : l2_default_qubits((size_t)126 << 20, 8);
        std::vector<L2Group> groups;
        err = form_l2_groups(plan, eligible, n, kT2Qubits, cap, 2 * 152, c.l2_chunk ? c.l2_chunk : 2, &groups);
        if (!err.empty()) return fail(SV_ERR_ARG, "L2 blocks: %s", err.c_str());
        j.raw(",\"l2_groups\":[");
        for (size_t g = 0; g < groups.size(); g++) {
            if (g) j.raw(",");
            j.raw("{\"first\":"); j.num(groups[g].first);
            j.raw(",\"count\":"); j.num(groups[g].count);
            j.raw(",\"l\":"); j.num(groups[g].l);
            j.raw(",\"bmask\":"); j.u64(groups[g].bmask);
            j.raw(",\"lag\":"); j.num(groups[g].lag);
            j.raw(",\"chunk\":"); j.num(1 << groups[g].chunk_log);
            j.raw(",\"segs\":"); j.arr(groups[g].segs.data(), (int)groups[g].segs.size());
            j.raw("}");
        }
        j.raw("]");
    }
    j.raw("}");
    *len = j.s.size();
    if (cap) {
        size_t k = std::min(cap - 1, j.s.size());
        std::memcpy(host_buf, j.s.data(), k);
        host_buf[k] = 0;
    }
    return SV_OK;
}
