// Host-side gate validation and FP64 gate matrices.
//
// Matrices follow the definitions in include/sv.h; the phase gate is Eq. 2 of
// arxiv 2605.15098 (P(phi) = diag(1, e^{i phi})) and its powers Eq. 3
// (U^a = P(2 pi 2^-n a)), which SV_PK / SV_CPK carry as an exact dyadic
// fraction of a turn.
#include <cmath>
#include <cstdarg>
#include <cstdio>

#include "common.h"

namespace sv {

static thread_local std::string g_last_error;

sv_status fail(sv_status code, const char *fmt, ...) {
    char buf[1024];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return code;
}

void clear_error() { g_last_error.clear(); }

const char *last_error_cstr() { return g_last_error.c_str(); }

bool is_diagonal_kind(int kind) {
    return kind == SV_P || kind == SV_CP || kind == SV_CZ || kind == SV_PK || kind == SV_CPK;
}

bool is_controlled_kind(int kind) {
    return kind == SV_CP || kind == SV_CZ || kind == SV_CU || kind == SV_CPK;
}

std::string check_gate(int n, const sv_gate &g) {
    char buf[160];
    if (g.kind < SV_X || g.kind > SV_MEASURE) {
        snprintf(buf, sizeof buf, "unknown gate kind %d", g.kind);
        return buf;
    }
    if (g.target < 0 || g.target >= n) {
        snprintf(buf, sizeof buf, "target %d outside 0..%d", g.target, n - 1);
        return buf;
    }
    if (is_controlled_kind(g.kind) || g.kind == SV_SWAP || g.kind == SV_U2Q || g.kind == SV_MAT) {
        if (g.control < 0 || g.control >= n) {
            snprintf(buf, sizeof buf, "second qubit %d outside 0..%d", g.control, n - 1);
            return buf;
        }
        if (g.control == g.target) return "control (or second SWAP qubit) equals target";
    }
    if (g.reserved != 0) return "reserved field must be 0";
    if ((g.kind == SV_PK || g.kind == SV_CPK) && (g.log2den < 0 || g.log2den > 62)) {
        snprintf(buf, sizeof buf, "log2den %d outside 0..62", g.log2den);
        return buf;
    }
    for (int i = 0; i < 8; i++)
        if (!std::isfinite(g.p[i])) return "non-finite parameter";
    if (g.kind == SV_MCU) {
        const uint64_t cm = (uint64_t)g.num;
        if (!cm) return "MCU control mask is empty";
        if (n < 64 && (cm >> n)) return "MCU control mask has qubits beyond n";
        if ((cm >> g.target) & 1) return "MCU control mask holds the target";
    }
    if (g.kind == SV_MEASURE && !(g.p[0] >= 0.0 && g.p[0] < 1.0)) return "MEASURE u outside [0, 1)";
    return "";
}

std::string check_list(int n, const sv_gate *g, size_t m) {
    char buf[200];
    for (size_t i = 0; i < m; i++) {
        std::string why = check_gate(n, g[i]);
        if (why.empty() && g[i].kind == SV_MAT) why = "a MAT row outside a U2Q";
        if (why.empty() && g[i].kind == SV_U2Q) {
            for (size_t r = 1; r <= 3 && why.empty(); r++)
                if (i + r >= m || g[i + r].kind != SV_MAT || g[i + r].target != g[i].target ||
                    g[i + r].control != g[i].control)
                    why = "a U2Q must be followed by three MAT rows on the same qubits";
            if (why.empty())
                for (size_t r = 1; r <= 3 && why.empty(); r++) why = check_gate(n, g[i + r]);
            if (why.empty()) i += 3;
        }
        if (!why.empty()) {
            snprintf(buf, sizeof buf, "gate %zu: %s", i, why.c_str());
            return buf;
        }
    }
    return "";
}

// cos / sin of a fraction of a turn given in units of 2^-64.  Quarter turns
// are returned exactly.
static void turns_cs(uint64_t t64, double *c, double *s) {
    if ((t64 & ((UINT64_C(1) << 62) - 1)) == 0) {
        switch (t64 >> 62) {
            case 0: *c = 1; *s = 0; return;
            case 1: *c = 0; *s = 1; return;
            case 2: *c = -1; *s = 0; return;
            default: *c = 0; *s = -1; return;
        }
    }
    const double two_pi = 6.283185307179586476925286766559;
    double f = (double)(int64_t)t64 * 0x1p-64;  // signed fraction in [-1/2, 1/2)
    *c = std::cos(two_pi * f);
    *s = std::sin(two_pi * f);
}

uint64_t diag_turns64(const sv_gate &g, bool *exact) {
    switch (g.kind) {
        case SV_CZ:
            *exact = true;
            return UINT64_C(1) << 63;
        case SV_PK:
        case SV_CPK:
            *exact = true;
            if (g.log2den == 0) return 0;
            return (uint64_t)g.num << (64 - g.log2den);
        case SV_P:
        case SV_CP: {
            *exact = false;
            const double inv_two_pi = 0.15915494309189533576888376337251;
            double f = g.p[0] * inv_two_pi;
            f -= std::floor(f);  // [0, 1)
            double scaled = std::ldexp(f, 64);
            if (scaled >= 0x1p64) return 0;
            return (uint64_t)scaled;
        }
        default:
            *exact = true;
            return 0;
    }
}

Mat2 gate_matrix(const sv_gate &g) {
    Mat2 m{};
    switch (g.kind) {
        case SV_X:
            m.re[1] = 1.0;
            m.re[2] = 1.0;
            break;
        case SV_H: {
            const double r = 0.70710678118654752440084436210485;
            m.re[0] = r;
            m.re[1] = r;
            m.re[2] = r;
            m.re[3] = -r;
            break;
        }
        case SV_P:
        case SV_CP:
            m.re[0] = 1.0;
            m.re[3] = std::cos(g.p[0]);
            m.im[3] = std::sin(g.p[0]);
            break;
        case SV_CZ:
            m.re[0] = 1.0;
            m.re[3] = -1.0;
            break;
        case SV_PK:
        case SV_CPK: {
            bool ex;
            double c, s;
            turns_cs(diag_turns64(g, &ex), &c, &s);
            m.re[0] = 1.0;
            m.re[3] = c;
            m.im[3] = s;
            break;
        }
        case SV_U3: {
            double ht = 0.5 * g.p[0], ph = g.p[1], la = g.p[2];
            double c = std::cos(ht), s = std::sin(ht);
            m.re[0] = c;
            m.re[1] = -std::cos(la) * s;
            m.im[1] = -std::sin(la) * s;
            m.re[2] = std::cos(ph) * s;
            m.im[2] = std::sin(ph) * s;
            m.re[3] = std::cos(ph + la) * c;
            m.im[3] = std::sin(ph + la) * c;
            break;
        }
        case SV_U:
        case SV_CU:
        case SV_MCU:
            for (int e = 0; e < 4; e++) {
                m.re[e] = g.p[2 * e];
                m.im[e] = g.p[2 * e + 1];
            }
            break;
        default:
            break;
    }
    return m;
}

}  // namespace sv
