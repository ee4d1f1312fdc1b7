/*
 * The paper's partitioned simulation on the host CPU (Sec. III-B), kept as a
 * second CPU baseline next to the oracle's plain Algorithm 1: the paper
 * reports that partitioning brings no gain on CPUs, and this program lets the
 * benchmark measure that on the GPU machine's host cores.  It is not part of the
 * library's GPU path and shares no code with it or with the oracle; the gate
 * record is declared here again with the library's byte layout.
 *
 * What it computes (FP64, interleaved complex):
 *  - Qubits 0..l-1 of the physical index are local, the others global; the
 *    state is 2^(n-l) contiguous blocks of 2^l amplitudes (Sec. III-B,
 *    Fig. 2).
 *  - A gate whose target is local is deferred.  A gate whose target is global
 *    first flushes the deferred gates, then swaps its target with the least
 *    recently used local qubit that the gate itself does not use (ties: the
 *    lowest), by moving amplitudes across the whole state, and updates the
 *    logical-to-physical map; the gate is then deferred like any other.
 *  - Flushing applies every deferred gate, in order, to one block before the
 *    next block (blocks run in parallel on the host threads).  Inside a
 *    block a gate is Algorithm 1 on the local target; a local control tests
 *    its bit of the index, a global control its bit of the block index.
 *  - A SWAP gate of the circuit only exchanges two entries of the map.
 *  - The result is returned in logical qubit order.
 * Gate matrices (X, H, P, CP, CZ, U3, U, CU, PK, CPK) follow the library's
 * definitions in sv.h; the general gate set is not supported here.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
    int32_t kind, target, control, log2den;
    int64_t num, reserved;
    double p[8];
} cp_gate;

enum { K_X = 0, K_H = 1, K_P = 2, K_CP = 3, K_CZ = 4, K_SWAP = 5, K_U3 = 6, K_U = 7, K_CU = 8, K_PK = 9, K_CPK = 10 };

typedef struct {
    int t, c;     /* physical target, physical control (-1: none) */
    double m[8];  /* U11, U12, U21, U22 as (re, im) */
} cp_op;

static const double kTwoPi = 6.283185307179586476925286766559;

static void phase(double ang, double *re, double *im) {
    *re = cos(ang);
    *im = sin(ang);
}

/* 2x2 matrix of a gate; returns 0, or -1 for a kind this program does not take. */
static int matrix_of(const cp_gate *g, double m[8]) {
    memset(m, 0, 8 * sizeof(double));
    switch (g->kind) {
        case K_X: m[2] = 1.0; m[4] = 1.0; return 0;
        case K_H: {
            const double s = 1.0 / sqrt(2.0);
            m[0] = s; m[2] = s; m[4] = s; m[6] = -s;
            return 0;
        }
        case K_P: case K_CP:
            m[0] = 1.0;
            phase(g->p[0], &m[6], &m[7]);
            return 0;
        case K_CZ: m[0] = 1.0; m[6] = -1.0; return 0;
        case K_PK: case K_CPK: {
            /* 2 pi k / 2^j with k reduced modulo 2^j as an integer first */
            const int j = g->log2den;
            const uint64_t mask = j >= 64 ? ~UINT64_C(0) : ((UINT64_C(1) << j) - 1);
            const uint64_t k = (uint64_t)g->num & mask;
            m[0] = 1.0;
            phase(kTwoPi * ldexp((double)k, -j), &m[6], &m[7]);
            return 0;
        }
        case K_U3: {
            const double th = g->p[0], ph = g->p[1], la = g->p[2];
            const double c = cos(th / 2.0), s = sin(th / 2.0);
            double er, ei;
            m[0] = c;
            phase(la, &er, &ei);
            m[2] = -er * s; m[3] = -ei * s;
            phase(ph, &er, &ei);
            m[4] = er * s; m[5] = ei * s;
            phase(ph + la, &er, &ei);
            m[6] = er * c; m[7] = ei * c;
            return 0;
        }
        case K_U: case K_CU:
            memcpy(m, g->p, 8 * sizeof(double));
            return 0;
        default:
            return -1;
    }
}

static int controlled(int kind) { return kind == K_CP || kind == K_CZ || kind == K_CU || kind == K_CPK; }

/* Deferred gates on one block of 2^l amplitudes with block index b. */
static void run_block(double *blk, int l, uint64_t b, const cp_op *ops, size_t nops) {
    const uint64_t len = UINT64_C(1) << l;
    for (size_t o = 0; o < nops; o++) {
        const cp_op *op = &ops[o];
        if (op->c >= l && !((b >> (op->c - l)) & 1)) continue;  /* a global control: the whole block */
        const uint64_t st = UINT64_C(1) << op->t;
        const int lc = op->c >= 0 && op->c < l;
        for (uint64_t i = 0; i < len; i += 2 * st)
            for (uint64_t j = i; j < i + st; j++) {
                if (lc && !((j >> op->c) & 1)) continue;
                double *a = blk + 2 * j, *c = blk + 2 * (j + st);
                const double ar = a[0], ai = a[1], br = c[0], bi = c[1];
                const double *m = op->m;
                a[0] = m[0] * ar - m[1] * ai + m[2] * br - m[3] * bi;
                a[1] = m[0] * ai + m[1] * ar + m[2] * bi + m[3] * br;
                c[0] = m[4] * ar - m[5] * ai + m[6] * br - m[7] * bi;
                c[1] = m[4] * ai + m[5] * ar + m[6] * bi + m[7] * br;
            }
    }
}

static void flush(double *psi, int n, int l, const cp_op *ops, size_t *nops, int64_t *passes) {
    if (!*nops) return;
    const int64_t nb = (int64_t)1 << (n - l);
#pragma omp parallel for schedule(static)
    for (int64_t b = 0; b < nb; b++) run_block(psi + 2 * ((uint64_t)b << l), l, (uint64_t)b, ops, *nops);
    *nops = 0;
    (*passes)++;
}

/* Exchange physical bits g and v of the index across the whole state. */
static void swap_bits(double *psi, int n, int g, int v) {
    const int64_t quarter = (int64_t)1 << (n - 2);
    const int lo = g < v ? g : v, hi = g < v ? v : g;
#pragma omp parallel for schedule(static)
    for (int64_t q = 0; q < quarter; q++) {
        uint64_t x = (uint64_t)q;
        x = ((x >> lo) << (lo + 1)) | (x & ((UINT64_C(1) << lo) - 1));
        x = ((x >> hi) << (hi + 1)) | (x & ((UINT64_C(1) << hi) - 1));
        const uint64_t a = x | (UINT64_C(1) << g), b = x | (UINT64_C(1) << v);  /* bit g set / bit v set */
        double t0 = psi[2 * a], t1 = psi[2 * a + 1];
        psi[2 * a] = psi[2 * b];
        psi[2 * a + 1] = psi[2 * b + 1];
        psi[2 * b] = t0;
        psi[2 * b + 1] = t1;
    }
}

int cp_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/*
 * Apply gates[0..m) to psi (2^n amplitudes, interleaved FP64, logical order,
 * in place) with blocks of 2^l amplitudes.  stats (may be NULL): passes
 * (flushes), swaps (global-local exchanges).  Returns 0, -1 for bad
 * arguments, -2 for an unsupported gate, -3 if out of memory.
 */
int cp_run(int n, int l, double *psi, const cp_gate *gates, size_t m, int64_t *stats) {
    if (n < 2 || n > 34 || l < 2 || !psi || (m && !gates)) return -1;
    if (l > n) l = n;
    int phys[64], logi[64];
    int64_t last[64];
    for (int q = 0; q < 64; q++) {
        phys[q] = q;
        logi[q] = q;
        last[q] = 0;
    }
    cp_op *ops = (cp_op *)malloc((m ? m : 1) * sizeof(cp_op));
    if (!ops) return -3;
    size_t nops = 0;
    int64_t passes = 0, swaps = 0, clock = 1;
    for (size_t i = 0; i < m; i++) {
        const cp_gate *g = &gates[i];
        if (g->target < 0 || g->target >= n) {
            free(ops);
            return -1;
        }
        if (g->kind == K_SWAP) {  /* a relabel of the map */
            const int a = g->target, b = g->control;
            if (b < 0 || b >= n || a == b) {
                free(ops);
                return -1;
            }
            const int pa = phys[a], pb = phys[b];
            phys[a] = pb;
            phys[b] = pa;
            logi[pa] = b;
            logi[pb] = a;
            continue;
        }
        cp_op op;
        if (matrix_of(g, op.m)) {
            free(ops);
            return -2;
        }
        op.c = -1;
        if (controlled(g->kind)) {
            if (g->control < 0 || g->control >= n || g->control == g->target) {
                free(ops);
                return -1;
            }
            op.c = phys[g->control];
        }
        op.t = phys[g->target];
        if (op.t >= l) {  /* a global target: flush, then bring it local */
            flush(psi, n, l, ops, &nops, &passes);
            int v = -1;
            for (int q = 0; q < l; q++) {
                if (q == op.c) continue;
                if (v < 0 || last[q] < last[v]) v = q;
            }
            swap_bits(psi, n, op.t, v);
            swaps++;
            const int lt = logi[op.t], lv = logi[v];
            phys[lt] = v;
            phys[lv] = op.t;
            logi[v] = lt;
            logi[op.t] = lv;
            last[op.t] = last[v];
            op.t = v;
        }
        ops[nops++] = op;
        last[op.t] = clock;
        if (op.c >= 0 && op.c < l) last[op.c] = clock;
        clock++;
    }
    flush(psi, n, l, ops, &nops, &passes);
    free(ops);
    /* back to logical order */
    int ident = 1;
    for (int q = 0; q < n; q++) ident &= phys[q] == q;
    if (!ident) {
        const uint64_t N = UINT64_C(1) << n;
        double *out = (double *)malloc(2 * N * sizeof(double));
        if (!out) return -3;
#pragma omp parallel for schedule(static)
        for (int64_t y = 0; y < (int64_t)N; y++) {
            uint64_t x = 0;
            for (int q = 0; q < n; q++)
                if (((uint64_t)y >> q) & 1) x |= UINT64_C(1) << phys[q];
            out[2 * y] = psi[2 * x];
            out[2 * y + 1] = psi[2 * x + 1];
        }
        memcpy(psi, out, 2 * N * sizeof(double));
        free(out);
    }
    if (stats) {
        stats[0] = passes;
        stats[1] = swaps;
    }
    return 0;
}
