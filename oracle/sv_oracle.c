/*
 * FP64 CPU oracle for dense state-vector simulation.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the library path may link, load or
 * call this file; only the test-suite, the smoke check and the CPU-baseline
 * leg of the benchmark use it.  It shares no code, header, table or helper
 * with the CUDA path: the gate record below is declared here a second time,
 * with the same byte layout as the library's (an interface that has to be
 * alike), and every gate matrix is built here from its definition.
 *
 * What it computes, and where the paper defines it
 * (arxiv 2605.15098, "Accelerating State-Vector Quantum Simulation on
 * Integrated GPUs via Cache Locality Optimization"):
 *
 *  - The state of n qubits is an array of 2^n complex amplitudes
 *    (Sec. III-A).  Stored interleaved (re, im) in double precision.
 *  - A single-qubit gate U on target t is applied by Algorithm 1: an outer
 *    loop over i = 0, 2^(t+1), 2*2^(t+1), ... and an inner loop over
 *    j = i .. i + 2^t - 1 that reads the pair (S[j], S[j + 2^t]) and writes
 *    back U times that pair.  Qubit q is bit q of the index (the stride
 *    2^t of Algorithm 1); Eq. 1's Kronecker form is read with qubit 0 as the
 *    least significant factor, the only ordering under which Eq. 1 and
 *    Algorithm 1 describe the same operator.
 *  - A controlled gate runs inner-loop iteration j only when bit c of j is 1
 *    (Sec. III-A, the paragraph after Algorithm 1).
 *  - SWAP(a, b) exchanges the amplitudes of every index pair that differs
 *    exactly in bits a and b (the state permutation of Sec. III-B).
 *  - Probabilities are |amp|^2 in FP64, marginalised over the qubits in a
 *    mask and renormalised by their total; argmax and inverse-CDF sampling
 *    read the measured outcome (Sec. IV-A, the measured bitstring).
 *
 * Gate definitions the paper leaves implicit (the phase gate of Eq. 2 is
 * the only one it writes out):
 *    X = [[0,1],[1,0]]                H = [[1,1],[1,-1]] / sqrt(2)
 *    P(phi) = diag(1, e^{i phi})      CP(phi): P(phi) on target if control=1
 *    CZ = diag(1,-1) on target if control=1
 *    U3(th,ph,la) = [[cos(th/2),           -e^{i la} sin(th/2)],
 *                    [e^{i ph} sin(th/2),  e^{i(ph+la)} cos(th/2)]]
 *    U  = explicit 2x2 (row-major, re/im interleaved in p[0..7])
 *    CU = U on target if control=1
 *    PK/CPK = P/CP with phi = 2*pi*k / 2^j, the integer k reduced mod 2^j
 *             first (Eq. 3: U^a = P(2*pi*2^-n*a)).
 *
 * The general gate set beyond the paper's circuits (its control rule taken
 * to a set of controls, a general two-qubit unitary, and a measurement that
 * collapses the state):
 *    MCU  = explicit 2x2 U on the target where EVERY qubit of the control
 *           mask (the record's num field, a bit per qubit) is 1: Algorithm 1's
 *           inner iteration j runs only when all those bits of j are 1.
 *    U2Q  = explicit 4x4 unitary on the qubit pair (a = target, b = control):
 *           the amplitudes of the four indices that agree off bits a and b,
 *           ordered by k = bit_a + 2 bit_b, are multiplied by the matrix.  Its
 *           rows 0..3 are the p[0..7] (re/im interleaved) of this record and
 *           of the next three records, which have kind MAT.
 *    MEASURE = projective measurement of the target with the caller's
 *           uniform u = p[0] in [0,1): p0 and p1 are the sums of |amp|^2 over
 *           the indices with the target bit 0 and 1 (index order); the
 *           outcome is the smallest i with C_i > u C_last for C = (p0,
 *           p0 + p1); the amplitudes of the other outcome become 0 and the
 *           kept ones are divided by sqrt(p_outcome).
 *
 * Sampling order (the paper is silent): the marginal vector is cut into
 * blocks of 1024 consecutive outcomes; each block is summed in index order,
 * the running total over blocks is kept in block order, and the inclusive
 * cumulative value of outcome i is (sum of earlier blocks) + (sum of its own
 * block up to i).  A shot with uniform u in [0,1) returns the smallest i with
 * C_i > u * C_last.  Argmax returns the lowest index among equal maxima.
 *
 * Build: gcc -O2 -fopenmp -ffp-contract=off -fno-fast-math -shared -fPIC.
 * The OpenMP pragma only splits Algorithm 1's loop nest across host threads;
 * each pair is still updated by the same arithmetic in the same order.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* Gate record, byte layout identical to the library's public gate record. */
typedef struct {
    int32_t kind;
    int32_t target;
    int32_t control;   /* control qubit, second qubit of SWAP, -1 if none */
    int32_t log2den;   /* PK / CPK: denominator exponent j */
    int64_t num;       /* PK / CPK: numerator k */
    int64_t reserved;
    double p[8];
} or_gate;

enum {
    OR_X = 0, OR_H = 1, OR_P = 2, OR_CP = 3, OR_CZ = 4, OR_SWAP = 5,
    OR_U3 = 6, OR_U = 7, OR_CU = 8, OR_PK = 9, OR_CPK = 10,
    OR_MCU = 11, OR_U2Q = 12, OR_MAT = 13, OR_MEASURE = 14
};

#ifndef OR_MUTATION
#define OR_MUTATION 0   /* >0 plants a known mistake: used only by the pin tests */
#endif

/* 2x2 complex matrix, row-major: m[0]=U11, m[1]=U12, m[2]=U21, m[3]=U22 */
typedef struct { double re[4], im[4]; } mat2;

static const double OR_PI = 3.14159265358979323846;

static void phase_of(double phi, double *c, double *s) {
    *c = cos(phi);
    *s = sin(phi);
}

/* phi = 2*pi*k/2^j with k reduced modulo 2^j as an integer (Eq. 3) */
static double dyadic_angle(int64_t num, int32_t log2den) {
    uint64_t mod = (log2den >= 64) ? 0 : ((uint64_t)1 << log2den);
    uint64_t r;
    if (log2den >= 64) {
        r = (uint64_t)num;
    } else {
        r = (uint64_t)num & (mod - 1);   /* two's complement: same as k mod 2^j */
    }
    return 2.0 * OR_PI * ((double)r / ldexp(1.0, log2den));
}

static int build_matrix(const or_gate *g, mat2 *u) {
    memset(u, 0, sizeof(*u));
    double c, s;
    switch (g->kind) {
    case OR_X:
        u->re[1] = 1.0; u->re[2] = 1.0;
        return 0;
    case OR_H: {
        double h = 1.0 / sqrt(2.0);
        u->re[0] = h; u->re[1] = h; u->re[2] = h; u->re[3] = -h;
#if OR_MUTATION == 1
        u->re[3] = h;            /* planted: wrong sign in H */
#endif
        return 0;
    }
    case OR_P:
    case OR_CP:
        phase_of(g->p[0], &c, &s);
        u->re[0] = 1.0; u->re[3] = c; u->im[3] = s;
#if OR_MUTATION == 2
        u->im[3] = -s;           /* planted: conjugated phase */
#endif
        return 0;
    case OR_PK:
    case OR_CPK:
        phase_of(dyadic_angle(g->num, g->log2den), &c, &s);
        u->re[0] = 1.0; u->re[3] = c; u->im[3] = s;
        return 0;
    case OR_CZ:
        u->re[0] = 1.0; u->re[3] = -1.0;
        return 0;
    case OR_U3: {
        double th = g->p[0], ph = g->p[1], la = g->p[2];
        double ct = cos(th / 2.0), st = sin(th / 2.0);
        u->re[0] = ct;
        u->re[1] = -cos(la) * st;       u->im[1] = -sin(la) * st;
        u->re[2] = cos(ph) * st;        u->im[2] = sin(ph) * st;
        u->re[3] = cos(ph + la) * ct;   u->im[3] = sin(ph + la) * ct;
#if OR_MUTATION == 3
        u->im[2] = -sin(ph) * st;       /* planted: sign of e^{i phi} */
#endif
        return 0;
    }
    case OR_U:
    case OR_CU:
    case OR_MCU:
        for (int e = 0; e < 4; e++) {
            u->re[e] = g->p[2 * e];
            u->im[e] = g->p[2 * e + 1];
        }
#if OR_MUTATION == 4
        { double t = u->re[1]; u->re[1] = u->re[2]; u->re[2] = t;
          t = u->im[1]; u->im[1] = u->im[2]; u->im[2] = t; } /* planted: transposed */
#endif
        return 0;
    default:
        return -1;
    }
}

static int has_control(int kind) {
    return kind == OR_CP || kind == OR_CZ || kind == OR_CU || kind == OR_CPK;
}

/* Algorithm 1 (ApplyGate) with the control rule of Sec. III-A, the controls
 * given as a mask of qubits that must all be 1 (0: none). */
static void apply_gate_alg1(int n, double *S, const mat2 *u, int t, uint64_t cmask) {
    const uint64_t N = (uint64_t)1 << n;
    const uint64_t st = (uint64_t)1 << t;
#if OR_MUTATION == 5
    const uint64_t st2 = st;     /* planted: outer step 2^t instead of 2^(t+1) */
#else
    const uint64_t st2 = st << 1;
#endif
    const uint64_t outer = N / st2;
    const double u0r = u->re[0], u0i = u->im[0], u1r = u->re[1], u1i = u->im[1];
    const double u2r = u->re[2], u2i = u->im[2], u3r = u->re[3], u3i = u->im[3];
    int64_t io, jo;
#pragma omp parallel for collapse(2) schedule(static) if (N >= (1u << 16))
    for (io = 0; io < (int64_t)outer; io++) {
        for (jo = 0; jo < (int64_t)st; jo++) {
            uint64_t i = (uint64_t)io * st2;
            uint64_t j = i + (uint64_t)jo;
            if (j + st >= N) continue;            /* only reachable with a planted mistake */
#if OR_MUTATION == 6
            if (cmask && !(j & cmask)) continue;        /* planted: any control instead of all */
#else
            if ((j & cmask) != cmask) continue;
#endif
            double ar = S[2 * j], ai = S[2 * j + 1];
            double br = S[2 * (j + st)], bi = S[2 * (j + st) + 1];
            /* S[j] = U11 a + U12 b ; S[j+2^t] = U21 a + U22 b */
            double xr = (u0r * ar - u0i * ai) + (u1r * br - u1i * bi);
            double xi = (u0r * ai + u0i * ar) + (u1r * bi + u1i * br);
            double yr = (u2r * ar - u2i * ai) + (u3r * br - u3i * bi);
            double yi = (u2r * ai + u2i * ar) + (u3r * bi + u3i * br);
            S[2 * j] = xr; S[2 * j + 1] = xi;
            S[2 * (j + st)] = yr; S[2 * (j + st) + 1] = yi;
        }
    }
}

/* SWAP(a, b): exchange S[x] and S[x ^ (2^a | 2^b)] for every x with bit a = 1, bit b = 0. */
static void apply_swap(int n, double *S, int a, int b) {
    const uint64_t N = (uint64_t)1 << n;
    const uint64_t ma = (uint64_t)1 << a, mb = (uint64_t)1 << b;
    int64_t x;
#pragma omp parallel for schedule(static) if (N >= (1u << 16))
    for (x = 0; x < (int64_t)N; x++) {
        uint64_t ux = (uint64_t)x;
        if ((ux & ma) && !(ux & mb)) {
            uint64_t y = ux ^ ma ^ mb;
            double tr = S[2 * ux], ti = S[2 * ux + 1];
            S[2 * ux] = S[2 * y]; S[2 * ux + 1] = S[2 * y + 1];
            S[2 * y] = tr; S[2 * y + 1] = ti;
        }
    }
}

/* U2Q on (a, b): for every index x with bits a and b both 0, the four
 * amplitudes x + k_a 2^a + k_b 2^b (k = k_a + 2 k_b) are replaced by
 * M times them; M row-major, re/im interleaved, 32 doubles. */
static void apply_u2q(int n, double *S, const double *M, int a, int b) {
    const uint64_t N = (uint64_t)1 << n;
    const uint64_t ma = (uint64_t)1 << a, mb = (uint64_t)1 << b;
    int64_t x;
#pragma omp parallel for schedule(static) if (N >= (1u << 16))
    for (x = 0; x < (int64_t)N; x++) {
        const uint64_t ux = (uint64_t)x;
        if (ux & (ma | mb)) continue;
        uint64_t idx[4];
        idx[0] = ux;
        idx[1] = ux | ma;
        idx[2] = ux | mb;
        idx[3] = ux | ma | mb;
        double vr[4], vi[4];
        for (int k = 0; k < 4; k++) {
            vr[k] = S[2 * idx[k]];
            vi[k] = S[2 * idx[k] + 1];
        }
        for (int r = 0; r < 4; r++) {
            double yr = 0.0, yi = 0.0;
            for (int k = 0; k < 4; k++) {
#if OR_MUTATION == 7
                const double mr = M[8 * k + 2 * r], mi = M[8 * k + 2 * r + 1]; /* planted: transposed */
#else
                const double mr = M[8 * r + 2 * k], mi = M[8 * r + 2 * k + 1];
#endif
                yr += mr * vr[k] - mi * vi[k];
                yi += mr * vi[k] + mi * vr[k];
            }
            S[2 * idx[r]] = yr;
            S[2 * idx[r] + 1] = yi;
        }
    }
}

/* Projective measurement of qubit t with uniform u (see the header);
 * returns the outcome (0 or 1), or -1 when the state has zero norm. */
static int apply_measure(int n, double *S, int t, double u) {
    const uint64_t N = (uint64_t)1 << n;
    const uint64_t mt = (uint64_t)1 << t;
    double p0 = 0.0, p1 = 0.0;
    for (uint64_t x = 0; x < N; x++) {
        const double q = S[2 * x] * S[2 * x] + S[2 * x + 1] * S[2 * x + 1];
        if (x & mt) p1 += q;
        else p0 += q;
    }
    const double last = p0 + p1;
    if (!(last > 0.0)) return -1;
    const int out = (p0 > u * last) ? 0 : 1;
    const double keep = out ? p1 : p0;
#if OR_MUTATION == 8
    const double sc = 1.0;                  /* planted: no renormalisation */
#else
    const double sc = 1.0 / sqrt(keep);
#endif
    int64_t x;
#pragma omp parallel for schedule(static) if (N >= (1u << 16))
    for (x = 0; x < (int64_t)N; x++) {
        const int bit = ((uint64_t)x & mt) ? 1 : 0;
        if (bit == out) {
            S[2 * x] *= sc;
            S[2 * x + 1] *= sc;
        } else {
            S[2 * x] = 0.0;
            S[2 * x + 1] = 0.0;
        }
    }
    return out;
}

int or_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void or_set_threads(int t) {
#ifdef _OPENMP
    if (t > 0) omp_set_num_threads(t);
#else
    (void)t;
#endif
}

/* psi = |0...0> */
int or_init(int n, double *psi) {
    if (n < 1 || n > 40 || !psi) return -1;
    uint64_t N = (uint64_t)1 << n;
    memset(psi, 0, sizeof(double) * 2 * N);
    psi[0] = 1.0;
    return 0;
}

/* Validate one gate against n; 0 if fine.  A U2Q must be followed by three
 * MAT records and a MAT record may appear only there (checked by the list
 * walk in or_apply_measured). */
static int check_gate(int n, const or_gate *g) {
    if (g->kind < OR_X || g->kind > OR_MEASURE) return -1;
    if (g->target < 0 || g->target >= n) return -1;
    if (has_control(g->kind) || g->kind == OR_SWAP || g->kind == OR_U2Q) {
        if (g->control < 0 || g->control >= n || g->control == g->target) return -1;
    }
    if ((g->kind == OR_PK || g->kind == OR_CPK) && (g->log2den < 0 || g->log2den > 64)) return -1;
    if (g->kind == OR_MCU) {
        const uint64_t cm = (uint64_t)g->num;
        if (!cm || (n < 64 && (cm >> n)) || ((cm >> g->target) & 1u)) return -1;
    }
    if (g->kind == OR_MEASURE && !(g->p[0] >= 0.0 && g->p[0] < 1.0)) return -1;
    return 0;
}

/* Apply m gates in list order; the outcome of each MEASURE, in list order,
 * goes to outcomes[] (optional).  Returns 0, or -(index+1) of the first bad
 * gate (nothing is applied when any gate is invalid), or -(m+2) when a
 * measurement meets a state of zero norm. */
int or_apply_measured(int n, double *psi, const or_gate *gates, uint64_t m, uint8_t *outcomes) {
    if (n < 1 || n > 40 || !psi || (m && !gates)) return -1;
    for (uint64_t e = 0; e < m; e++) {
        if (check_gate(n, &gates[e])) return -(int)(e + 1);
        if (gates[e].kind == OR_MAT) return -(int)(e + 1);
        if (gates[e].kind == OR_U2Q) {
            for (uint64_t k = 1; k <= 3; k++)
                if (e + k >= m || gates[e + k].kind != OR_MAT) return -(int)(e + 1);
            e += 3;
        }
    }
    uint64_t nm = 0;
    for (uint64_t e = 0; e < m; e++) {
        const or_gate *g = &gates[e];
        if (g->kind == OR_SWAP) {
            apply_swap(n, psi, g->target, g->control);
            continue;
        }
        if (g->kind == OR_U2Q) {
            double M[32];
            for (int r = 0; r < 4; r++)
                for (int c = 0; c < 8; c++) M[8 * r + c] = gates[e + r].p[c];
            apply_u2q(n, psi, M, g->target, g->control);
            e += 3;
            continue;
        }
        if (g->kind == OR_MEASURE) {
            const int out = apply_measure(n, psi, g->target, g->p[0]);
            if (out < 0) return -(int)(m + 2);
            if (outcomes) outcomes[nm] = (uint8_t)out;
            nm++;
            continue;
        }
        mat2 u;
        build_matrix(g, &u);
        uint64_t cmask = 0;
        if (has_control(g->kind)) cmask = (uint64_t)1 << g->control;
        if (g->kind == OR_MCU) cmask = (uint64_t)g->num;
        apply_gate_alg1(n, psi, &u, g->target, cmask);
    }
    return 0;
}

int or_apply(int n, double *psi, const or_gate *gates, uint64_t m) {
    return or_apply_measured(n, psi, gates, m, NULL);
}

/* Marginal probabilities over the qubits in mask, renormalised by their total.
 * Output index: bit j of the outcome is the j-th lowest qubit of mask.
 * Summation: for every outcome, the amplitudes contributing to it are added
 * in increasing index order; the total is then summed in outcome order. */
int or_marginal(int n, const double *psi, uint64_t mask, double *out) {
    if (n < 1 || n > 40 || !psi || !out) return -1;
    if (mask >> n) return -1;
    int q[64], nq = 0;
    for (int b = 0; b < n; b++)
        if ((mask >> b) & 1u) q[nq++] = b;
    uint64_t M = (uint64_t)1 << nq;
    memset(out, 0, sizeof(double) * M);
    uint64_t N = (uint64_t)1 << n;
    for (uint64_t x = 0; x < N; x++) {
        uint64_t o = 0;
        for (int j = 0; j < nq; j++) o |= ((x >> q[j]) & 1u) << j;
        double re = psi[2 * x], im = psi[2 * x + 1];
        out[o] += re * re + im * im;
    }
    double tot = 0.0;
    for (uint64_t o = 0; o < M; o++) tot += out[o];
    if (!(tot > 0.0)) return -2;
    for (uint64_t o = 0; o < M; o++) out[o] /= tot;
    return 0;
}

/* Lowest index holding the maximum probability. */
int or_argmax(const double *p, uint64_t len, uint64_t *idx, double *pmax) {
    if (!p || !len || !idx) return -1;
    uint64_t best = 0;
    for (uint64_t i = 1; i < len; i++)
        if (p[i] > p[best]) best = i;
    *idx = best;
    if (pmax) *pmax = p[best];
    return 0;
}

/* Inclusive CDF in the documented block order (blocks of 1024). */
int or_cdf(const double *p, uint64_t len, double *cdf) {
    if (!p || !cdf || !len) return -1;
    double before = 0.0;
    for (uint64_t b0 = 0; b0 < len; b0 += 1024) {
        uint64_t b1 = b0 + 1024 < len ? b0 + 1024 : len;
        double run = 0.0;
        for (uint64_t i = b0; i < b1; i++) {
            run += p[i];
            cdf[i] = before + run;
        }
        before += run;
    }
    return 0;
}

/* Inverse-CDF sampling.  margin[s] (optional) receives the distance between
 * u*C_last and the nearest CDF boundary of the chosen outcome, so that a
 * comparison can tell a genuine disagreement from a boundary tie. */
int or_sample(const double *p, uint64_t len, const double *u, uint64_t shots,
              uint64_t *out, double *margin) {
    if (!p || !len || (shots && (!u || !out))) return -1;
    double *cdf = (double *)malloc(sizeof(double) * len);
    if (!cdf) return -2;
    or_cdf(p, len, cdf);
    double last = cdf[len - 1];
    for (uint64_t s = 0; s < shots; s++) {
        double target = u[s] * last;
        uint64_t pick = len - 1;
        for (uint64_t i = 0; i < len; i++)
            if (cdf[i] > target) { pick = i; break; }
        out[s] = pick;
        if (margin) {
            double hi = cdf[pick] - target;
            double lo = pick ? target - cdf[pick - 1] : target;
            margin[s] = hi < lo ? hi : lo;
        }
    }
    free(cdf);
    return 0;
}
