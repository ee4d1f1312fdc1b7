/*
 * sv.h - C ABI of libsv, a GB300 (sm_103a) dense state-vector simulator.
 *
 * Method: arxiv 2605.15098, "Accelerating State-Vector Quantum Simulation on
 * Integrated GPUs via Cache Locality Optimization".  The problem the calls
 * follow is the paper's: an n-qubit state is an array of 2^n complex
 * amplitudes that starts in |0...0>, a list of single-qubit and controlled
 * gates is applied to it (Sec. III-A, Eq. 1, Algorithm 1), and the result is
 * read out as measured bitstrings (Sec. IV-A).  The partitioned execution
 * (Sec. III-B: local/global qubits, deferred local gates applied block by
 * block, global qubits brought local, controls on global qubits decided per
 * block) is an implementation strategy: it changes the order of work, never
 * the result beyond floating-point rounding.
 *
 * Conventions shared by every call
 *  - Qubit q is bit q of the amplitude index (the stride 2^t of Algorithm 1).
 *  - Amplitudes are interleaved complex: SV_C64 = (float re, float im),
 *    8 bytes; SV_C128 = (double re, double im), 16 bytes.
 *  - All pointers named host_* are host memory owned by the caller; dev_*
 *    are device pointers on the handle's device, owned by the caller.  The
 *    library owns the state buffer unless the handle was made by
 *    sv_create_on.
 *  - Every argument is validated on the host before any kernel is launched;
 *    a call that returns an error has not modified the state.
 *  - Work is ordered on the handle's CUDA stream.  Calls that return data to
 *    host memory synchronise that stream before returning; sv_apply_circuit
 *    returns once its kernels are enqueued.
 *  - A handle must not be used from two threads at once.  sv_last_error()
 *    is per thread.
 *  - Nothing here allocates host memory that the caller must free.
 */
#ifndef LIBSV_SV_H_
#define LIBSV_SV_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sv_state *sv_handle;

typedef enum { SV_C64 = 0, SV_C128 = 1 } sv_dtype;

typedef enum {
    SV_OK = 0,
    SV_ERR_ARG = -1,         /* invalid argument (nothing was run)              */
    SV_ERR_OOM = -2,         /* device or host allocation failed                */
    SV_ERR_CUDA = -3,        /* a CUDA runtime call failed (message has the code) */
    SV_ERR_TIMEOUT = -4,     /* a bounded device wait gave up                    */
    SV_ERR_STATE = -5,       /* handle in a state that does not allow the call  */
    SV_ERR_UNSUPPORTED = -6  /* valid request this build cannot serve           */
} sv_status;

/* Gate kinds.  Matrices (row-major, U11 acts |0> -> |0>):
 *   SV_X    [[0,1],[1,0]]
 *   SV_H    [[1,1],[1,-1]]/sqrt(2)
 *   SV_P    diag(1, e^{i p[0]})                       (Eq. 2's phase gate)
 *   SV_CP   SV_P on `target` when bit `control` is 1  (control rule, Sec. III-A)
 *   SV_CZ   diag(1,-1) on `target` when bit `control` is 1
 *   SV_SWAP exchange qubits `target` and `control`    (the SWAP of Sec. III-B)
 *   SV_U3   [[cos(a/2), -e^{ic} sin(a/2)], [e^{ib} sin(a/2), e^{i(b+c)} cos(a/2)]]
 *           with a, b, c = p[0], p[1], p[2]
 *   SV_U    explicit 2x2: p = {U11.re, U11.im, U12.re, U12.im, U21.re, U21.im,
 *           U22.re, U22.im}
 *   SV_CU   SV_U on `target` when bit `control` is 1
 *   SV_PK   diag(1, e^{2 pi i k / 2^j}) with k = num, j = log2den (0..62); k is
 *           reduced modulo 2^j as an integer, so the phase is exact (Eq. 3,
 *           U^a = P(2 pi 2^-n a))
 *   SV_CPK  SV_PK on `target` when bit `control` is 1
 *
 * The general gate set (the control rule of Sec. III-A taken to a set of
 * controls, a general two-qubit unitary, and a collapsing measurement).  In
 * the partitioned modes each of them is its own step between tile passes,
 * run by the per-gate kernels:
 *   SV_MCU      the explicit 2x2 of p (as SV_U) on `target` where EVERY qubit
 *               of the mask `num` (bit q = qubit q; nonzero, target not in it)
 *               is 1; `control` is -1
 *   SV_U2Q      a 4x4 unitary M on the qubits a = `target`, b = `control`: the
 *               four amplitudes that agree off a and b, ordered by
 *               k = bit_a + 2 bit_b, are multiplied by M.  Row r of M (4
 *               complex entries, re/im interleaved) is the p of record r: this
 *               record holds row 0 and the next three records, of kind
 *               SV_MAT with the same target and control, rows 1..3
 *   SV_MAT      a row of the preceding SV_U2Q (valid only there)
 *   SV_MEASURE  projective measurement of `target` with the caller's uniform
 *               u = p[0] in [0,1): p0 and p1 are the FP64 sums of |amp|^2 over
 *               the amplitudes with that qubit 0 and 1; the outcome is the
 *               smallest i with C_i > u * C_last for C = (p0, p0 + p1) (as
 *               sv_sample); the other half of the state becomes 0 and the kept
 *               half is divided by sqrt(p_outcome).  Outcomes are read with
 *               sv_last_measurements.
 */
enum {
    SV_X = 0, SV_H = 1, SV_P = 2, SV_CP = 3, SV_CZ = 4, SV_SWAP = 5,
    SV_U3 = 6, SV_U = 7, SV_CU = 8, SV_PK = 9, SV_CPK = 10,
    SV_MCU = 11, SV_U2Q = 12, SV_MAT = 13, SV_MEASURE = 14
};

/* One gate, 96 bytes.  `control` is the control qubit of CP/CZ/CU/CPK and
 * the second qubit of SWAP, U2Q and MAT; it must differ from `target` and is
 * ignored (set it to -1) for the other kinds.  `num` is PK/CPK's numerator
 * and MCU's control mask.  `reserved` must be 0. */
typedef struct sv_gate {
    int32_t kind;
    int32_t target;
    int32_t control;
    int32_t log2den;
    int64_t num;
    int64_t reserved;
    double p[8];
} sv_gate;

/* Execution strategy for sv_apply_circuit. */
typedef enum {
    SV_MODE_AUTO = 0,        /* partitioned when n is larger than a tile      */
    SV_MODE_PERGATE = 1,     /* one HBM sweep per gate (Algorithm 1 per gate)  */
    SV_MODE_PARTITIONED = 2, /* tile passes (Sec. III-B), shared-memory tiles  */
    SV_MODE_FUSED = 3        /* partitioned + 5-qubit blocks on tensor cores   */
} sv_mode;

/* Flags for sv_config.flags. */
enum {
    SV_FLAG_NO_DIAG_MERGE = 1,  /* keep every diagonal gate as its own step  */
    SV_FLAG_PAPER_SWAP = 2,     /* bring global targets local by explicit
                                   remap passes with LRU eviction, as the
                                   paper does, instead of gathering them
                                   into the tile                               */
    SV_FLAG_NO_RELABEL = 4,     /* execute SWAP gates as data movement        */
    SV_FLAG_GENERIC_TILE = 8,   /* use the generic shared-memory tile kernel
                                   for every pass (no register stages)        */
    SV_FLAG_NO_PLAN_CACHE = 16, /* plan, compile and upload the list on this
                                   call even if the handle holds its programme */
    SV_FLAG_EARLY_DIAG = 32,    /* keep each diagonal gate in the first pass
                                   where it is ready (default: the pass of the
                                   first later gate it does not commute with)  */
    SV_FLAG_GREEDY_ONLY = 64,   /* take each pass's local qubits as the greedy
                                   list scheduling picks them, without the
                                   local search that refines the set          */
    SV_FLAG_L2_BLOCKS = 128,    /* two-level blocking (Sec. III-B's block sized
                                   to the last-level cache): consecutive
                                   register-stage passes whose tile qubits
                                   together span at most l2_qubits qubits run
                                   as one launch, block by block, so that the
                                   state moves between them through L2        */
    SV_FLAG_NARROW_FIRST = 256  /* the first tile pass of the list gathers
                                   16-amplitude chunks (4 chunk qubits) whatever
                                   chunk_qubits says, so that more of its tile
                                   qubits are free to choose; it pays when that
                                   pass generates a recorded basis state and
                                   reads nothing (sv_create, sv_reset)        */
};

/* Planner choice for partitioned modes. */
typedef enum { SV_PLANNER_GREEDY = 0, SV_PLANNER_LEARNED = 1 } sv_planner;

/* All-zero means "library defaults".  tile_qubits = k, the number of qubits
 * whose amplitudes one shared-memory tile holds (2^k amplitudes);
 * chunk_qubits = c, the lowest qubits that every tile contains as one
 * contiguous run (the unit of a bulk copy). */
typedef struct sv_config {
    int32_t mode;          /* sv_mode                                          */
    int32_t tile_qubits;   /* k; 0 = default for the dtype                     */
    int32_t chunk_qubits;  /* c; 0 = default                                   */
    int32_t fuse_qubits;   /* width of a tensor-core fused block; 0 = 5        */
    int32_t planner;       /* sv_planner                                       */
    int32_t flags;         /* SV_FLAG_*                                        */
    int32_t l2_qubits;     /* with SV_FLAG_L2_BLOCKS: the widest union of tile
                              qubits a group of passes may span (its L2 block
                              holds 2^l2_qubits amplitudes); 0 = from the
                              device's L2 size (a block of at most 1/8 of it) */
    int32_t l2_chunk;      /* with SV_FLAG_L2_BLOCKS: consecutive tiles a CTA
                              takes per claim (1, 2, 4, 8 or 16; 0 = 2).  More
                              tiles per claim mean fewer programme reloads and
                              a larger lag between a block's passes           */
    int32_t batch_split;   /* batched launches: an instance of at least this
                              many qubits has each pass's tiles shared out
                              among CTAs (claims of 8 tiles), its read-out
                              following its last pass; smaller instances run
                              whole on one CTA.  25 = never split; 0 =
                              automatic: 16 if the largest instance costs
                              more than half of an even share of the work
                              per CTA, else never                            */
    int32_t reserved[7];   /* must be 0                                        */
} sv_config;

/* Counters of the last sv_apply_circuit on a handle. */
typedef struct sv_stats {
    int32_t gates;          /* gates in the list                                */
    int32_t passes;         /* full sweeps over the state: tile passes, per-gate
                               sweeps and remap passes                          */
    int32_t remaps;         /* of which explicit remap (permutation) passes     */
    int32_t kernels;        /* kernel launches enqueued                         */
    int32_t relabels;       /* SWAP gates absorbed into the qubit map           */
    int32_t fused_blocks;   /* tensor-core blocks applied                       */
    double sweep_bytes;     /* 2 * passes * 2^n * sizeof(amplitude)             */
    double touched_bytes;   /* bytes the kernels had to move (diagonal and SWAP
                               per-gate sweeps touch part of the state)         */
    double h2d_bytes;       /* host-to-device bytes copied (the pass programme)  */
    int32_t planner;        /* sv_planner that produced the executed plan        */
    int32_t candidates;     /* learned planner: candidate passes it scored        */
    double predicted_ms;    /* learned planner: the cost model's estimate (0 if
                               the greedy plan ran)                             */
    int32_t ctas_per_sm;    /* resident CTAs per SM of the call's register-stage
                               and L2 block launches (the smallest; 0 if none)  */
    int32_t reserved;
} sv_stats;

/* ---- lifetime --------------------------------------------------------- */

/* Allocate a state of n qubits (1 <= n <= 34) on the current CUDA device and
 * set it to |0...0> (recorded; see sv_reset).  Defining passage: Sec. III-A,
 * an n-qubit state is a vector of 2^n complex amplitudes; Sec. IV-A starts
 * every circuit from the all-zero basis state.  The library owns the memory; it uses its own stream.
 * Errors: SV_ERR_ARG (n, dt, out), SV_ERR_OOM, SV_ERR_CUDA. */
sv_status sv_create(int n, sv_dtype dt, sv_handle *out);

/* Same (Sec. III-A state, Sec. IV-A initial |0...0>), on a caller-owned
 * device buffer of `bytes` >= 2^n * sizeof(amp),
 * 256-byte aligned, and the caller's stream (NULL = legacy default stream).
 * The buffer must outlive the handle; sv_destroy does not free it.
 * The state is set to |0...0>. */
sv_status sv_create_on(int n, sv_dtype dt, void *dev_buf, size_t bytes,
                       void *cuda_stream, sv_handle *out);

/* Free the handle (and the state, if owned).  NULL is accepted.  Ends the
 * lifetime of the Sec. III-A state vector that sv_create made; the paper's
 * simulator has no call of its own for this. */
sv_status sv_destroy(sv_handle h);

/* Set the state to |0...0> and the qubit map to the identity.  The library
 * only records the basis state (as it does at creation): the buffer is
 * written by the first call that needs it.  Until then, sv_apply_circuit
 * drops X gates whose qubit no earlier gate of the list touches (they only
 * flip a bit of the recorded basis index) and its first register-stage pass
 * generates the state instead of reading the buffer.  sv_info with dev_amps,
 * the read-outs and sv_copy_out write the buffer first, so a caller who
 * reads an adopted buffer directly calls sv_info before doing so. */
sv_status sv_reset(sv_handle h);

/* Number of qubits, dtype, and device address of the state buffer.  The
 * buffer holds amplitudes in PHYSICAL order; see sv_qubit_map.  Asking for
 * dev_amps writes a recorded basis state into the buffer (see sv_reset). */
sv_status sv_info(sv_handle h, int *n, sv_dtype *dt, void **dev_amps);

/* Physical bit position of each logical qubit (array of n ints).  SWAP gates
 * are absorbed into this map in partitioned modes (Sec. III-B keeps a
 * logical-to-physical qubit mapping updated after each SWAP). */
sv_status sv_qubit_map(sv_handle h, int *host_phys_of_logical);

/* ---- applying gates --------------------------------------------------- */

/* Apply gates g[0..m-1] in order.  cfg may be NULL (defaults).  Defining
 * passage: Algorithm 1 (Sec. III-A) applied gate by gate, each gate's 2x2
 * matrix on the amplitude pairs (j, j + 2^t) and a controlled gate only where
 * bit c of j is 1; Eq. 1 states that this equals multiplying the state by
 * I x .. x U x .. x I.  The partitioned modes follow Sec. III-B (deferred
 * local gates applied block by block, global qubits made local) and give the
 * same result up to floating-point rounding.
 * Partitioned modes keep the compiled programmes (host and device copies) of
 * the last 8 distinct keys on the handle; a key is the whole gate list, the
 * configuration and the qubit map at the call.  A repeated key skips the
 * planning, compilation and upload, never any amplitude arithmetic.  The
 * programmes are freed with the handle.
 * Errors: SV_ERR_ARG with the index of the first bad gate in the message
 * (qubit out of range, control == target, unknown kind, nonzero reserved,
 * log2den outside 0..62); nothing is applied in that case. */
sv_status sv_apply_circuit(sv_handle h, const sv_gate *host_gates, size_t m,
                           const sv_config *cfg);

/* Counters of the last sv_apply_circuit. */
sv_status sv_last_stats(sv_handle h, sv_stats *out);

/* Outcomes (0 or 1, in list order) of the SV_MEASURE gates of the last
 * sv_apply_circuit: the first min(cap, count) go to host_out (may be NULL
 * when cap is 0) and their number to *count.  Synchronises the handle's
 * stream.  The outcome rule is the one of Sec. IV-A's measured bitstring
 * (inverse CDF over the qubit's two values with the caller's u), applied
 * one qubit at a time with collapse.  Errors: SV_ERR_ARG, SV_ERR_CUDA. */
sv_status sv_last_measurements(sv_handle h, uint8_t *host_out, size_t cap, size_t *count);

/* ---- batches: many independent circuits in one launch ------------------ */

/* One circuit of a batch: n qubits (1..24) starting from |0...0>, its gate
 * list (caller-owned, read during sv_batch_create only) and the logical
 * qubits whose marginal is read out. */
typedef struct sv_batch_item {
    int32_t n;
    int32_t reserved;
    const sv_gate *gates;
    size_t m;
    uint64_t qubit_mask;
} sv_batch_item;

typedef struct sv_batch_state *sv_batch;

/* Plan every item (tiles of 2^13 complex64 amplitudes; smaller circuits are
 * padded with untouched qubits), allocate all states, and capture one CUDA
 * graph that runs the whole batch as a single persistent launch: CTAs take
 * items from a queue ordered by decreasing cost, apply all their passes and
 * reduce the FP64 marginal of the read-out qubits to its most probable
 * outcome.  cfg may be NULL; cfg->chunk_qubits (4..11) sets the bulk-copy
 * unit, and SV_FLAG_NO_DIAG_MERGE, SV_FLAG_EARLY_DIAG, SV_FLAG_GREEDY_ONLY and
 * SV_FLAG_NARROW_FIRST act as for sv_apply_circuit (each item's first pass
 * generates its starting state) (SV_FLAG_PAPER_SWAP is refused with
 * SV_ERR_UNSUPPORTED).  Errors: SV_ERR_ARG (bad item), SV_ERR_UNSUPPORTED (a pass the
 * register-stage kernel cannot run), SV_ERR_OOM, SV_ERR_CUDA. */
sv_status sv_batch_create(const sv_batch_item *items, size_t count, const sv_config *cfg,
                          sv_batch *out);

/* Replay the batch (every state restarts from |0...0>) and wait for it.
 * host_idx[i] / host_p[i] (either may be NULL) receive item i's most probable
 * outcome (lowest index among exact ties; bit j = j-th lowest qubit of its
 * mask) and that outcome's probability; *ms (may be NULL) the launch's device
 * time measured with CUDA events. */
sv_status sv_batch_run(sv_batch b, uint64_t *host_idx, double *host_p, double *ms);

/* Items, HBM/L2 sweeps and their algorithmic bytes (2 x 2^n x 8 per sweep). */
sv_status sv_batch_info(sv_batch b, size_t *count, int *passes, double *sweep_bytes);

sv_status sv_batch_destroy(sv_batch b);

/* sv_batch_create + sv_batch_run + sv_batch_destroy. */
sv_status sv_apply_circuit_batch(const sv_batch_item *items, size_t count, const sv_config *cfg,
                                 uint64_t *host_idx, double *host_p);

/* Measure the batch for every chunk width c in 4..7, each with the
 * automatic and with a forced split of instances of 16 qubits or more
 * (batch_split 0 and 16), and for c in 5..7 also with SV_FLAG_NARROW_FIRST
 * (one warm-up run and three timed runs each, median), and return the
 * fastest configuration in *best (and its time in *best_ms, may be NULL). */
sv_status sv_batch_autotune(const sv_batch_item *items, size_t count, sv_config *best,
                            double *best_ms);

/* ---- autotuning --------------------------------------------------------- */

/* Run the circuit under each candidate configuration (execution mode:
 * per-gate for small n, register-stage tiles, tensor-core fused tiles; chunk
 * width c; for complex128 the tile width k; diagonal placement
 * (SV_FLAG_EARLY_DIAG), a narrow first pass (SV_FLAG_NARROW_FIRST), L2 block
 * groups (SV_FLAG_L2_BLOCKS) when the state exceeds L2), one warm-up and three timed runs
 * each from |0...0> (the paper keeps the fastest block size, median of three
 * runs, Sec. IV-B), and return the fastest in *best and its median device
 * time in *best_ms (may be NULL).  The handle's state is overwritten and left
 * at |0...0>.  cache_path (may be NULL) names a text file of earlier results
 * keyed by the circuit's structure (kinds and qubits, not angles), n and the
 * dtype: a hit returns without timing; a new result is appended. */
sv_status sv_autotune(sv_handle h, const sv_gate *host_gates, size_t m, const char *cache_path,
                      sv_config *best, double *best_ms);

/* ---- reading out (Sec. IV-A: the measured bitstring) ------------------ */

/* Marginal probabilities over the logical qubits in `qubit_mask`, computed
 * in FP64 from the amplitudes and renormalised by their total.  Output index
 * bit j is the j-th lowest qubit of the mask; host_out holds
 * 2^popcount(mask) doubles.  Errors: SV_ERR_ARG (mask empty or beyond n,
 * popcount > 30), SV_ERR_OOM. */
sv_status sv_probabilities(sv_handle h, uint64_t qubit_mask, double *host_out);

/* Same, into a caller-owned device buffer of 2^popcount(mask) doubles;
 * returns without synchronising. */
sv_status sv_probabilities_device(sv_handle h, uint64_t qubit_mask, double *dev_out);

/* Allocation-free variant of sv_probabilities_device.  The paper has no
 * counterpart; it exists for callers that cannot call cudaMalloc when they
 * read a state out (a runtime that reserves all device memory up front and
 * forbids further allocation, or code that must not take the device-wide
 * synchronisation cudaMalloc/cudaFree may cause).  Its result agrees with
 * sv_probabilities_device to about 1e-13 (another summation order and, for
 * SV_C64, squares formed in FP64), not bit for bit.
 *   dev_amps  the state, 2^n amplitudes of dtype dt in physical order
 *             (e.g. the buffer of sv_info), 16-byte aligned, read only;
 *   host_phys_of_logical  n ints, the physical bit of each logical qubit
 *             (sv_qubit_map), or NULL for the identity;
 *   dev_out   2^popcount(mask) doubles, caller-owned device memory;
 *   cuda_stream  stream the kernels are enqueued on (NULL = legacy default);
 *             the call returns without synchronising.
 * Partial sums live in a fixed 1 MiB + 8 KiB device array compiled into
 * the library (held by every GPU that loads it until the process exits);
 * it holds at most 2^17 partial sums, and the reduction is split so that it
 * fits for every mask of up to 30 qubits.  The first call on each device
 * looks the array's address up (cudaGetSymbolAddress) with that device
 * current; make that first call before any stream capture.  All calls share
 * the array and leave their partial sums in it; nothing needs clearing, but
 * calls that overlap on the GPU race on it and must be ordered by the
 * caller.  The array's address stays valid until the device is reset: do
 * not call this after a cudaDeviceReset of that device in the same process.
 * Allocates no memory (no cudaMalloc / cudaFree).  Errors:
 * SV_ERR_ARG (NULL pointer, n outside 1..34, mask empty, beyond n or over
 * 30 qubits, map not a permutation, misaligned state), SV_ERR_CUDA. */
sv_status sv_marginal_noalloc(const void *dev_amps, int n, sv_dtype dt,
                              const int *host_phys_of_logical, uint64_t qubit_mask,
                              double *dev_out, void *cuda_stream);

/* Most probable outcome of the marginal over `qubit_mask` (lowest index
 * among exact ties) and its probability (p_out may be NULL). */
sv_status sv_argmax(sv_handle h, uint64_t qubit_mask, uint64_t *host_idx,
                    double *host_p);

/* Inverse-CDF sampling of the marginal over `qubit_mask`, one outcome per
 * caller-supplied uniform u[s] in [0,1): the smallest i with C_i > u*C_last,
 * where C is the inclusive CDF accumulated in blocks of 1024 outcomes
 * (in-block sums in index order, block totals in block order). */
sv_status sv_sample(sv_handle h, uint64_t qubit_mask, const double *host_u,
                    size_t shots, uint64_t *host_out);

/* Copy the amplitudes, in LOGICAL qubit order, to / from host memory of
 * 2^n * sizeof(amp) bytes.  Amplitude j belongs to the basis state whose bit
 * q is qubit q (Algorithm 1's stride 2^t, Sec. III-A); the logical order is
 * the one Sec. III-B restores by undoing its logical-to-physical qubit map.  sv_copy_out may physically reorder the state
 * to make the qubit map the identity first (results are unchanged). */
sv_status sv_copy_out(sv_handle h, void *host_amps);
sv_status sv_copy_in(sv_handle h, const void *host_amps);

/* ---- timing recorder ---------------------------------------------------- */

/* Kernel families named in launch records. */
enum {
    SV_KERNEL_PERGATE = 0,  /* one gate, one HBM sweep                       */
    SV_KERNEL_TILE = 1,     /* one tile pass (shared-memory programme)        */
    SV_KERNEL_REMAP = 2,    /* explicit qubit-remap permutation pass           */
    SV_KERNEL_FUSED = 3,    /* tile pass with tensor-core fused blocks         */
    SV_KERNEL_L2BLOCK = 4   /* several register-stage tile passes run block by
                               block through L2 (SV_FLAG_L2_BLOCKS): k holds
                               the block qubits, nops the passes             */
};

/* One kernel launch of sv_apply_circuit, timed with CUDA events recorded on
 * the handle's stream right before and after the launch. */
typedef struct sv_launch_record {
    int32_t kind;      /* SV_KERNEL_*                                          */
    int32_t pass;      /* launch index within its sv_apply_circuit call        */
    int32_t n;         /* qubits                                              */
    int32_t k;         /* tile qubits (0 for per-gate)                         */
    int32_t nops;      /* programme steps of the pass (1 for per-gate)         */
    int32_t ngates;    /* circuit gates the launch applies                     */
    int32_t dtype;     /* sv_dtype                                             */
    int32_t gate_kind; /* per-gate: the gate kind; tile kernels: -1 generic,
                          -2 register-stage, -3 fused (tensor cores);
                          remap: -4; L2 block group: -5                       */
    double bytes;      /* algorithmic bytes: 2 * 2^n * sizeof(amp) per sweep,
                          the touched share for per-gate diagonal/SWAP, the
                          moved share for a remap; an L2 block group counts
                          its first read and last write                       */
    double ms;         /* measured duration (0 in planning descriptors)        */
    uint64_t feat;     /* tile: bit mask of the physical qubits in the tile;
                          per-gate: bit mask of the gate's qubits; remap: bit
                          mask of the exchanged bits                           */
    int32_t c;         /* tile: chunk qubits (contiguous low bits)             */
    int32_t stages;    /* register-stage / fused: stage layouts                */
    int32_t blocks;    /* fused: 32x32 tensor-core blocks                      */
    int32_t nins;      /* register-stage / fused: programme instructions       */
    int32_t nfactors;  /* register-stage / fused: diagonal factor applications */
    int32_t generated; /* 1: a register-stage pass that generated a recorded
                          basis state (written only: bytes count the write)  */
} sv_launch_record;

/* Start (enable=1) or stop (0) recording launch records on this handle.
 * Starting clears earlier records.  Recording adds two event records per
 * launch and does not change what the kernels compute. */
sv_status sv_profile(sv_handle h, int enable);

/* Synchronise the handle's stream and copy up to `cap` records (oldest
 * first) into host_out; *count receives the number available.  Records
 * that were copied are removed. */
sv_status sv_profile_read(sv_handle h, sv_launch_record *host_out, size_t cap, size_t *count);

/* Number of kernels this library has launched in the process so far. */
uint64_t sv_launch_count(void);

/* ---- cost model and learned planner ------------------------------------- */

/* A small MLP predicts the duration of one launch from a feature vector
 * that sv_cost_features derives from a launch record.  Layers:
 * SV_COST_FEATURES -> 64 -> ReLU -> 64 -> ReLU -> 1, FP32.  Parameters are one
 * flat vector (row-major): W1[F][64], b1[64], W2[64][64], b2[64], W3[64], b3,
 * with z1_j = b1_j + sum_i x_i W1[i][j].  The output estimates
 * ln(ms / (bytes / 1e9)), the log of the launch time per algorithmic GB.
 * Training minimises the mean squared error with Adam; forward, backward
 * and update run in this library's kernels.  The model only ranks schedules,
 * so it never changes what a plan computes. */
#define SV_COST_FEATURES 52
#define SV_COST_HIDDEN 64
#define SV_COST_PARAMS 7617

typedef struct sv_cost_model_s *sv_cost_model;

typedef struct sv_train_config {
    int32_t epochs;   /* passes over the data (default 100)                    */
    int32_t batch;    /* samples per Adam step (default 4096)                  */
    float lr;         /* default 1e-3                                          */
    float beta1;      /* default 0.9                                           */
    float beta2;      /* default 0.999                                         */
    float eps;        /* default 1e-8                                          */
    uint64_t seed;    /* shuffling (SplitMix64 Fisher-Yates per epoch)         */
    int32_t reserved[6];
} sv_train_config;

/* Feature vector of one launch record (SV_COST_FEATURES floats): physical
 * qubit mask bits 0..31, stride class of the highest qubit (<5, 5-9,
 * 10..k-1, >=k), a pass that generates its state, complex128, kernel
 * family, and scaled logs of gates, instructions, stages, blocks and
 * factors, plus c, n, k and k - c.  Host only. */
sv_status sv_cost_features(const sv_launch_record *rec, float *host_out);

/* Create a model on the current device with He-uniform weights drawn from
 * `seed` (SplitMix64), zero biases and zero Adam moments. */
sv_status sv_cost_model_create(uint64_t seed, sv_cost_model *out);
sv_status sv_cost_model_destroy(sv_cost_model m);
/* SV_COST_PARAMS floats, layout above. */
sv_status sv_cost_model_get_params(sv_cost_model m, float *host_params);
sv_status sv_cost_model_set_params(sv_cost_model m, const float *host_params);
/* y[i] = network(x[i]) for `count` rows of SV_COST_FEATURES floats. */
sv_status sv_cost_model_predict(sv_cost_model m, const float *host_x, size_t count,
                                float *host_y);
/* Gradient of the mean squared error over all `count` samples with respect
 * to the parameters (SV_COST_PARAMS floats) and the loss itself. */
sv_status sv_cost_model_gradient(sv_cost_model m, const float *host_x, const float *host_t,
                                 size_t count, float *host_grad, double *host_loss);
/* Adam training; host_epoch_loss (may be NULL) receives the mean training
 * loss of each epoch.  cfg NULL or zero fields = defaults. */
sv_status sv_cost_model_train(sv_cost_model m, const float *host_x, const float *host_t,
                              size_t count, const sv_train_config *cfg,
                              float *host_epoch_loss);
/* Binary file: "SVCM", version, F, hidden, parameter count, parameters. */
sv_status sv_cost_model_save(sv_cost_model m, const char *path);
sv_status sv_cost_model_load(const char *path, sv_cost_model *out);

/* Attach a model to a handle (not owned; NULL detaches).  With
 * sv_config.planner = SV_PLANNER_LEARNED, sv_apply_circuit then scores
 * candidate schedules (chunk width, tile gathering or the paper's explicit
 * remaps, and per pass the register-stage or the fused tensor-core kernel)
 * by the model's predicted time and runs the cheapest.  Without a model, or
 * when sv_planner_judge found the greedy plan faster for this circuit
 * structure, the greedy plan of the configuration runs instead. */
sv_status sv_set_cost_model(sv_handle h, sv_cost_model m);

/* Outcome of a learned-planner decision. */
typedef struct sv_plan_choice {
    int32_t chunk_qubits;        /* c of the chosen candidate                  */
    int32_t paper_swap;          /* 1: explicit remaps (Sec. III-B literal)    */
    int32_t passes;              /* tile passes of the chosen plan             */
    int32_t remaps;              /* remap passes of the chosen plan            */
    int32_t fused_passes;        /* passes given to the fused kernel           */
    int32_t candidates;          /* candidate passes scored                    */
    double predicted_ms;         /* predicted time of the chosen plan          */
    double greedy_predicted_ms;  /* predicted time of the greedy plan          */
    double learned_ms;           /* measured by sv_planner_judge, else 0       */
    double greedy_ms;            /* measured by sv_planner_judge, else 0       */
    int32_t verdict;             /* planner sv_planner_judge kept (sv_planner) */
    int32_t early_diag;          /* 1: the chosen plan keeps diagonal gates in
                                    the first pass where they are ready       */
    int32_t rule_kernels;        /* 1: sv_planner_judge measured the chosen
                                    options faster with the greedy rule's
                                    kernel per pass and kept those            */
    int32_t narrow_first;        /* 1: the chosen plan's first pass gathers
                                    16-amplitude chunks (SV_FLAG_NARROW_FIRST) */
    double rule_ms;              /* measured by sv_planner_judge: the chosen
                                    options with the rule's kernels (0 if the
                                    model chose the same kernels)             */
    int32_t reserved[2];
} sv_plan_choice;

/* The learned planner's choice for this gate list (no kernel runs). */
sv_status sv_learned_plan(sv_handle h, const sv_gate *host_gates, size_t m,
                          const sv_config *cfg, sv_plan_choice *out);

/* Run the greedy plan of cfg and the learned plan from |0...0>, once to warm
 * up and three times each under CUDA events, and keep the faster (median)
 * for this circuit structure on this handle.  Where the model picked a
 * kernel per pass other than the greedy rule's, the learned plan's options
 * (tile and chunk widths, remaps, diagonal placement) are also timed with
 * the rule's kernels, and the faster kernel choice becomes the learned plan.
 * The state is reset to |0...0> afterwards. */
sv_status sv_planner_judge(sv_handle h, const sv_gate *host_gates, size_t m,
                           const sv_config *cfg, sv_plan_choice *out);

/* ---- diagnostics ------------------------------------------------------ */

/* Describe, as JSON text, the programme sv_apply_circuit would run in a
 * partitioned mode for n qubits of dtype dt, starting from the qubit map
 * host_phys_of_logical (NULL = identity): the passes (tile qubits, gathered
 * physical bits, gate steps, merged diagonal terms) and, per pass, the
 * register-stage programme or the reason the generic tile kernel is used.
 * Host only: it plans but calls no CUDA function.  Writes at most cap bytes
 * (NUL-terminated) to host_buf and the full length to *len.  The planner is
 * the paper's partitioning (Sec. III-B); the format is this library's.
 * The list is planned as given: the X gates sv_apply_circuit drops from a
 * recorded basis state (see sv_reset) are planned like other gates. */
sv_status sv_plan_export(int n, sv_dtype dt, const int *host_phys_of_logical,
                         const sv_gate *host_gates, size_t m, const sv_config *cfg,
                         char *host_buf, size_t cap, size_t *len);

/* Message of the last failed call on this thread ("" if none). */
/* ---- failure paths, exercised from the host ------------------------------ */

/* Host-side fault injection for tests of the error paths (the paper has no
 * counterpart).  After `after` further calls at `site` (0: the next one), one
 * call fails as if the CUDA runtime had refused it, then the site is off
 * again; after < 0 turns the site off at once.  Sites:
 *   SV_FAULT_ALLOC   a device allocation: the call returns SV_ERR_OOM
 *   SV_FAULT_UPLOAD  a programme upload to the device: SV_ERR_CUDA
 *   SV_FAULT_LAUNCH  a kernel launch, refused before it starts: SV_ERR_CUDA
 * A call that fails before any kernel wrote the state leaves the state as it
 * was; one that fails after some of its kernels ran leaves it undefined (as a
 * real CUDA failure would), and sv_reset or sv_copy_in make it usable again.
 * The setting is process-wide.  Errors: SV_ERR_ARG (unknown site). */
enum { SV_FAULT_ALLOC = 0, SV_FAULT_UPLOAD = 1, SV_FAULT_LAUNCH = 2 };
sv_status sv_fault_inject(int site, int after);

/* Set the handle's device error word from the host, as a tile kernel does
 * when one of its bounded waits gives up.  The next call that returns data
 * to the host (sv_probabilities, sv_argmax, sv_sample, sv_copy_out,
 * sv_last_measurements) reports SV_ERR_TIMEOUT and clears the word; the
 * state is then undefined.  Lets tests reach the timeout reporting without a
 * device wait running out.  Errors: SV_ERR_ARG, SV_ERR_OOM, SV_ERR_CUDA. */
sv_status sv_fault_raise_device_flag(sv_handle h);

const char *sv_last_error(void);

/* Library version string. */
const char *sv_version(void);

#ifdef __cplusplus
}
#endif

#endif /* LIBSV_SV_H_ */
