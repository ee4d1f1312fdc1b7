// Fused tile kernel (complex64): register stages with 32x32 blocks on tensor cores.
//
// One CTA per SM (persistent), 256 threads, two 64 KiB tile buffers: while
// the CTA works on tile i in one buffer, the bulk copies (TMA) of tile i+1
// fill the other and the write-back of tile i-1 drains.  In a stage each
// thread holds 32 amplitudes (register bits 0..4); a fused block multiplies
// them by a 32x32 complex matrix U formed on the host in FP64 from every gate
// of the stage that acts on register bits only (Sec. III-B's deferred local
// gates, applied to a block at once).  The product runs on the tensor cores:
//   * each thread writes its row of A = [Re x | Im x] (64 values) to tensor
//     memory as TF32 hi and lo parts (tcgen05.st);
//   * one thread issues tcgen05.mma kind::tf32 with A from tensor memory and
//     B = Re U / Im U (hi, lo) from shared memory: Re y = A_re U_re^T -
//     A_im U_im^T, Im y = A_re U_im^T + A_im U_re^T, each as the three
//     split-precision products hi*hi + hi*lo + lo*hi accumulated in FP32;
//   * the accumulator is read back with tcgen05.ld.
// Diagonal factors that depend on thread or tile bits (the twiddles between
// blocks) and gates on tile bits 1..3 (warp shuffles) run on the CUDA cores.
#include <algorithm>

#include "common.h"
#include "plan.h"
#include "stagecomp.h"
#include "tiledev.cuh"
#include "tileprog.h"

namespace sv {
namespace {

using namespace tiledev;

constexpr int kTileAmps = 1 << kT2Qubits;
constexpr uint32_t kTileBytes = kTileAmps * 8u;
constexpr uint32_t kBlockBytes = kBlockFloats * 4u;  // 16 KiB
constexpr int kTabN = 256;                           // four 8-bit phase tables
constexpr size_t kOffBuf1 = kTileBytes;
constexpr size_t kOffBlk = 2 * (size_t)kTileBytes;
constexpr size_t kOffTab = kOffBlk + (size_t)kMaxBlocks * kBlockBytes;
constexpr size_t kOffLin = kOffTab + 4 * kTabN * 8;
constexpr size_t kOffCst = kOffLin + (size_t)kT2MaxRuns * 16 * 4;
constexpr size_t kOffBar = kOffCst + (size_t)kT2MaxRuns * 4;
constexpr size_t kOffChunk = kOffBar + 128;  // chunk offsets >> c (<= 512)
constexpr size_t kSmemBytes = kOffChunk + 2048;
constexpr uint32_t kTmemCols = 512;

struct T3Args {
    uint64_t gmask, ntiles;
    int c, nins, nruns, ntterms, nblocks;
    int slot_phys[kMaxTileQubits];
    const int4 *ins;
    const int4 *stages;
    const float4 *mats;
    const int4 *fac;
    const uint32_t *stat;
    const T2TileTerm *tterms;
    const float *blocks;
    const float2 *tables;  // 4 x 256: e^{2 pi i j / 2^8}, ^16, ^24, ^32
    int *err;
    const double *norm_in;  // per-CTA squared norms of the previous fused pass (or NULL)
    int norm_in_count;
    double *norm_out;       // this pass's per-CTA squared norms
};

// ---------------------------------------------------------------- tensor memory / MMA
__device__ __forceinline__ void tc_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tmem_st32(uint32_t taddr, const uint32_t (&v)[32]) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
        "%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,%32};" ::"r"(taddr),
        "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7]),
        "r"(v[8]), "r"(v[9]), "r"(v[10]), "r"(v[11]), "r"(v[12]), "r"(v[13]), "r"(v[14]),
        "r"(v[15]), "r"(v[16]), "r"(v[17]), "r"(v[18]), "r"(v[19]), "r"(v[20]), "r"(v[21]),
        "r"(v[22]), "r"(v[23]), "r"(v[24]), "r"(v[25]), "r"(v[26]), "r"(v[27]), "r"(v[28]),
        "r"(v[29]), "r"(v[30]), "r"(v[31])
        : "memory");
}
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&v)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,"
        "%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
          "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]),
          "=r"(v[14]), "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]),
          "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]), "=r"(v[25]),
          "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
        : "r"(taddr)
        : "memory");
}
__device__ __forceinline__ void tmem_wait_st() {
    asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_wait_ld() {
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}
// Shared-memory matrix descriptor: K-major, no swizzle; lbo = byte stride of
// core matrices along K, sbo = byte stride of 8-row groups along N.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = (uint64_t)((addr >> 4) & 0x3FFFu);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;  // descriptor version (sm_100 family)
    return d;
}
__device__ __forceinline__ void mma_tf32(uint32_t dtm, uint32_t atm, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n}\n" ::"r"(dtm),
        "r"(atm), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}
__device__ __forceinline__ void mma_commit(uint64_t *bar) {
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            saddr(bar))
        : "memory");
}
__device__ __forceinline__ uint32_t tf32_bits(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}

// e^{2 pi i u / 2^32} from the four 8-bit tables
__device__ __forceinline__ float2 phase_factor(const float2 *tab, uint32_t u) {
    const float2 a = tab[u >> 24], b = tab[kTabN + ((u >> 16) & 255u)];
    const float2 c = tab[2 * kTabN + ((u >> 8) & 255u)], d = tab[3 * kTabN + (u & 255u)];
    return cx(cx(a, b), cx(c, d));
}

__device__ __forceinline__ void issue_tile_load(unsigned char *buf, const float *state, uint64_t base,
                                                const T3Args &a, uint64_t *bar, int lane,
                                                const uint32_t *choff) {
    const int nchunks = 1 << (kT2Qubits - a.c);
    const uint32_t chunk_bytes = 8u << a.c;
    if (lane == 0) {
        fence_async_smem();
        mbar_expect_tx(bar, kTileBytes);
    }
    __syncwarp();
    for (int j = lane; j < nchunks; j += 32) {
        const uint64_t off = (uint64_t)choff[j] << a.c;
        bulk_g2s(buf + (size_t)j * chunk_bytes, state + 2 * (base + off), chunk_bytes, bar);
    }
}

__device__ __forceinline__ void issue_tile_store(float *state, const unsigned char *buf,
                                                 uint64_t base, const T3Args &a, int lane,
                                                 const uint32_t *choff) {
    const int nchunks = 1 << (kT2Qubits - a.c);
    const uint32_t chunk_bytes = 8u << a.c;
    for (int j = lane; j < nchunks; j += 32) {
        const uint64_t off = (uint64_t)choff[j] << a.c;
        bulk_s2g(state + 2 * (base + off), buf + (size_t)j * chunk_bytes, chunk_bytes);
    }
    bulk_commit();
}

__global__ void __launch_bounds__(kT3Threads, 1) k_tile3(float *__restrict__ state, const T3Args a) {
    extern __shared__ __align__(1024) unsigned char sm[];
    float2 *tab = reinterpret_cast<float2 *>(sm + kOffTab);
    uint32_t *lin = reinterpret_cast<uint32_t *>(sm + kOffLin);
    uint32_t *cst = reinterpret_cast<uint32_t *>(sm + kOffCst);
    uint64_t *full = reinterpret_cast<uint64_t *>(sm + kOffBar);       // [2]
    uint64_t *mma_bar = reinterpret_cast<uint64_t *>(sm + kOffBar + 16);
    uint64_t *slot_bar = reinterpret_cast<uint64_t *>(sm + kOffBar + 24);  // [kMaxBlocks]
    uint32_t *tslot = reinterpret_cast<uint32_t *>(sm + kOffBar + 24 + 8 * kMaxBlocks);
    uint32_t *choff = reinterpret_cast<uint32_t *>(sm + kOffChunk);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    for (int i = tid; i < 4 * kTabN; i += blockDim.x) tab[i] = a.tables[i];
    for (int j = tid; j < (1 << (kT2Qubits - a.c)); j += blockDim.x) {
        uint64_t off = 0;
        for (int b = 0; b < kT2Qubits - a.c; b++)
            if ((j >> b) & 1) off |= UINT64_C(1) << a.slot_phys[a.c + b];
        choff[j] = (uint32_t)(off >> a.c);
    }
    if (tid == 0) {
        mbar_init(&full[0], 1);
        mbar_init(&full[1], 1);
        mbar_init(mma_bar, 1);
        for (int i = 0; i < kMaxBlocks; i++) mbar_init(&slot_bar[i], 1);
        fence_mbar_init();
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         saddr(tslot)),
                     "r"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tbase = *tslot;
    const uint32_t lane_off = (uint32_t)(32 * (warp & 3)) << 16;
    // norm correction of the previous fused pass: 1 / sqrt(sum of its per-CTA squared norms)
    double s_norm = 1.0;
    if (a.norm_in) {
        double nn = 0.0;
        for (int i = 0; i < a.norm_in_count; i++) nn += a.norm_in[i];
        if (nn > 0.0) s_norm = 1.0 / sqrt(nn);
    }
    double nacc = 0.0;
    const int half = warp >> 2;
    bool failed = false;

    // Blocks: up to kMaxBlocks stay resident in their slots; otherwise block
    // use u (counted over this CTA's tiles) sits in slot u % kMaxBlocks and the
    // copy for use u + kMaxBlocks starts as soon as use u's products are done.
    const bool resident = a.nblocks <= kMaxBlocks;
    const uint64_t my_tiles =
        a.ntiles > blockIdx.x ? (a.ntiles - blockIdx.x + gridDim.x - 1) / gridDim.x : 0;
    const uint64_t total_uses = my_tiles * (uint64_t)a.nblocks;
    auto load_block = [&](int slot, int blk) {
        fence_async_smem();
        mbar_expect_tx(&slot_bar[slot], kBlockBytes);
        bulk_g2s(sm + kOffBlk + (size_t)slot * kBlockBytes, a.blocks + (size_t)blk * kBlockFloats,
                 kBlockBytes, &slot_bar[slot]);
    };
    if (tid == 0 && a.nblocks > 0) {
        if (resident) {
            for (int b = 0; b < a.nblocks; b++) load_block(b, b);
        } else {
            for (int u = 0; u < kMaxBlocks && (uint64_t)u < total_uses; u++) load_block(u, u % a.nblocks);
        }
    }
    if (resident && a.nblocks > 0) {
        bool to = false;
        for (int b = 0; b < a.nblocks; b++) to |= !mbar_wait(&slot_bar[b], 0);
        failed = __syncthreads_or(to);
    }
    uint64_t use = 0;

    uint32_t mma_phase = 0;
    uint64_t tile = blockIdx.x;
    if (!failed && warp == 0 && tile < a.ntiles)
        issue_tile_load(sm, state, pdep(tile, a.gmask), a, &full[0], lane, choff);

    for (int it = 0; !failed && tile < a.ntiles; it++, tile += gridDim.x) {
        const int b = it & 1;
        unsigned char *buf = sm + (b ? kOffBuf1 : 0);
        float4 *tile4 = reinterpret_cast<float4 *>(buf);
        const uint64_t base = pdep(tile, a.gmask);
        // prefetch the next tile into the other buffer once its write-back has been read
        const uint64_t next = tile + gridDim.x;
        if (warp == 0 && next < a.ntiles) {
            bulk_wait_read();
            __syncwarp();
            issue_tile_load(sm + (b ? 0 : kOffBuf1), state, pdep(next, a.gmask), a, &full[b ^ 1],
                            lane, choff);
        }
        for (int i = tid; i < a.nruns * 16; i += blockDim.x) lin[i] = 0u;
        for (int i = tid; i < a.nruns; i += blockDim.x) cst[i] = 0u;
        __syncthreads();
        for (int i = tid; i < a.ntterms; i += blockDim.x) {
            const T2TileTerm t = a.tterms[i];
            bool on = (base >> t.g0) & 1;
            if (t.g1 >= 0) on = on && ((base >> t.g1) & 1);
            if (on) atomicAdd(t.tb >= 0 ? &lin[t.run * 16 + t.tb] : &cst[t.run], t.theta);
        }
        const bool to = !mbar_wait(&full[b], (uint32_t)(it >> 1) & 1u);
        if (__syncthreads_or(to)) {
            failed = true;
            break;
        }

        Regs r;
        int bt = 0, s1 = 0, s2 = 0, s3 = 0, s4 = 0;
        int stage = 0;
        bool live = false;
        auto sidx = [&](int q) {
            return (bt + ((q & 1) ? s1 : 0) + ((q & 2) ? s2 : 0) + ((q & 4) ? s3 : 0) +
                    ((q & 8) ? s4 : 0)) >> 1;
        };
        for (int pc = 0; pc < a.nins && !failed; pc++) {
            const int4 w = __ldg(a.ins + pc);
            const int op = w.x & 0xff;
            if (op == T2_STAGE) {
                if (live) {
                    // every warp has read the previous layout before any overwrites it
                    __syncthreads();
#pragma unroll
                    for (int q = 0; q < kNP; q++)
                        tile4[sidx(q)] = make_float4(r.re[q].x, r.re[q].y, r.im[q].x, r.im[q].y);
                    __syncthreads();
                }
                stage = w.w;
                const int4 st = __ldg(a.stages + stage);
                auto tbyte = [&](int i) {
                    const int word = i < 4 ? st.x : i < 8 ? st.y : i < 12 ? st.z : st.w;
                    return (word >> (8 * (i & 3))) & 0xff;
                };
                bt = 0;
#pragma unroll
                for (int t = 0; t < 8; t++) bt |= ((tid >> t) & 1) << tbyte(5 + t);
                s1 = 1 << tbyte(1);
                s2 = 1 << tbyte(2);
                s3 = 1 << tbyte(3);
                s4 = 1 << tbyte(4);
                if (live) {
#pragma unroll
                    for (int q = 0; q < kNP; q++) {
                        const float4 v = tile4[sidx(q)];
                        r.re[q] = make_float2(v.x, v.y);
                        r.im[q] = make_float2(v.z, v.w);
                    }
                } else {
#pragma unroll
                    for (int q = 0; q < kNP; q++) {
                        const float4 v = tile4[sidx(q)];
                        r.re[q] = make_float2(v.x, v.z);
                        r.im[q] = make_float2(v.y, v.w);
                    }
                }
                live = true;
                continue;
            }
            if (op == T2_BLOCK) {
                // A operand: this thread's row, TF32 hi at [half*64, +64), lo at 128 + that
                {
                    uint32_t h[32], l[32];
#pragma unroll
                    for (int q = 0; q < kNP; q++) {
                        const uint32_t h0 = tf32_bits(r.re[q].x), h1 = tf32_bits(r.re[q].y);
                        h[2 * q] = h0;
                        h[2 * q + 1] = h1;
                        l[2 * q] = __float_as_uint(r.re[q].x - __uint_as_float(h0));
                        l[2 * q + 1] = __float_as_uint(r.re[q].y - __uint_as_float(h1));
                    }
                    tmem_st32(tbase + lane_off + half * 64, h);
                    tmem_st32(tbase + lane_off + 128 + half * 64, l);
#pragma unroll
                    for (int q = 0; q < kNP; q++) {
                        const uint32_t h0 = tf32_bits(r.im[q].x), h1 = tf32_bits(r.im[q].y);
                        h[2 * q] = h0;
                        h[2 * q + 1] = h1;
                        l[2 * q] = __float_as_uint(r.im[q].x - __uint_as_float(h0));
                        l[2 * q + 1] = __float_as_uint(r.im[q].y - __uint_as_float(h1));
                    }
                    tmem_st32(tbase + lane_off + half * 64 + 32, h);
                    tmem_st32(tbase + lane_off + 128 + half * 64 + 32, l);
                    tmem_wait_st();
                }
                int slot = w.w;
                if (!resident) {
                    slot = (int)(use % kMaxBlocks);
                    const bool sto = !mbar_wait(&slot_bar[slot], (uint32_t)(use / kMaxBlocks) & 1u);
                    if (sto) failed = true;
                }
                tc_fence_before();
                if (__syncthreads_or(failed)) {
                    failed = true;
                    break;
                }
                if (tid == 0) {
                    tc_fence_after();
                    // D f32, A tf32, B tf32, K-major, N = 32, M = 128; bit 14 negates B
                    const uint32_t idesc =
                        (1u << 4) | (2u << 7) | (2u << 10) | ((32u >> 3) << 17) | ((128u >> 4) << 24);
                    const uint32_t bblk = saddr(sm + kOffBlk) + (uint32_t)slot * kBlockBytes;
                    const uint64_t d0 = smem_desc(bblk, 128, 1024);
#pragma unroll
                    for (int hh = 0; hh < 2; hh++) {
#pragma unroll
                        for (int out = 0; out < 2; out++) {  // 0: Re y, 1: Im y
                            const uint32_t dtm = tbase + 256 + hh * 64 + out * 32;
#pragma unroll
                            for (int prod = 0; prod < 3; prod++) {  // hi*hi, hi*lo, lo*hi
#pragma unroll
                                for (int src = 0; src < 2; src++) {  // 0: Re x, 1: Im x
                                    // Re y: Re x * Re U - Im x * Im U ; Im y: Re x * Im U + Im x * Re U
                                    const bool use_im = (out == 0) ? (src == 1) : (src == 0);
                                    const uint32_t id = idesc | ((out == 0 && src == 1) ? (1u << 14) : 0u);
                                    const uint32_t acol = (prod == 2 ? 128u : 0u) + hh * 64 + src * 32;
                                    const uint32_t boff =
                                        (prod == 1 ? 2u * 4096u : 0u) + (use_im ? 4096u : 0u);
#pragma unroll
                                    for (int s = 0; s < 4; s++)
                                        mma_tf32(dtm, tbase + acol + s * 8, d0 + ((boff + s * 256) >> 4),
                                                 id, (prod | src | s) ? 1u : 0u);
                                }
                            }
                        }
                    }
                    mma_commit(mma_bar);
                }
                const bool mto = !mbar_wait(mma_bar, mma_phase);
                mma_phase ^= 1u;
                if (__syncthreads_or(mto)) {
                    mbar_wait(mma_bar, mma_phase ^ 1u);  // second bounded wait before freeing TMEM
                    failed = true;
                    break;
                }
                tc_fence_after();
                if (!resident) {
                    if (tid == 0 && use + kMaxBlocks < total_uses)
                        load_block(slot, (int)((use + kMaxBlocks) % (uint64_t)a.nblocks));
                    use++;
                }
                {
                    uint32_t v[32];
                    tmem_ld32(tbase + lane_off + 256 + half * 64, v);
                    tmem_wait_ld();
#pragma unroll
                    for (int q = 0; q < kNP; q++)
                        r.re[q] = make_float2(__uint_as_float(v[2 * q]), __uint_as_float(v[2 * q + 1]));
                    tmem_ld32(tbase + lane_off + 256 + half * 64 + 32, v);
                    tmem_wait_ld();
#pragma unroll
                    for (int q = 0; q < kNP; q++)
                        r.im[q] = make_float2(__uint_as_float(v[2 * q]), __uint_as_float(v[2 * q + 1]));
                }
                tc_fence_before();
                continue;
            }
            if (op == T2_SCALE) {
                const float4 mm = __ldg(a.mats + 2 * w.w);
                const double tot = ((double)mm.x + (double)mm.y) * s_norm;
                const float hi = (float)tot, lo = (float)(tot - (double)(float)tot);
#pragma unroll
                for (int q = 0; q < kNP; q++) {
                    r.re[q] = fma2(r.re[q], f2(hi), mul2(r.re[q], f2(lo)));
                    r.im[q] = fma2(r.im[q], f2(hi), mul2(r.im[q], f2(lo)));
                }
                continue;
            }
            if (op == T2_DIAG) {
                const int e0 = (int16_t)(w.z & 0xffff), e1 = (int16_t)(w.z >> 16);
                for (int e = e0; e < e1; e++) {
                    const int4 fd = __ldg(a.fac + e);
                    const uint32_t w0 = (uint32_t)fd.x;
                    const int run = fd.y;
                    float fr, fi;
                    if (!(w0 & 0x100u)) {
                        const int pb = (int)((w0 >> 10) & 0xfu);  // thread-bit predicate
                        if (pb && !((tid >> (pb - 1)) & 1)) continue;
                        fr = __int_as_float(fd.z);
                        fi = __int_as_float(fd.w);
                    } else {
                        uint32_t u = __ldg(a.stat + fd.z * kT3Threads + tid);
                        if (w0 & 0x200u) u += cst[run];
                        const int lr = (int)((w0 >> kFacLinShift) & 0x1fu) - 1;
                        if (lr >= 0) u += lin[run * 16 + lr];
                        uint32_t dm = (w0 >> kFacDynShift) & 0x1ffu & (uint32_t)tid;
                        while (dm) {
                            const int t = __ffs(dm) - 1;
                            dm &= dm - 1;
                            const int8_t *tbp = reinterpret_cast<const int8_t *>(a.stages + stage);
                            u += lin[run * 16 + tbp[5 + t]];
                        }
                        const float2 ff = phase_factor(tab, u);
                        fr = ff.x;
                        fi = ff.y;
                    }
                    apply_factor_any(r, (int)(w0 & 0xffu), fr, fi);
                }
                continue;
            }
            // CUDA-core gates: shuffles on lane bits, or register gates with a thread / tile control
            const int cls = (w.x >> 8) & 0xff;
            const int j = (int8_t)((w.x >> 16) & 0xff);
            const int ccls = (w.x >> 24) & 0xff;
            const int cidx = (int16_t)(w.y & 0xffff);
            bool pred = true;
            const int jc = -1;  // register-bit controls are not compiled for these kernels
            if (ccls == T2C_GLOBAL) {
                if (!((base >> cidx) & 1)) continue;
            } else if (ccls == T2C_THREAD) {
                pred = (tid >> cidx) & 1;
            }
            if (op == T2_GATE || op == T2_RGATE) {  // a real matrix runs as a general one here
                float m[8];
                const float4 m0 = __ldg(a.mats + 2 * w.w), m1 = __ldg(a.mats + 2 * w.w + 1);
                m[0] = m0.x; m[1] = m0.y; m[2] = m0.z; m[3] = m0.w;
                m[4] = m1.x; m[5] = m1.y; m[6] = m1.z; m[7] = m1.w;
                if (cls == T2C_LANE)
                    lane_gate(r, T2_GATE, j, jc, pred, m);
                else if (pred)
                    reg_gate(r, T2_GATE, j, jc, m);
                continue;
            }
            const float mz[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
            if (cls == T2C_LANE) {
                lane_gate(r, op, j, jc, pred, mz);
                continue;
            }
            if (!pred) continue;
            reg_gate(r, op, j, jc, mz);
        }
        if (failed) break;
        if (live) {
            float2 ss = make_float2(0.f, 0.f);
#pragma unroll
            for (int q = 0; q < kNP; q++) {
                ss = fma2(r.re[q], r.re[q], ss);
                ss = fma2(r.im[q], r.im[q], ss);
                tile4[sidx(q)] = make_float4(r.re[q].x, r.im[q].x, r.re[q].y, r.im[q].y);
            }
            nacc += (double)ss.x + (double)ss.y;
        }
        fence_async_smem();
        __syncthreads();
        if (warp == 0) issue_tile_store(state, buf, base, a, lane, choff);
    }
    if (failed && tid == 0) atomicExch(a.err, 1);
    if (warp == 0) asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
    tc_fence_before();
    __syncthreads();
    if (a.norm_out) {  // per-CTA squared norm, fixed reduction order
        double *red = reinterpret_cast<double *>(lin);
        red[tid] = nacc;
        __syncthreads();
        for (int w2 = kT3Threads / 2; w2; w2 >>= 1) {
            if (tid < w2) red[tid] += red[tid + w2];
            __syncthreads();
        }
        if (tid == 0) a.norm_out[blockIdx.x] = red[0];
    }
    tc_fence_after();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase),
                     "r"(kTmemCols)
                     : "memory");
}

// 4 x 256 entries: e^{2 pi i j / 2^(8 (l + 1))}, FP64 then rounded.
__global__ void k_phase_tables4(float2 *t) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= 4 * kTabN) return;
    const int l = i / kTabN, j = i % kTabN;
    const double x = (double)j * ldexp(1.0, -8 * (l + 1));
    double s, c;
    sincospi(2.0 * x, &s, &c);
    t[i] = make_float2((float)c, (float)s);
}

}  // namespace

sv_status t3_prepare(sv_state *h) {
    if (h->t3_tables) return SV_OK;
    SV_TRY(t2_prepare(h));  // error flag lives with the register-stage tables
    void *p = nullptr;
    if (dev_malloc(&p, 4 * kTabN * sizeof(float2)) != cudaSuccess) {
        cudaGetLastError();
        return fail(SV_ERR_OOM, "cannot allocate phase tables");
    }
    h->t3_tables = p;
    k_phase_tables4<<<(4 * kTabN + 255) / 256, 256, 0, h->stream>>>(reinterpret_cast<float2 *>(p));
    SV_CUDA(cudaGetLastError());
    note_launch();
    static bool configured = false;
    if (!configured) {
        SV_CUDA(cudaFuncSetAttribute(k_tile3, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)kSmemBytes));
        configured = true;
    }
    return SV_OK;
}

sv_status t3_launch(sv_state *h, const T2Pass &p, const T2Device &d, const sv_launch_record &meta) {
    SV_TRY(launch_check());
    T3Args a{};
    if (!h->norm_buf) {
        void *nb = nullptr;
        if (dev_malloc(&nb, 2 * 256 * sizeof(double)) != cudaSuccess) {
            cudaGetLastError();
            return fail(SV_ERR_OOM, "cannot allocate the norm buffer");
        }
        h->norm_buf = reinterpret_cast<double *>(nb);
        h->norm_pending = false;
    }
    const int out_idx = h->norm_pending ? (h->norm_idx ^ 1) : 0;
    a.norm_in = h->norm_pending ? h->norm_buf + 256 * h->norm_idx : nullptr;
    a.norm_in_count = h->norm_pending ? h->norm_cnt : 0;
    a.norm_out = h->norm_buf + 256 * out_idx;
    a.gmask = p.gmask;
    a.ntiles = UINT64_C(1) << (h->n - p.k);
    a.c = p.c;
    a.nins = (int)p.ins.size();
    a.nruns = p.nruns;
    a.ntterms = (int)p.tterms.size();
    a.nblocks = p.nblocks;
    for (int s = 0; s < p.k; s++) a.slot_phys[s] = p.slot_phys[s];
    a.ins = reinterpret_cast<const int4 *>(d.ins);
    a.stages = reinterpret_cast<const int4 *>(d.stages);
    a.mats = reinterpret_cast<const float4 *>(d.mats);
    a.fac = reinterpret_cast<const int4 *>(d.fac);
    a.stat = d.stat;
    a.tterms = d.tterms;
    a.blocks = d.blocks;
    a.tables = reinterpret_cast<const float2 *>(h->t3_tables);
    a.err = h->t2_err;
    const uint64_t grid = std::min<uint64_t>(a.ntiles, std::min<uint64_t>((uint64_t)h->sm_count, 256));
    const int slot = prof_begin(h);
    k_tile3<<<(unsigned)grid, kT3Threads, kSmemBytes, h->stream>>>(reinterpret_cast<float *>(h->amps), a);
    SV_CUDA(cudaGetLastError());
    note_launch();
    prof_end(h, slot, meta);
    h->stats.kernels++;
    h->stats.fused_blocks += p.nblocks;
    h->norm_pending = true;
    h->norm_idx = out_idx;
    h->norm_cnt = (int)grid;
    return SV_OK;
}

namespace {
__global__ void k_norm_scale(float4 *__restrict__ v, uint64_t nvec, const double *__restrict__ parts,
                             int nparts) {
    __shared__ float sh[2];
    if (threadIdx.x == 0) {
        double nn = 0.0;
        for (int i = 0; i < nparts; i++) nn += parts[i];
        const double s = nn > 0.0 ? 1.0 / sqrt(nn) : 1.0;
        sh[0] = (float)s;
        sh[1] = (float)(s - (double)(float)s);
    }
    __syncthreads();
    const float hi = sh[0], lo = sh[1];
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nvec; i += stride) {
        float4 x = v[i];
        x.x = fmaf(x.x, hi, x.x * lo);
        x.y = fmaf(x.y, hi, x.y * lo);
        x.z = fmaf(x.z, hi, x.z * lo);
        x.w = fmaf(x.w, hi, x.w * lo);
        v[i] = x;
    }
}
}  // namespace

// Apply a fused pass's pending norm correction to the whole state (complex64).
sv_status resolve_norm(sv_state *h) {
    if (!h->norm_pending) return SV_OK;
    h->norm_pending = false;
    if (h->dt != SV_C64) return SV_OK;
    const uint64_t nvec = ((uint64_t)1 << h->n) / 2;
    const uint64_t blocks = std::min<uint64_t>((nvec + 255) / 256, (uint64_t)h->sm_count * 16);
    k_norm_scale<<<(unsigned)std::max<uint64_t>(blocks, 1), 256, 0, h->stream>>>(
        reinterpret_cast<float4 *>(h->amps), nvec, h->norm_buf + 256 * h->norm_idx, h->norm_cnt);
    SV_CUDA(cudaGetLastError());
    note_launch();
    h->stats.kernels++;
    return SV_OK;
}

}  // namespace sv
