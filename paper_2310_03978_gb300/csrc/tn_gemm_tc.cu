// Complex GEMM on the 5th-generation tensor cores (tcgen05, sm_103a).
//
// C[m, n] = 2^(eA + eB) * sum_k A[m, k] * B[n, k] for one slice per grid row, where A and B are
// stored as planar numbers (a real plane and an imaginary plane: FP16 or BF16 with kind::f16, or
// FP32 rounded to TF32 with kind::tf32) scaled by per-slice powers of two (the dynamic scaling that
// Sec. 4.2 proposes, made exact by using powers of two), and the sum runs in FP32 in tensor memory.
// The complex product is formed from four real products (4M):
//     Cre = Are*Bre - Aim*Bim,   Cim = Are*Bim + Aim*Bre,
// with the minus sign taken by the instruction descriptor's negate-A bit, from three (3M,
// Gauss's product):
//     P1 = Are*Bre, P2 = Aim*Bim, P3 = (Are+Aim)*(Bre+Bim);  Cre = P1 - P2, Cim = P3 - P1 - P2,
// where the sum planes Are+Aim and Bre+Bim are rounded once from FP32 by the conversion kernel, or
// from compensated hi / lo planes (x = hi + lo, xy ~ hi hi + hi lo + lo hi, Sec. 4.2's 3xTF32
// scheme) with the accumulator promoted to an FP32 running sum every 512 of K.
//
// k_gemm_tc: one CTA per output tile (128 x 128 or 128 x 256): warp 0 lane 0 issues TMA loads
// into a shared-memory ring, warp 1 lane 0 issues tcgen05.mma into the TMEM accumulators, and the
// epilogue warps drain TMEM through tcgen05.ld, apply the exponent and scatter the result into the
// consumer's memory order (Sec. 4.1 index reordering, done at the producer's store).
// k_gemm_tc_pers: the persistent 4M kernel for short contractions (see its comment below).
// Every mbarrier wait gives up after a device-time limit, records a timeout in a status word and
// lets the CTA release its TMEM and exit.
#include <type_traits>
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <vector>

#include "tn_internal.h"
#include "tn_planar_out.cuh"
#include "tn_thin_stage.cuh"

namespace tn {

namespace {

constexpr int BM = 128;
constexpr int CW = 64;       // epilogue column chunk
constexpr int SLD = CW + 1;  // padded row stride of the epilogue staging tile (float2)

// NPL planes per operand (2: 4M; 3: 3M; 4: split 4M with hi and lo planes); shared-memory rows
// of 2 * BKT bytes (BKT = 64: 128-byte rows with the 128-byte swizzle, 32: 64-byte rows with the
// 64-byte swizzle), which hold KEL = 2 * BKT / ESZ elements of K (ESZ = 2: FP16 / BF16 with
// kind::f16, ESZ = 4: FP32 storage read as TF32 with kind::tf32); an N tile of BNT columns; STG
// pipeline stages; MINB CTAs per SM.  One MMA consumes 32 bytes of K per row in both kinds
// (16 16-bit or 8 TF32 elements), so the shared-memory geometry depends on BKT alone.
template <int NPL, int BKT, int BNT, int STG, int MINB, int ESZ>
struct Cfg {
    static constexpr int KEL = 2 * BKT / ESZ;
    static constexpr int TILE_A = BM * BKT * 2;
    static constexpr int TILE_B = BNT * BKT * 2;
    static constexpr int STAGE_BYTES = NPL * (TILE_A + TILE_B);
    static constexpr int RING = STG * STAGE_BYTES;
    static constexpr int STAGING = BM * SLD * 8 + 64 * 12;  // tile chunk + per-iteration tables
    static constexpr int BODY = RING > STAGING ? RING : STAGING;
    static constexpr int BODY_MIN = MINB == 2 ? 80 * 1024 : 0;  // at most 2 CTAs per SM
    static constexpr int SMEM_BYTES = (BODY > BODY_MIN ? BODY : BODY_MIN) + 1024 + 256;
    // accumulators: 4M 2 (re, im), 3M 3, split 4M 2 plus 2 running sums for the promotion
    static constexpr int ACC = NPL == 3 ? 3 * BNT : (NPL == 4 ? 4 * BNT : 2 * BNT);
    static constexpr int TMEM_COLS = ACC <= 256 ? 256 : 512;
    static constexpr int SBO = 8 * BKT * 2;                 // bytes between 8-row groups
    static constexpr uint64_t LAYOUT = BKT == 64 ? 2 : 4;   // 128-byte / 64-byte swizzle
    static_assert(ACC <= 512, "accumulators exceed tensor memory");
    static_assert(MINB * TMEM_COLS <= 512, "co-resident CTAs exceed tensor memory");
    static_assert(ESZ == 2 || ESZ == 4, "16-bit or TF32 operands");
};

constexpr unsigned long long kWaitLimitNs = 4000000000ull;  // default bound of every wait: 4 s

__device__ unsigned int g_tc_status;  // bit 0: an mbarrier wait timed out

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ unsigned long long globaltimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n"
        ".reg .pred p;\n"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        "selp.u32 %0, 1, 0, p;\n"
        "}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait: false (and the status word set) once the deadline has passed.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity,
                                          unsigned long long deadline) {
    while (!mbar_try_wait(bar, parity)) {
        if (globaltimer() > deadline) {
            atomicOr(&g_tc_status, 1u);
            return false;
        }
    }
    return true;
}

__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *map, uint64_t *bar,
                                            int c0, int c1, int c2) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(smem_u32(bar))
        : "memory");
}

// Shared-memory matrix descriptor of a K-major tile written by TMA with a 128- or 64-byte
// swizzle: rows of 128 (64) bytes, 8-row groups 1024 (512) bytes apart.
template <int SBO, uint64_t LAYOUT>
__device__ __forceinline__ uint64_t sdesc_sw(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);  // start address (16-byte units)
    d |= (uint64_t)1 << 16;                    // leading byte offset (unused for these layouts)
    d |= (uint64_t)(SBO >> 4) << 32;           // stride byte offset: next 8-row group
    d |= (uint64_t)1 << 46;                    // descriptor version of tcgen05
    d |= LAYOUT << 61;                         // swizzle mode
    return d;
}

// Instruction descriptor of kind::f16 (fmt 0 = F16, 1 = BF16) or kind::tf32 (fmt 2 = TF32)
// with FP32 accumulation, both operands K-major.
__host__ __device__ constexpr uint32_t idesc_mma(uint32_t fmt, int M, int N, bool neg_a) {
    return (1u << 4)                          // D format: F32
           | (fmt << 7)                       // A format
           | (fmt << 10)                      // B format
           | ((neg_a ? 1u : 0u) << 13)        // negate A
           | ((uint32_t)(N >> 3) << 17)       // N / 8
           | ((uint32_t)(M >> 4) << 24);      // M / 16
}

template <int ESZ>
__device__ __forceinline__ void umma(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                     uint32_t accumulate) {
    if constexpr (ESZ == 2) {
        asm volatile(
            "{\n"
            ".reg .pred p;\n"
            "setp.ne.b32 p, %4, 0;\n"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n"
            "}\n" ::"r"(d_tmem),
            "l"(a), "l"(b), "r"(idesc), "r"(accumulate));
    } else {
        asm volatile(
            "{\n"
            ".reg .pred p;\n"
            "setp.ne.b32 p, %4, 0;\n"
            "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n"
            "}\n" ::"r"(d_tmem),
            "l"(a), "l"(b), "r"(idesc), "r"(accumulate));
    }
}

__device__ __forceinline__ void umma_commit(uint64_t *bar) {
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
        "%11, %12, %13, %14, %15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
          "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
}


__device__ __forceinline__ void tmem_st16(uint32_t taddr, const uint32_t (&r)[16]) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
        "%11, %12, %13, %14, %15, %16};" ::"r"(taddr),
        "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]),
        "r"(r[8]), "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]),
        "r"(r[15]));
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ uint64_t deposit(uint64_t x, int n, const int8_t *pos) {
    uint64_t r = 0;
    for (int i = 0; i < n; ++i)
        if ((x >> i) & 1ull) r |= 1ull << pos[i];
    return r;
}

// Compensated (split) products restart their TMEM accumulator every kPromoteK elements of K and
// four warps fold each chunk into a running FP32 sum (round to nearest) kept in the other half
// of tensor memory: the tensor core's own accumulation over a long K loses low-order bits at
// every step, which shows as an error growing linearly with K and would swamp the ~2^-22
// accuracy of hi + lo operands.
constexpr int kPromoteK = 512;

template <int NPL, int BKT, int BNT, int STG, int MINB, int ESZ>
__global__ void __launch_bounds__(NPL == 4 ? 192 : 128, MINB)
    k_gemm_tc(const __grid_constant__ TcGemmDesc d, int64_t tiles_n) {
    using F = Cfg<NPL, BKT, BNT, STG, MINB, ESZ>;
    // split 4M: warps 2..5 fold chunk accumulators into the running sums and write the result
    constexpr bool PROMOTE = NPL == 4;
    constexpr int CHUNK_KB = kPromoteK / F::KEL;
    constexpr int STAGES = STG;
    constexpr int STAGE_BYTES = F::STAGE_BYTES;
    constexpr int TMEM_COLS = F::TMEM_COLS;
    constexpr int TILE_A = F::TILE_A, TILE_B = F::TILE_B;
    constexpr int BK = F::KEL, BN = BNT;  // K elements per stage, N tile
    // epilogue chunk: 64 columns (13 bits with the 7 row bits), or the whole 32-column tile
    constexpr int CWK = BN < CW ? BN : CW;
    constexpr int CHB = CWK == 64 ? 13 : 12;       // bits of a chunk
    constexpr int ITERS = (BM * CWK) / (8 * 128);  // 8-element stores per thread and chunk
    static_assert(CWK == 64 || CWK == 32, "epilogue chunk of 64 or 32 columns");
    auto sdesc = [](uint32_t a) { return sdesc_sw<F::SBO, F::LAYOUT>(a); };
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + F::BODY);
    uint64_t *empty = full + STAGES;
    uint64_t *done = empty + STAGES;
    uint64_t *chunk_full = done + 1;   // MMA -> fold warps: a chunk accumulator is complete
    uint64_t *chunk_free = done + 2;   // fold warps -> MMA: the chunk accumulator was folded
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(done + 3);
    int *aborted = reinterpret_cast<int *>(tmem_slot + 1);  // set when a wait gave up

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t s = blockIdx.y;
    // grouped raster: 16 m-tiles share a group so that concurrent CTAs reuse A and B in L2
    const int64_t tile = blockIdx.x;
    const int64_t tiles_m = (1ll << d.lm) / BM;
    const int64_t group = 16;
    const int64_t per_group = group * tiles_n;
    const int64_t g = tile / per_group;
    const int64_t first_m = g * group;
    const int64_t gsize = (tiles_m - first_m) < group ? (tiles_m - first_m) : group;
    const int64_t mt = first_m + (tile % per_group) % gsize;
    const int64_t nt = (tile % per_group) / gsize;
    const int m0 = (int)(mt * BM), n0 = (int)(nt * BN);
    // K below the K tile: one block, the tensor map zero-fills the columns past K
    const int num_kb = ((1 << d.lk) + BK - 1) / BK;
    const int sa = d.a_sliced ? (int)s : 0, sbi = d.b_sliced ? (int)s : 0;

    if (threadIdx.x == 0) {
        for (int i = 0; i < STAGES; ++i) {
            mbar_init(&full[i], 1);
            mbar_init(&empty[i], 1);
        }
        mbar_init(done, 1);
        mbar_init(chunk_full, 1);
        mbar_init(chunk_free, 4);
        *aborted = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&d.tmA))
                     : "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&d.tmB))
                     : "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(tmem_slot)),
                     "r"(TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;
    const unsigned long long limit = d.wait_limit_ns ? d.wait_limit_ns : kWaitLimitNs;
    const unsigned long long deadline = globaltimer() + limit;

    int issued = 0;  // k blocks whose loads the producer issued
    if (threadIdx.x == 0) {
        // TMA producer
        for (int kb = 0; kb < num_kb; ++kb) {
            const int st = kb % STAGES;
            const uint32_t ph = (uint32_t)(kb / STAGES) & 1u;
            if (kb >= STAGES && !mbar_wait(&empty[st], ph ^ 1u, deadline)) {
                *aborted = 1;
                break;
            }
            if (d.selftest_no_loads) break;  // nothing will arrive on full[]
            uint8_t *base = smem + st * STAGE_BYTES;
            mbar_expect_tx(&full[st], STAGE_BYTES);
            const int k0 = kb * BK;
#pragma unroll
            for (int pl = 0; pl < NPL; ++pl) {
                tma_load_3d(base + pl * TILE_A, &d.tmA, &full[st], k0, m0,
                            pl * (int)d.slices_a + sa);
                tma_load_3d(base + NPL * TILE_A + pl * TILE_B, &d.tmB, &full[st], k0, n0,
                            pl * (int)d.slices_b + sbi);
            }
            issued = kb + 1;
        }
    } else if (threadIdx.x == 32) {
        // MMA issuer: 4M = four real products into the re and im accumulators,
        // 3M = three products into three accumulators
        const uint32_t fmt = ESZ == 4 ? 2u : (d.dtype == 1 ? 1u : 0u);
        const uint32_t id_pos = idesc_mma(fmt, BM, BNT, false);
        const uint32_t id_neg = idesc_mma(fmt, BM, BNT, true);
        bool ok = true;
        for (int kb = 0; kb < num_kb && ok; ++kb) {
            const int st = kb % STAGES;
            const uint32_t ph = (uint32_t)(kb / STAGES) & 1u;
            const int chunk = kb / CHUNK_KB, kc = kb % CHUNK_KB;
            if (PROMOTE && kc == 0 && chunk > 0) {
                // the previous chunk must be folded before its accumulator is restarted
                if (!mbar_wait(chunk_free, (uint32_t)(chunk - 1) & 1u, deadline)) {
                    ok = false;
                    *aborted = 1;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            }
            if (!mbar_wait(&full[st], ph, deadline)) {
                ok = false;
                *aborted = 1;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t base = smem_u32(smem + st * STAGE_BYTES);
            const uint64_t a_re = sdesc(base), a_im = sdesc(base + TILE_A);
            const uint64_t b_re = sdesc(base + NPL * TILE_A);
            const uint64_t b_im = sdesc(base + NPL * TILE_A + TILE_B);
#pragma unroll
            for (int kk = 0; kk < BKT / 16; ++kk) {
                const uint64_t adv = (uint64_t)(kk * 32) >> 4;  // one MMA's 32 bytes of K,
                                                                 // inside one swizzled row
                const uint32_t first = ((PROMOTE ? kc : kb) > 0 || kk > 0) ? 1u : 0u;
                if constexpr (NPL == 2) {
                    umma<ESZ>(tmem, a_re + adv, b_re + adv, id_pos, first);
                    umma<ESZ>(tmem, a_im + adv, b_im + adv, id_neg, 1u);
                    umma<ESZ>(tmem + BN, a_re + adv, b_im + adv, id_pos, first);
                    umma<ESZ>(tmem + BN, a_im + adv, b_re + adv, id_pos, 1u);
                } else if constexpr (NPL == 4) {
                    // compensated products: x = x_hi + x_lo, xy ~ x_hi y_hi + x_hi y_lo + x_lo y_hi
                    const uint64_t a_rl = sdesc(base + 2 * TILE_A), a_il = sdesc(base + 3 * TILE_A);
                    const uint64_t b_rl = sdesc(base + NPL * TILE_A + 2 * TILE_B);
                    const uint64_t b_il = sdesc(base + NPL * TILE_A + 3 * TILE_B);
                    umma<ESZ>(tmem, a_re + adv, b_re + adv, id_pos, first);
                    umma<ESZ>(tmem, a_im + adv, b_im + adv, id_neg, 1u);
                    umma<ESZ>(tmem, a_re + adv, b_rl + adv, id_pos, 1u);
                    umma<ESZ>(tmem, a_im + adv, b_il + adv, id_neg, 1u);
                    umma<ESZ>(tmem, a_rl + adv, b_re + adv, id_pos, 1u);
                    umma<ESZ>(tmem, a_il + adv, b_im + adv, id_neg, 1u);
                    umma<ESZ>(tmem + BN, a_re + adv, b_im + adv, id_pos, first);
                    umma<ESZ>(tmem + BN, a_im + adv, b_re + adv, id_pos, 1u);
                    umma<ESZ>(tmem + BN, a_re + adv, b_il + adv, id_pos, 1u);
                    umma<ESZ>(tmem + BN, a_im + adv, b_rl + adv, id_pos, 1u);
                    umma<ESZ>(tmem + BN, a_rl + adv, b_im + adv, id_pos, 1u);
                    umma<ESZ>(tmem + BN, a_il + adv, b_re + adv, id_pos, 1u);
                } else {
                    const uint64_t a_sm = sdesc(base + 2 * TILE_A);
                    const uint64_t b_sm = sdesc(base + NPL * TILE_A + 2 * TILE_B);
                    umma<ESZ>(tmem, a_re + adv, b_re + adv, id_pos, first);
                    umma<ESZ>(tmem + BN, a_im + adv, b_im + adv, id_pos, first);
                    umma<ESZ>(tmem + 2 * BN, a_sm + adv, b_sm + adv, id_pos, first);
                }
            }
            umma_commit(&empty[st]);
            if (PROMOTE && (kc == CHUNK_KB - 1 || kb == num_kb - 1)) umma_commit(chunk_full);
        }
        umma_commit(done);
    } else if (PROMOTE && warp >= 2) {
        // fold warps: running sum (columns 2BN..4BN) += chunk accumulator (columns 0..2BN)
        const uint32_t lb = (uint32_t)((warp & 3) * 32) << 16;
        const int nchunks = (num_kb + CHUNK_KB - 1) / CHUNK_KB;
        for (int c = 0; c < nchunks; ++c) {
            bool ok = true;
            if (lane == 0) ok = mbar_wait(chunk_full, (uint32_t)c & 1u, deadline);
            ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
            if (!ok) {
                if (lane == 0) *aborted = 1;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll 1
            for (int col = 0; col < 2 * BN; col += 16) {
                uint32_t a[16], r[16];
                tmem_ld16(tmem + lb + (uint32_t)col, a);
                if (c > 0) {
                    tmem_ld16(tmem + lb + (uint32_t)(2 * BN + col), r);
                    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
                    for (int j = 0; j < 16; ++j)
                        r[j] = __float_as_uint(__uint_as_float(r[j]) + __uint_as_float(a[j]));
                } else {
                    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
                    for (int j = 0; j < 16; ++j) r[j] = a[j];
                }
                tmem_st16(tmem + lb + (uint32_t)(2 * BN + col), r);
            }
            asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncwarp();
            if (lane == 0) mbar_arrive(chunk_free);
        }
    }
    __syncwarp();

    // epilogue: every warp drains its 32 TMEM lanes (rows) into a shared-memory tile (the idle
    // pipeline buffers), which is then written out in the order of C's memory index: the 14 tile
    // bits are sorted by their position in C, so consecutive threads store consecutive addresses
    // whenever C's low bits fall inside the tile.  The wait result is made warp-uniform because
    // tcgen05.ld is a warp-collective instruction.
    bool have = false;
    if (lane == 0) have = mbar_wait(done, 0, deadline) && *(volatile int *)aborted == 0;
    have = __shfl_sync(0xffffffffu, have ? 1 : 0, 0) != 0;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (threadIdx.x == 0) {
        // every load this CTA issued must have landed before its shared memory is reused or
        // released; after a normal run the MMA warp consumed them all and these waits return
        const unsigned long long drain = globaltimer() + limit;
        for (int st = 0; st < STAGES && st < issued; ++st) {
            const int last = ((issued - 1 - st) / STAGES) * STAGES + st;
            mbar_wait(&full[st], (uint32_t)(last / STAGES) & 1u, drain);
        }
    }
    have = __syncthreads_and(have && *(volatile int *)aborted == 0 ? 1 : 0) != 0;
    if (have) {
        // The tile is written in chunks of CWK columns (64, or the whole tile when it is 32
        // wide): each chunk is staged in shared memory and written out in the order of C's
        // memory index.  A chunk has CHB bits (7 row bits and 6 or 5 column bits), sorted on the
        // host by their position in C; element t of the chunk in that order takes bits 0..2 from
        // the thread's own 8 elements, bits 3..9 from the thread index and the rest from the
        // iteration.
        float2 *stage = reinterpret_cast<float2 *>(smem);
        uint64_t *hi_off = reinterpret_cast<uint64_t *>(smem + BM * SLD * 8);
        int *hi_w = reinterpret_cast<int *>(hi_off + 64);
        const Pow2 pe = pow2_of(d.expA[sa] + d.expB[sbi]);
        // epilogue threads: all four warps, or the four fold warps (the running sums) when
        // promoting; et is the epilogue thread index 0..127
        const bool epi = !PROMOTE || warp >= 2;
        const int et = PROMOTE ? (int)threadIdx.x - 64 : (int)threadIdx.x;
        const int row = (warp & 3) * 32 + lane;
        const uint32_t lane_base = (uint32_t)((warp & 3) * 32) << 16;
        const uint32_t src = PROMOTE ? 2 * BN : 0;  // accumulator columns to read
        // sorted chunk bits 0..2 are C's positions 0..2 (the lowest three bits of C always lie
        // among the chunk's 7 row and 6 column bits), so each thread writes 8 consecutive
        // elements: bits 0..2 are its own, bits 3..9 come from the thread index and bits 10..12
        // from the iteration
        int w8[8];
        {
            int dq[3];
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                const int sq = d.tb_src[q];
                dq[q] = (sq & 128) ? (1 << (sq & 127)) * SLD : (1 << sq);
            }
#pragma unroll
            for (int j = 0; j < 8; ++j)
                w8[j] = ((j & 1) ? dq[0] : 0) + ((j & 2) ? dq[1] : 0) + ((j & 4) ? dq[2] : 0);
        }
        int mlo = 0, nlo = 0;
        uint64_t olo = 0;
#pragma unroll
        for (int q = 3; q < 10; ++q)
            if ((et >> (q - 3)) & 1) {
                const int sq = d.tb_src[q];
                if (sq & 128) mlo |= 1 << (sq & 127);
                else nlo |= 1 << sq;
                olo |= 1ull << d.tb_pos[q];
            }
        const int wlo = mlo * SLD + nlo;
        if (epi && et < ITERS) {
            int mi = 0, ni = 0;
            uint64_t off = 0;
#pragma unroll
            for (int q = 10; q < CHB; ++q)
                if ((et >> (q - 10)) & 1) {
                    const int sq = d.tb_src[q];
                    if (sq & 128) mi |= 1 << (sq & 127);
                    else ni |= 1 << sq;
                    off |= 1ull << d.tb_pos[q];
                }
            hi_off[et] = off;
            hi_w[et] = mi * SLD + ni;
        }
        const uint64_t mbase = deposit((uint64_t)m0, d.lm, d.posC_m);
        const int eo = d.planar_out ? planar_out_exponent(d.pout, s) : 0;
        if (d.planar_out && blockIdx.x == 0 && threadIdx.x == 0) d.pout.exps[s] = eo;
        float amx = 0.f;
#pragma unroll 1
        for (int cb = 0; cb < BN; cb += CWK) {
#pragma unroll 1
            for (int c0 = cb; c0 < cb + CWK && epi; c0 += 16) {
                uint32_t r0[16], r1[16];
                tmem_ld16(tmem + lane_base + src + (uint32_t)c0, r0);
                tmem_ld16(tmem + lane_base + src + (uint32_t)(BN + c0), r1);
                if constexpr (NPL != 3) {
                    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
                    for (int j = 0; j < 16; ++j)
                        stage[row * SLD + (c0 - cb) + j] =
                            make_float2(scale_pow2(__uint_as_float(r0[j]), pe),
                                        scale_pow2(__uint_as_float(r1[j]), pe));
                } else {
                    uint32_t r2[16];
                    tmem_ld16(tmem + lane_base + (uint32_t)(2 * BN + c0), r2);
                    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
                    for (int j = 0; j < 16; ++j) {
                        const float p1 = __uint_as_float(r0[j]), p2 = __uint_as_float(r1[j]);
                        const float p3 = __uint_as_float(r2[j]);
                        stage[row * SLD + (c0 - cb) + j] =
                            make_float2(scale_pow2(p1 - p2, pe), scale_pow2(p3 - p1 - p2, pe));
                    }
                }
            }
            __syncthreads();
            const uint64_t cbase = mbase | deposit((uint64_t)(n0 + cb), d.ln, d.posC_n);
            if (!epi) {
                // producer and MMA warps only join the barriers
            } else {
                float2 *C = d.C + s * d.sC + cbase;
#pragma unroll 2
                for (int it = 0; it < ITERS; ++it) {
                    const int w = wlo + hi_w[it];
                    float2 v[8];
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        v[j] = stage[w + w8[j]];
                        amx = fmaxf(amx, fmaxf(fabsf(v[j].x), fabsf(v[j].y)));
                    }
                    const uint64_t o = olo | hi_off[it];
                    if (d.planar_out) {
                        planar_out_store8(d.pout, s, cbase | o, v, eo);
                    } else {
                        float4 *c4 = reinterpret_cast<float4 *>(C + o);
#pragma unroll
                        for (int j = 0; j < 4; ++j)
                            c4[j] = make_float4(v[2 * j].x, v[2 * j].y, v[2 * j + 1].x,
                                                v[2 * j + 1].y);
                    }
                }
            }
            __syncthreads();
        }
        if (d.amax_out && epi) amax_publish(d.amax_out + s, amx);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(TMEM_COLS));
}

// Persistent 4M kernel for short contractions (K up to 512; with 64-byte rows also up to 4096,
// where the autotuner finds it faster than one tile per CTA): each CTA walks the tiles
// t = blockIdx.x, blockIdx.x + gridDim.x, ... (tiles of all slices, slice-major, grouped raster
// inside a slice).  Such steps write far more than they compute, so what matters is keeping the
// stores going: the MMA of the next tile fills the other half of a double-buffered TMEM
// accumulator (2 x (re, im) x 128 columns = 512) while eight epilogue warps drain the current
// one, and a CTA's setup (barriers, TMEM allocation) is paid once per SM instead of per tile.
// Warps 0-7 are the epilogue (warp w reads TMEM lanes 32 (w % 4).., columns 64 (w / 4).., and
// stages its half of the tile, 32 columns at a time, in its own shared-memory buffer), warp 8
// issues the TMA loads, warp 9 the MMAs.  Every wait is bounded; a wait that runs out sets the status word and
// the abort flag, and every role leaves its loop.
// 4 ring stages keep the TMA loads of the next tiles in flight; the epilogue stages 32 columns
// at a time (a 128 x 32 chunk: 7 row and 5 column bits)
constexpr int PERS_BN = 128, PERS_STG = 4, PERS_THREADS = 320, PCW = 32;

// Shared-memory rows of RB bytes: 64 (64-byte swizzle, K elements 32 / 16 per stage for 16-bit /
// TF32), 32 (32-byte swizzle) or 16 (no swizzle, 16-bit K = 8).  Each stage's TMA box is exactly
// K wide for the short contractions, so no zero fill is fetched; with 16-byte rows the MMA's
// second K half (elements 8..15) reads a zero page that sits one tile further (the descriptor's
// leading-dimension offset).
// BNP is the N tile (128, or 64 / 32 for results that narrow); B's planes then fill only the
// first BNP rows of their 128-row slots.  NPL planes per operand: 2 (re, im: 4M) or 4 (hi and lo
// planes of re and im: compensated products, K <= 512 needs no accumulator promotion); the
// compensated form with 128-byte rows keeps 2 ring stages to fit shared memory.
template <int ESZ, int RB, int BNP = PERS_BN, int NPL = 2>
struct PersCfg {
    static constexpr int KEL = RB / ESZ;                  // K elements per stage
    static constexpr int TILE = BM * RB;                  // one plane of A (128 rows)
    static constexpr int TILE_B = BNP * RB;               // one plane of B (BNP rows)
    static constexpr int TSTRIDE = RB == 16 ? 2 * TILE : TILE;  // tile + zero page
    static constexpr int STAGE_BYTES = 2 * NPL * TSTRIDE;  // A planes, then B planes
    static constexpr int TX_BYTES = NPL * (TILE + TILE_B);  // bytes the TMA writes per stage
    static constexpr int LBN = BNP == 128 ? 7 : (BNP == 64 ? 6 : 5);  // log2 of the N tile
    static constexpr int STG = NPL == 4 && RB == 64 ? 2 : PERS_STG;   // ring stages
    static constexpr int RING = STG * STAGE_BYTES;
    static constexpr int STAGE_HALF = BM * PCW * 8;       // staging of one 128 x 32 chunk
    static constexpr int DEP = 6 * 256 * 8;               // byte-wise deposit tables of m0, n0
    static constexpr int BODY = RING + 2 * STAGE_HALF;
    static constexpr int SMEM_BYTES = BODY + DEP + 1024 + 512;
    static constexpr int SBO = 8 * RB;                    // next 8-row group
    static constexpr int LBO = RB == 16 ? TILE : 16;      // next 16 bytes of K (no swizzle)
    static constexpr uint64_t LAYOUT = RB == 64 ? 4 : (RB == 32 ? 6 : 0);
    static constexpr int KSTEPS = RB == 16 ? 1 : RB / 32; // MMAs (32 bytes of K) per stage
    static_assert(RB == 16 ? ESZ == 2 : (RB == 32 || RB == 64), "row width");
    static_assert(BNP == 128 || BNP == 64 || BNP == 32, "N tile");
    static_assert(NPL == 2 || NPL == 4, "4M or compensated planes");
};

// Shared-memory matrix descriptor with an explicit leading-dimension offset (K-major tiles).
template <int SBO, int LBO, uint64_t LAYOUT>
__device__ __forceinline__ uint64_t sdesc_lbo(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)((LBO >> 4) & 0x3FFF) << 16;
    d |= (uint64_t)(SBO >> 4) << 32;
    d |= (uint64_t)1 << 46;
    d |= LAYOUT << 61;
    return d;
}

struct TileCoord {
    int s;
    uint32_t mt, nt;  // tile row and column
    int first;        // the slice's tile 0
};

// Tile t of the walk (all counts below 2^31, so 32-bit divisions suffice): slice-major, then
// groups of 16 m-tiles that sweep the n-tiles together (they share B in L2).
__device__ __forceinline__ TileCoord pers_tile(uint32_t t, uint32_t tiles_m, uint32_t tiles_n) {
    const uint32_t per_slice = tiles_m * tiles_n;
    TileCoord c;
    c.s = (int)(t / per_slice);
    const uint32_t tile = t - (uint32_t)c.s * per_slice;
    const uint32_t per_group = 16u * tiles_n;
    const uint32_t g = tile / per_group, r = tile - g * per_group;
    const uint32_t first_m = g * 16u;
    const uint32_t gsize = (tiles_m - first_m) < 16u ? (tiles_m - first_m) : 16u;
    const uint32_t q = r / gsize;
    c.mt = first_m + (r - q * gsize);
    c.nt = q;
    c.first = tile == 0;
    return c;
}

__device__ __forceinline__ void named_sync(int id, int threads) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(threads) : "memory");
}

__device__ __forceinline__ void named_arrive(int id, int threads) {
    asm volatile("bar.arrive %0, %1;" ::"r"(id), "r"(threads) : "memory");
}

// One 32-bit word holding re (low half) and im (high half) as FP16 (DT 0) or BF16 (DT 1).
template <int DT>
__device__ __forceinline__ uint32_t pack_re_im(float re, float im) {
    if constexpr (DT == 1) {
        const __nv_bfloat162 h = __floats2bfloat162_rn(re, im);
        return *reinterpret_cast<const uint32_t *>(&h);
    } else {
        const __half2 h = __floats2half2_rn(re, im);
        return *reinterpret_cast<const uint32_t *>(&h);
    }
}

// (a, b) times the power of two p.f1 * p.f2.  ONE (p.f2 == 1, the usual case: the exponents of a
// step's inputs and output differ by a few dozen) takes one paired FP32 multiply for both; each
// lane is rounded like a scalar multiply, so the result equals scale_pow2 of each.
template <bool ONE>
__device__ __forceinline__ void scale_pair(float a, float b, const Pow2 &p, float &x, float &y) {
    if constexpr (ONE) {
        asm("{\n\t.reg .b64 t, u;\n\tmov.b64 t, {%2, %3};\n\tmov.b64 u, {%4, %4};\n\t"
            "mul.rn.f32x2 t, t, u;\n\tmov.b64 {%0, %1}, t;\n\t}"
            : "=f"(x), "=f"(y)
            : "f"(a), "f"(b), "f"(p.f1));
    } else {
        x = scale_pow2(a, p);
        y = scale_pow2(b, p);
    }
}

// max(a, b, c) in one instruction (NaN operands are ignored, as by fmaxf)
__device__ __forceinline__ float max3f(float a, float b, float c) {
    float r;
    asm("max.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
}

template <bool V>
using BoolC = std::integral_constant<bool, V>;
template <int V>
using IntC = std::integral_constant<int, V>;

// Barrier over `threads` threads that also ANDs a predicate across them: every participant
// learns whether all of them had v set (so a group leaves a loop together).
__device__ __forceinline__ bool named_and(int id, int threads, bool v) {
    uint32_t r;
    asm volatile(
        "{\n"
        ".reg .pred p, q;\n"
        "setp.ne.u32 p, %1, 0;\n"
        "bar.red.and.pred q, %2, %3, p;\n"
        "selp.u32 %0, 1, 0, q;\n"
        "}\n"
        : "=r"(r)
        : "r"((uint32_t)(v ? 1 : 0)), "r"(id), "r"(threads)
        : "memory");
    return r != 0;
}

template <int ESZ, int RB, bool PACKED, int BNP, int NPL>
__global__ void __launch_bounds__(PERS_THREADS, 1)
    k_gemm_tc_pers(const __grid_constant__ TcGemmDesc d, int64_t tiles_n, int64_t slices) {
    using F = PersCfg<ESZ, RB, BNP, NPL>;
    constexpr int BK = F::KEL, BN = BNP, STG = F::STG;
    auto sdesc = [](uint32_t a) { return sdesc_lbo<F::SBO, F::LBO, F::LAYOUT>(a); };
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + F::BODY + F::DEP);
    uint64_t *empty = full + STG;
    uint64_t *tfull = empty + STG;        // MMA -> epilogue: accumulator buffer b is complete
    uint64_t *tempty = tfull + 2;         // epilogue -> MMA: buffer b was read (4 arrivals)
    uint64_t *mdone = tempty + 2;         // the MMA warp's last commit
    uint64_t *hi_off = mdone + 1;         // [8] epilogue table: C offsets of bits 10..12
    int *hi_w = reinterpret_cast<int *>(hi_off + 8);  // [8] their staging offsets
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(hi_w + 8);
    int *aborted = reinterpret_cast<int *>(tmem_slot + 1);
    int *drain_stop = aborted + 1;        // the drain warps ended the staging hand-off

    // deposit tables: dep[j][b] = C offset of byte b of the tile row index (j = 0..2) or of
    // the tile column index (j = 3..5), i.e. of m bits 7 + 8 j .. and n bits LBN + 8 (j - 3) ..
    // (LBN = log2 of the N tile)
    uint64_t (*dep)[256] = reinterpret_cast<uint64_t (*)[256]>(smem + F::BODY);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t tiles_m = (uint32_t)((1ll << d.lm) / BM);
    const uint32_t tn32 = (uint32_t)tiles_n;
    const uint32_t total = tiles_m * tn32 * (uint32_t)slices;
    const int num_kb = ((1 << d.lk) + BK - 1) / BK;
    const unsigned long long limit = d.wait_limit_ns ? d.wait_limit_ns : kWaitLimitNs;
    if (RB == 16) {
        // zero pages: the second 16 bytes of K of every tile of every stage (never loaded)
        for (int e = threadIdx.x; e < STG * 2 * NPL * (F::TILE / 16); e += PERS_THREADS) {
            const int tile = e / (F::TILE / 16), q = e % (F::TILE / 16);
            *reinterpret_cast<uint4 *>(smem + tile * F::TSTRIDE + F::TILE + q * 16) =
                make_uint4(0u, 0u, 0u, 0u);
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    for (int e = threadIdx.x; e < 6 * 256; e += PERS_THREADS) {
        const int j = e >> 8, b = e & 255;
        const bool nside = j >= 3;
        const int first = (nside ? F::LBN + 8 * (j - 3) : 7 + 8 * j), nb = nside ? d.ln : d.lm;
        const int8_t *pos = nside ? d.posC_n : d.posC_m;
        uint64_t v = 0;
        for (int i = 0; i < 8; ++i)
            if (((b >> i) & 1) && first + i < nb) v |= 1ull << pos[first + i];
        dep[j][b] = v;
    }

    if (threadIdx.x == 0) {
        for (int i = 0; i < STG; ++i) {
            mbar_init(&full[i], 1);
            mbar_init(&empty[i], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&tfull[b], 1);
            mbar_init(&tempty[b], 4);
        }
        mbar_init(mdone, 1);
        *aborted = 0;
        *drain_stop = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&d.tmA))
                     : "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&d.tmB))
                     : "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(tmem_slot)),
                     "r"(512));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    // epilogue tables of the 128 x 32 chunk (12 bits sorted by position in C; bits 0..2 are
    // C's positions 0..2): offsets of the high bits 10..11 (one entry per write iteration)
    if (threadIdx.x < 4) {
        int mi = 0, ni = 0;
        uint64_t off = 0;
        for (int q = 10; q < 12; ++q)
            if ((threadIdx.x >> (q - 10)) & 1) {
                const int sq = d.tb_src[q];
                if (sq & 128) mi |= 1 << (sq & 127);
                else ni |= 1 << sq;
                off |= 1ull << d.tb_pos[q];
            }
        hi_off[threadIdx.x] = off;
        hi_w[threadIdx.x] = (mi << 8) | ni;  // row and column parts of the chunk element
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;

    if (warp == 8) {
        // TMA producer: k blocks of all this CTA's tiles through the ring
        if (lane == 0) {
            int it = 0, issued = 0;
            for (uint32_t t = blockIdx.x; t < total && !*(volatile int *)aborted; t += gridDim.x) {
                const TileCoord c = pers_tile(t, tiles_m, tn32);
                const int sa = d.a_sliced ? c.s : 0, sbi = d.b_sliced ? c.s : 0;
                const int m0 = (int)(c.mt * BM), n0 = (int)(c.nt * BN);
                bool ok = true;
                for (int kb = 0; kb < num_kb; ++kb, ++it) {
                    const int st = it % STG;
                    const uint32_t ph = (uint32_t)(it / STG) & 1u;
                    if (it >= STG &&
                        !mbar_wait(&empty[st], ph ^ 1u, globaltimer() + limit)) {
                        *aborted = 1;
                        ok = false;
                        break;
                    }
                    uint8_t *base = smem + st * F::STAGE_BYTES;
                    mbar_expect_tx(&full[st], F::TX_BYTES);
                    const int k0 = kb * BK;
#pragma unroll
                    for (int pl = 0; pl < NPL; ++pl) {
                        tma_load_3d(base + pl * F::TSTRIDE, &d.tmA, &full[st], k0, m0,
                                    pl * (int)d.slices_a + sa);
                        tma_load_3d(base + (NPL + pl) * F::TSTRIDE, &d.tmB, &full[st], k0, n0,
                                    pl * (int)d.slices_b + sbi);
                    }
                    issued = it + 1;
                }
                if (!ok) break;
            }
            // loads still in flight must land before the CTA's shared memory is released: wait
            // for the last arrival of every stage that was used (after a normal run the MMA
            // warp has consumed them all and these waits return at once)
            const unsigned long long drain = globaltimer() + limit;
            for (int st = 0; st < STG && st < issued; ++st) {
                const int last = ((issued - 1 - st) / STG) * STG + st;
                mbar_wait(&full[st], (uint32_t)(last / STG) & 1u, drain);
            }
        }
    } else if (warp == 9) {
        // MMA issuer: tile i accumulates into TMEM buffer i & 1 (columns 256 (i & 1) ..)
        if (lane == 0) {
            const uint32_t fmt = ESZ == 4 ? 2u : (d.dtype == 1 ? 1u : 0u);
            const uint32_t id_pos = idesc_mma(fmt, BM, BN, false);
            const uint32_t id_neg = idesc_mma(fmt, BM, BN, true);
            int it = 0, i = 0;
            bool any = false;
            for (uint32_t t = blockIdx.x; t < total && !*(volatile int *)aborted;
                 t += gridDim.x, ++i) {
                const int buf = i & 1;
                if (i >= 2 && !mbar_wait(&tempty[buf], (uint32_t)((i >> 1) - 1) & 1u,
                                         globaltimer() + limit)) {
                    *aborted = 1;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t acc = tmem + (uint32_t)(buf * 2 * BN);
                bool ok = true;
                for (int kb = 0; kb < num_kb; ++kb, ++it) {
                    const int st = it % STG;
                    const uint32_t ph = (uint32_t)(it / STG) & 1u;
                    if (!mbar_wait(&full[st], ph, globaltimer() + limit)) {
                        *aborted = 1;
                        ok = false;
                        break;
                    }
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    const uint32_t base = smem_u32(smem + st * F::STAGE_BYTES);
                    const uint64_t a_re = sdesc(base), a_im = sdesc(base + F::TSTRIDE);
                    const uint64_t b_re = sdesc(base + NPL * F::TSTRIDE);
                    const uint64_t b_im = sdesc(base + (NPL + 1) * F::TSTRIDE);
#pragma unroll
                    for (int kk = 0; kk < F::KSTEPS; ++kk) {
                        const uint64_t adv = (uint64_t)(kk * 32) >> 4;
                        const uint32_t first = (kb > 0 || kk > 0) ? 1u : 0u;
                        umma<ESZ>(acc, a_re + adv, b_re + adv, id_pos, first);
                        umma<ESZ>(acc, a_im + adv, b_im + adv, id_neg, 1u);
                        umma<ESZ>(acc + BN, a_re + adv, b_im + adv, id_pos, first);
                        umma<ESZ>(acc + BN, a_im + adv, b_re + adv, id_pos, 1u);
                        if constexpr (NPL == 4) {
                            // compensated: x = hi + lo, xy ~ hi hi + hi lo + lo hi (Sec. 4.2)
                            const uint64_t a_rl = sdesc(base + 2 * F::TSTRIDE);
                            const uint64_t a_il = sdesc(base + 3 * F::TSTRIDE);
                            const uint64_t b_rl = sdesc(base + (NPL + 2) * F::TSTRIDE);
                            const uint64_t b_il = sdesc(base + (NPL + 3) * F::TSTRIDE);
                            umma<ESZ>(acc, a_re + adv, b_rl + adv, id_pos, 1u);
                            umma<ESZ>(acc, a_im + adv, b_il + adv, id_neg, 1u);
                            umma<ESZ>(acc, a_rl + adv, b_re + adv, id_pos, 1u);
                            umma<ESZ>(acc, a_il + adv, b_im + adv, id_neg, 1u);
                            umma<ESZ>(acc + BN, a_re + adv, b_il + adv, id_pos, 1u);
                            umma<ESZ>(acc + BN, a_im + adv, b_rl + adv, id_pos, 1u);
                            umma<ESZ>(acc + BN, a_rl + adv, b_im + adv, id_pos, 1u);
                            umma<ESZ>(acc + BN, a_il + adv, b_re + adv, id_pos, 1u);
                        }
                    }
                    umma_commit(&empty[st]);
                    any = true;
                }
                if (!ok) break;
                umma_commit(&tfull[buf]);
            }
            if (any) {
                // every MMA this warp issued has completed before the CTA tears down
                umma_commit(mdone);
                mbar_wait(mdone, 0, globaltimer() + limit);
            }
        }
    } else if (warp < 4) {
        // drain warps: warp w reads TMEM lanes 32 w.. (rows) of each tile, 32 columns at a time,
        // scales them and stages the 128 x 32 chunk in staging buffer n & 1 (n counts chunks)
        const int row = warp * 32 + lane;
        const uint32_t lane_base = (uint32_t)(warp * 32) << 16;
        // a planar two-plane result is staged as one 32-bit word per element (16-bit re | im),
        // which halves the shared-memory traffic; other results as complex64
        constexpr bool packed = PACKED;
        int phr = 0;  // column swizzle of this row (see tc_choose_swizzle)
#pragma unroll
        for (int b = 0; b < 7; ++b)
            if ((row >> b) & 1) phr ^= packed ? d.phi5[b] : d.phi[b];
        int cur_s = -1, eo = 0;
        Pow2 pe{1.f, 1.f};
        bool one = true;  // pe.f2 == 1: a single multiply scales a value
        int n = 0, i = 0;
        bool left = false;
        for (uint32_t t = blockIdx.x; t < total; t += gridDim.x, ++i) {
            const int buf = i & 1;
            bool ok = true;
            if (lane == 0)
                ok = mbar_wait(&tfull[buf], (uint32_t)(i >> 1) & 1u, globaltimer() + limit) &&
                     !*(volatile int *)aborted;
            ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
            ok = named_and(5, 128, ok);  // the four drain warps decide together
            if (!ok) {
                if (lane == 0) {
                    *aborted = 1;
                    *drain_stop = 1;
                }
                // wake the store warps (they see the stop flag and leave); buffer n & 1 is
                // theirs to wait on next
                if (n >= 2) named_sync(3 + (n & 1), 256);
                named_arrive(1 + (n & 1), 256);
                left = true;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const TileCoord c = pers_tile(t, tiles_m, tn32);
            if (c.s != cur_s) {
                // staged values are the result times 2^-eo when it is written as scaled planar
                // numbers (one power-of-two factor here, none in the store warps)
                cur_s = c.s;
                const int sa = d.a_sliced ? c.s : 0, sbi = d.b_sliced ? c.s : 0;
                eo = d.planar_out ? planar_out_exponent(d.pout, c.s) : 0;
                pe = pow2_of(d.expA[sa] + d.expB[sbi] - eo);
                one = pe.f2 == 1.f;
            }
            const uint32_t acc = tmem + lane_base + (uint32_t)(buf * 2 * BN);
            // the accumulator is read 16 columns (re, im) at a time, the next 16 being loaded
            // while the current ones are staged, so most of each TMEM round trip is hidden; a
            // 128 x 32 chunk is two such units
            uint32_t re0[16], im0[16], re1[16], im1[16];
            float amx = 0.f;  // packed mode: max-abs of the staged (scaled) values
            auto stage_unit = [&](const uint32_t (&re)[16], const uint32_t (&im)[16], int h) {
                float2 *stage = reinterpret_cast<float2 *>(smem + F::RING + (n & 1) * F::STAGE_HALF);
                if (h == 0 && n >= 2) named_sync(3 + (n & 1), 256);  // buffer freed
                // column c of this row sits at word row * PCW + (c ^ phr) = rowp ^ c (PCW = 32)
                const int rowp = row * PCW | phr;
                // the unrolled loops are specialised on the output type and on whether one
                // multiply scales a value (both uniform over the tile)
                if constexpr (packed) {
                    uint32_t *stage32 = reinterpret_cast<uint32_t *>(stage);
                    auto put = [&](auto dt, auto one_c) {
#pragma unroll
                        for (int j = 0; j < 16; ++j) {
                            float r, m;
                            scale_pair<decltype(one_c)::value>(__uint_as_float(re[j]),
                                                               __uint_as_float(im[j]), pe, r, m);
                            amx = max3f(amx, fabsf(r), fabsf(m));
                            stage32[rowp ^ (16 * h + j)] = pack_re_im<decltype(dt)::value>(r, m);
                        }
                    };
                    if (d.dtype == 1) {
                        if (one) put(IntC<1>{}, BoolC<true>{});
                        else put(IntC<1>{}, BoolC<false>{});
                    } else {
                        if (one) put(IntC<0>{}, BoolC<true>{});
                        else put(IntC<0>{}, BoolC<false>{});
                    }
                } else {
                    auto put = [&](auto one_c) {
#pragma unroll
                        for (int j = 0; j < 16; ++j) {
                            float r, m;
                            scale_pair<decltype(one_c)::value>(__uint_as_float(re[j]),
                                                               __uint_as_float(im[j]), pe, r, m);
                            stage[rowp ^ (16 * h + j)] = make_float2(r, m);
                        }
                    };
                    if (one) put(BoolC<true>{});
                    else put(BoolC<false>{});
                }
                if (h == 1) {
                    named_arrive(1 + (n & 1), 256);  // chunk n is staged
                    ++n;
                }
            };
            auto load_unit = [&](int u, uint32_t (&re)[16], uint32_t (&im)[16]) {
                tmem_ld16(acc + (uint32_t)(16 * u), re);
                tmem_ld16(acc + (uint32_t)(BN + 16 * u), im);
            };
            load_unit(0, re0, im0);
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
            for (int u = 0; u < BN / 16; u += 2) {
                load_unit(u + 1, re1, im1);
                stage_unit(re0, im0, 0);
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                if (u + 2 < BN / 16) {
                    load_unit(u + 2, re0, im0);
                    stage_unit(re1, im1, 1);
                    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                } else {
                    // every column of the accumulator buffer has been read: it may be refilled
                    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                    __syncwarp();
                    if (lane == 0) mbar_arrive(&tempty[buf]);
                    stage_unit(re1, im1, 1);
                }
            }
            // packed mode publishes the tile's max-abs here, at the true scale (2^eo times)
            if (packed && d.amax_out) amax_publish(d.amax_out + c.s, scale_pow2(amx, pow2_of(eo)));
        }
        // take the store warps' releases of the last two chunks, so every arrival is matched
        if (!left)
            for (int k = n - 2; k < n; ++k)
                if (k >= 0) named_sync(3 + (k & 1), 256);
    } else {
        // store warps: write staged chunk n of each tile in the order of C's memory index; a
        // chunk element is (row r, column c) = the OR of the row / column parts of its sorted bits
        // 0..2 (j), 3..9 (the thread) and 10..11 (the iteration), stored at r * 32 + (c ^ phi(r))
        const int et = threadIdx.x - 128;
        constexpr bool packed = PACKED;
        auto phi_of = [&](int r) {
            int p = 0;
#pragma unroll
            for (int b = 0; b < 7; ++b)
                if ((r >> b) & 1) p ^= packed ? d.phi5[b] : d.phi[b];
            return p;
        };
        // element j of an 8-run sits at row part rj, column part cj (disjoint from the other
        // parts), so its address is (rb + rj) * 32 + ((cb ^ phi(rb)) ^ (cj ^ phi(rj))):
        // rj32[j] = 32 rj and yj[j] = cj ^ phi(rj) are constants of the thread
        int rj32[8], yj[8];
        {
            int rq[3], cq[3];
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                const int sq = d.tb_src[q];
                rq[q] = (sq & 128) ? 1 << (sq & 127) : 0;
                cq[q] = (sq & 128) ? 0 : 1 << sq;
            }
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const int r = ((j & 1) ? rq[0] : 0) | ((j & 2) ? rq[1] : 0) | ((j & 4) ? rq[2] : 0);
                const int c = ((j & 1) ? cq[0] : 0) | ((j & 2) ? cq[1] : 0) | ((j & 4) ? cq[2] : 0);
                rj32[j] = r * PCW;
                yj[j] = c ^ phi_of(r);
            }
        }
        int mlo = 0, nlo = 0;
        uint64_t olo = 0;
#pragma unroll
        for (int q = 3; q < 10; ++q)
            if ((et >> (q - 3)) & 1) {
                const int sq = d.tb_src[q];
                if (sq & 128) mlo |= 1 << (sq & 127);
                else nlo |= 1 << sq;
                olo |= 1ull << d.tb_pos[q];
            }
        // row base (times 32) and swizzled column base of the thread's 8-run in iteration k
        int rbk32[4], xk[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int hk = hi_w[k];
            const int rb = mlo | (hk >> 8), cb = nlo | (hk & 255);
            rbk32[k] = rb * PCW;
            xk[k] = cb ^ phi_of(rb);
        }
        // C offsets of the column chunk inside the tile: n bits 5 and 6 (those the tile has)
        const uint64_t off5 = BN > 32 ? 1ull << d.posC_n[5] : 0ull;
        const uint64_t off6 = BN > 64 ? 1ull << d.posC_n[6] : 0ull;
        int cur_s = -1, eo = 0;
        int n = 0;
        bool stop = false;
        for (uint32_t t = blockIdx.x; t < total && !stop; t += gridDim.x) {
            const TileCoord c = pers_tile(t, tiles_m, tn32);
            if (c.s != cur_s) {
                cur_s = c.s;
                eo = d.planar_out ? planar_out_exponent(d.pout, c.s) : 0;
            }
            if (d.planar_out && c.first && et == 0) d.pout.exps[c.s] = eo;
            const uint64_t cbase0 = dep[0][c.mt & 255] | dep[1][(c.mt >> 8) & 255] |
                                    dep[2][(c.mt >> 16) & 255] | dep[3][c.nt & 255] |
                                    dep[4][(c.nt >> 8) & 255] | dep[5][(c.nt >> 16) & 255];
            float amj[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};  // independent chains
#pragma unroll 1
            for (int q = 0; q < BN / PCW; ++q, ++n) {
                named_sync(1 + (n & 1), 256);  // chunk n is staged
                // only the drain warps end the hand-off early (after a wait of theirs ran out),
                // so every barrier the other side waits on is still arrived at
                if (*(volatile int *)drain_stop) {
                    stop = true;
                    break;
                }
                const float2 *stage =
                    reinterpret_cast<const float2 *>(smem + F::RING + (n & 1) * F::STAGE_HALF);
                const uint64_t cbase = cbase0 | ((q & 1) ? off5 : 0ull) | ((q & 2) ? off6 : 0ull);
                float2 *C = d.C + (int64_t)c.s * d.sC + cbase;
#pragma unroll
                for (int k = 0; k < (BM * PCW) / (8 * 128); ++k) {
                    const int rb32 = rbk32[k], xb = xk[k];
                    if constexpr (packed) {
                        // 8 words (re | im) -> one 16-byte word of 8 16-bit numbers per plane
                        const uint32_t *stage32 = reinterpret_cast<const uint32_t *>(stage);
                        uint32_t w[8];
#pragma unroll
                        for (int j = 0; j < 8; ++j) w[j] = stage32[rb32 + rj32[j] + (xb ^ yj[j])];
                        const uint4 re = make_uint4(
                            __byte_perm(w[0], w[1], 0x5410), __byte_perm(w[2], w[3], 0x5410),
                            __byte_perm(w[4], w[5], 0x5410), __byte_perm(w[6], w[7], 0x5410));
                        const uint4 im = make_uint4(
                            __byte_perm(w[0], w[1], 0x7632), __byte_perm(w[2], w[3], 0x7632),
                            __byte_perm(w[4], w[5], 0x7632), __byte_perm(w[6], w[7], 0x7632));
                        uint16_t *pb = static_cast<uint16_t *>(d.pout.base) +
                                       (int64_t)c.s * d.pout.sstride +
                                       (int64_t)(cbase | olo | hi_off[k]);
                        *reinterpret_cast<uint4 *>(pb) = re;
                        *reinterpret_cast<uint4 *>(pb + d.pout.plane_stride) = im;
                    } else {
                        float2 v[8];
#pragma unroll
                        for (int j = 0; j < 8; ++j) {
                            v[j] = stage[rb32 + rj32[j] + (xb ^ yj[j])];
                            amj[j] = fmaxf(amj[j], fmaxf(fabsf(v[j].x), fabsf(v[j].y)));
                        }
                        const uint64_t o = olo | hi_off[k];
                        if (d.planar_out) {
                            planar_out_store8_prescaled(d.pout, c.s, cbase | o, v);
                        } else {
                            float4 *c4 = reinterpret_cast<float4 *>(C + o);
#pragma unroll
                            for (int j = 0; j < 4; ++j)
                                c4[j] = make_float4(v[2 * j].x, v[2 * j].y, v[2 * j + 1].x,
                                                    v[2 * j + 1].y);
                        }
                    }
                }
                named_arrive(3 + (n & 1), 256);  // buffer n & 1 is free again
            }
            if (!stop && d.amax_out && !packed) {
                float amx = amj[0];
#pragma unroll
                for (int j = 1; j < 8; ++j) amx = fmaxf(amx, amj[j]);
                // the true scale of planar values is 2^eo times the staged one
                amax_publish(d.amax_out + c.s, d.planar_out ? scale_pow2(amx, pow2_of(eo)) : amx);
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(512));
}

// Thin steps on the tensor cores (the low-intensity contractions of App. A.2):
// C[m, n] = sum_k A[m, k] B[n, k] for a complex64 A of 2^lm rows, NT = 2^ln in {4, 8, 16}
// columns and KC = 2^lk in {4, 8, 16} terms.  The complex product is one real product: A read
// as 2^lm x 2 KC real numbers (re, im interleaved along k) times the 2 KC x 2 NT real matrix B'
// with B'[2k, 2n] = B'[2k+1, 2n+1] = Re B[n, k], B'[2k+1, 2n] = -Im B[n, k] and
// B'[2k, 2n+1] = Im B[n, k] gives C as 2^lm x 2 NT real numbers (re, im interleaved along n).
// The products run in TF32 with compensated operands (x = hi + lo, hi = x rounded to TF32,
// A B' ~ Ahi B'lo + Alo B'hi + Ahi B'hi: Sec. 4.2's 3xTF32 scheme), which keeps the result at
// FP32-level accuracy while the tensor cores take the 4 NT KC multiply-adds per row that bound
// the CUDA-core form once NT and KC reach 8-16.
// A 128-row tile is loaded by TMA into a ring of raw stages (rows of 8 KC bytes with the
// matching swizzle; as many stages as shared memory holds, so enough reads stay in flight),
// split into hi / lo parts in one of two slots the MMAs read (which frees the raw stage at once),
// and accumulated in TMEM as a 128 x 32 block (B' has zero rows beyond 2 NT), four such buffers
// in turn.  Two drain groups of 4 warps take the tiles in turn (warp w reads TMEM lanes
// 32 (w % 4).., so thread t of a group holds row t of its tile) and write them in C's order
// through shared-memory stages, 8 consecutive elements of C per task as the CUDA-core thin
// kernel does; with two groups one tile's stores overlap the next tile's TMEM reads and
// staging.  Warps 8-11 split the tiles; warp 12 issues the TMA loads, warp 13 the MMAs; B'
// hi / lo is built by all threads before the roles start.
// Grid row y is slice y (about one CTA per SM in all); its CTAs walk the slice's tiles.  Every
// wait is bounded; a wait that runs out sets the status word and the abort flag, and every role
// leaves its loop.
template <int NT, int KC>
struct ThinTcCfg {
    static constexpr int RB = 8 * KC;             // bytes of one row of A (2 KC floats)
    static constexpr int NR = 2 * NT;             // real result columns
    static constexpr int NP = 32;                 // MMA N (the 32-column shape of the
                                                  // narrow tiles; B' rows past NR are zero)
    static constexpr int HALF = BM * RB;          // one 128-row tile of A
    static constexpr int CS = 2;                  // hi / lo slots the MMAs read
    static constexpr int SLOT = 2 * HALF;         // hi, then lo
    static constexpr int BPL = ((NP * RB + 1023) / 1024) * 1024;  // one plane of B'
    static constexpr int NB = 4;                  // TMEM accumulator buffers (2 per drain group)
    static constexpr int ESTAGE = 256 * NT * 8;   // two output stages of 128 rows (one group)
    static constexpr int FIXED = CS * SLOT + 2 * BPL + 2 * ESTAGE;
    // raw TMA stages: what is left of shared memory, at most 32 and 128 KB
    static constexpr int RS_FIT = (232448 - 2048 - FIXED) / HALF;
    static constexpr int RS_CAP = (131072 / HALF) < 32 ? (131072 / HALF) : 32;
    static constexpr int RS = RS_FIT < RS_CAP ? RS_FIT : RS_CAP;
    static constexpr int RAW = RS * HALF;
    static constexpr int BODY = RAW + FIXED;
    static constexpr int SMEM_BYTES = BODY + 1024 + 1024;
    static constexpr int SBO = 8 * RB;            // next 8-row group
    static constexpr uint64_t LAYOUT = RB == 128 ? 2 : (RB == 64 ? 4 : 6);
    static constexpr int KSTEPS = RB / 32;        // MMAs (8 TF32 of K) per tile
    static constexpr int TMEM_COLS = NB * NP;
    static constexpr int THREADS = 448;
    static_assert(NT == 4 || NT == 8 || NT == 16, "columns");
    static_assert(KC == 4 || KC == 8 || KC == 16, "terms");
    static_assert(RS >= 4, "raw stages");
    static_assert((2 * RS + 2 * CS + 2 * NB + 1) * 8 + 8 <= 1024, "barriers");
    static_assert(SMEM_BYTES <= 232448, "shared memory");
};

// Byte offset, inside a tile written with the TMA swizzle of rows of RB bytes (128: 16-byte
// chunk index XOR bits 7-9 of the offset; 64: XOR bits 7-8; 32: XOR bit 7), of the logical
// byte offset `o` = row * RB + byte; the tile starts on a 1024-byte boundary.
template <int RB>
__device__ __forceinline__ uint32_t swizzled(uint32_t o) {
    constexpr uint32_t mask = RB == 128 ? 7u : (RB == 64 ? 3u : 1u);
    return o ^ (((o >> 7) & mask) << 4);
}

// x rounded to the nearest TF32 number (the low 13 bits of the result are zero)
__device__ __forceinline__ float tf32_rna(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

template <int N>
__device__ __forceinline__ void tmem_ld_cols(uint32_t taddr, uint32_t (&r)[N]) {
    static_assert(N == 8 || N == 16 || N == 32, "columns per load");
    if constexpr (N == 8) {
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
            : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]),
              "=r"(r[6]), "=r"(r[7])
            : "r"(taddr));
    } else {
#pragma unroll
        for (int q = 0; q < N / 16; ++q) {
            uint32_t (&part)[16] = *reinterpret_cast<uint32_t (*)[16]>(&r[16 * q]);
            tmem_ld16(taddr + (uint32_t)(16 * q), part);
        }
    }
}

template <int NT, int KC>
__global__ void __launch_bounds__(448, 1)
    k_gemm_thin_tc(const __grid_constant__ ThinTcDesc d, int64_t slices) {
    using F = ThinTcCfg<NT, KC>;
    constexpr int RS = F::RS, CS = F::CS, NB = F::NB, ROWS = ThinStage<NT>::ROWS;
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    uint8_t *raw = smem;                   // RS raw stages (TMA)
    uint8_t *slots = smem + F::RAW;        // CS slots: hi, lo (MMA operands)
    uint8_t *bhi = slots + CS * F::SLOT, *blo = bhi + F::BPL;
    float2 *estage = reinterpret_cast<float2 *>(blo + F::BPL);  // [group][2][ROWS * NT]
    uint64_t *rfull = reinterpret_cast<uint64_t *>(smem + F::BODY);  // TMA -> split
    uint64_t *rempty = rfull + RS;  // split -> TMA: the raw stage was read (128 arrivals)
    uint64_t *cfull = rempty + RS;  // split -> MMA: hi / lo are in place (128 arrivals)
    uint64_t *cempty = cfull + CS;  // MMA -> split: the slot was consumed
    uint64_t *tfull = cempty + CS;  // MMA -> drain: accumulator buffer b is complete
    uint64_t *tempty = tfull + NB;  // drain -> MMA: buffer b was read (4 arrivals)
    uint64_t *mdone = tempty + NB;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(mdone + 1);
    int *aborted = reinterpret_cast<int *>(tmem_slot + 1);
    const GemmDesc &g = d.g;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // grid row y = slice s; the CTAs of a row walk the slice's 128-row tiles
    const uint32_t s = blockIdx.y;
    const uint32_t tps = (uint32_t)((1ll << g.lm) / ROWS);  // tiles per slice
    const unsigned long long limit = d.wait_limit_ns ? d.wait_limit_ns : kWaitLimitNs;

    if (threadIdx.x == 0) {
        for (int i = 0; i < RS; ++i) {
            mbar_init(&rfull[i], 1);
            mbar_init(&rempty[i], 128);
        }
        for (int i = 0; i < CS; ++i) {
            mbar_init(&cfull[i], 128);
            mbar_init(&cempty[i], 1);
        }
        for (int b = 0; b < NB; ++b) {
            mbar_init(&tfull[b], 1);
            mbar_init(&tempty[b], 4);
        }
        mbar_init(mdone, 1);
        *aborted = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&d.tmA))
                     : "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(tmem_slot)),
                     "r"(F::TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    // B' of the slice (hi / lo parts), written by every thread before the roles start
    {
        const float2 *Bs = g.B + (g.sB ? (int64_t)s : 0) * g.sB;
        for (int e = threadIdx.x; e < F::NP * 2 * KC; e += F::THREADS) {
            const int nr = e / (2 * KC), kf = e % (2 * KC);
            float v = 0.f;
            if (nr < F::NR) {
                const float2 b = Bs[(nr >> 1) * KC + (kf >> 1)];
                const int c = nr & 1, cp = kf & 1;
                v = c == cp ? b.x : (c == 0 ? -b.y : b.y);
            }
            const float hi = tf32_rna(v);
            const uint32_t o = swizzled<F::RB>((uint32_t)(nr * F::RB + kf * 4));
            *reinterpret_cast<float *>(bhi + o) = hi;
            *reinterpret_cast<float *>(blo + o) = v - hi;
        }
        // generic-proxy writes, read by the tensor cores (async proxy) after the barrier
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;

    if (warp == 12) {
        // TMA producer: every tile of this CTA through the raw ring
        if (lane == 0) {
            const int z = g.sA ? (int)s : 0;
            int it = 0, issued = 0;
            for (uint32_t tile = blockIdx.x; tile < tps && !*(volatile int *)aborted;
                 tile += gridDim.x, ++it) {
                const int rs = it % RS;
                if (it >= RS && !mbar_wait(&rempty[rs], ((uint32_t)(it / RS) & 1u) ^ 1u,
                                           globaltimer() + limit)) {
                    *aborted = 1;
                    break;
                }
                mbar_expect_tx(&rfull[rs], F::HALF);
                tma_load_3d(raw + rs * F::HALF, &d.tmA, &rfull[rs], 0, (int)(tile * ROWS), z);
                issued = it + 1;
            }
            // loads in flight land before the CTA's shared memory is released
            const unsigned long long drain = globaltimer() + limit;
            for (int rs = 0; rs < RS && rs < issued; ++rs) {
                const int last = ((issued - 1 - rs) / RS) * RS + rs;
                mbar_wait(&rfull[rs], (uint32_t)(last / RS) & 1u, drain);
            }
        }
    } else if (warp == 13) {
        // MMA issuer: tile i accumulates into TMEM buffer i % NB (32 columns each)
        if (lane == 0) {
            const uint32_t idesc = idesc_mma(2u, BM, F::NP, false);
            auto sd = [](uint32_t a) { return sdesc_lbo<F::SBO, 16, F::LAYOUT>(a); };
            const uint64_t bh = sd(smem_u32(bhi)), bl = sd(smem_u32(blo));
            int it = 0;
            bool any = false;
            for (uint32_t tile = blockIdx.x; tile < tps && !*(volatile int *)aborted;
                 tile += gridDim.x, ++it) {
                const int buf = it % NB, cs = it % CS;
                if (it >= NB && !mbar_wait(&tempty[buf], (uint32_t)((it / NB) - 1) & 1u,
                                           globaltimer() + limit)) {
                    *aborted = 1;
                    break;
                }
                if (!mbar_wait(&cfull[cs], (uint32_t)(it / CS) & 1u, globaltimer() + limit)) {
                    *aborted = 1;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t acc = tmem + (uint32_t)(buf * F::NP);
                const uint32_t base = smem_u32(slots + cs * F::SLOT);
                const uint64_t ah = sd(base), al = sd(base + F::HALF);
#pragma unroll
                for (int kk = 0; kk < F::KSTEPS; ++kk) {
                    const uint64_t adv = (uint64_t)(kk * 32) >> 4;
                    // the two correction products first, the main one last
                    umma<4>(acc, ah + adv, bl + adv, idesc, kk > 0 ? 1u : 0u);
                    umma<4>(acc, al + adv, bh + adv, idesc, 1u);
                    umma<4>(acc, ah + adv, bh + adv, idesc, 1u);
                }
                umma_commit(&cempty[cs]);
                umma_commit(&tfull[buf]);
                any = true;
            }
            if (any) {
                umma_commit(mdone);
                mbar_wait(mdone, 0, globaltimer() + limit);
            }
        }
    } else if (warp >= 8) {
        // split warps: every tile's hi / lo parts
        const int ts = threadIdx.x - 256;
        int it = 0;
        for (uint32_t tile = blockIdx.x; tile < tps; tile += gridDim.x, ++it) {
            const int rs = it % RS, cs = it % CS;
            // every thread waits itself: it reads what the TMA wrote, and rewrites a slot the
            // tensor cores read before
            bool ok = !*(volatile int *)aborted &&
                      mbar_wait(&rfull[rs], (uint32_t)(it / RS) & 1u, globaltimer() + limit);
            if (ok && it >= CS)
                ok = mbar_wait(&cempty[cs], ((uint32_t)(it / CS) & 1u) ^ 1u,
                               globaltimer() + limit);
            if (ok) {
                const float4 *r4 = reinterpret_cast<const float4 *>(raw + rs * F::HALF);
                float4 *hi4 = reinterpret_cast<float4 *>(slots + cs * F::SLOT);
                float4 *lo4 = reinterpret_cast<float4 *>(slots + cs * F::SLOT + F::HALF);
                constexpr int U = F::HALF / 16 / 128;  // 16-byte words per thread
#pragma unroll
                for (int q = 0; q < U; ++q) {
                    const float4 v = r4[ts + 128 * q];
                    const float4 hv = make_float4(tf32_rna(v.x), tf32_rna(v.y), tf32_rna(v.z),
                                                  tf32_rna(v.w));
                    hi4[ts + 128 * q] = hv;
                    lo4[ts + 128 * q] = make_float4(v.x - hv.x, v.y - hv.y, v.z - hv.z,
                                                    v.w - hv.w);
                }
                // the slot's generic-proxy writes, then the tensor cores (async proxy) read
                // them; the raw stage is released only now, after every value read from it has
                // been used: an arrive right after the loads let the next TMA write (fast when
                // the rows come from L2, as when all slices share the large operand) overtake
                // loads still queued, and a few rows of a tile came out wrong
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                mbar_arrive(&rempty[rs]);
                mbar_arrive(&cfull[cs]);
            }
            // the group leaves together once any of its waits ran out
            if (!named_and(5, 128, ok)) {
                if (ts == 0) *aborted = 1;
                break;
            }
        }
    } else {
        // two drain groups (warps 0-3 and 4-7) take the CTA's tiles in turn, each with its own
        // barriers and stages, so one group's stores overlap the other's TMEM reads; thread
        // gt of a group holds row gt of its tile (TMEM lane 32 (warp % 4) + lane)
        const int grp = warp >> 2, gt = threadIdx.x - ROWS * grp;
        const uint32_t lane_base = (uint32_t)((warp & 3) * 32) << 16;
        ThinStage<NT> stg;
        stg.init(g, gt);
        constexpr int TASKS = ThinStage<NT>::TASKS, SUBS = ThinStage<NT>::SUBS;
        constexpr int SPT = ThinStage<NT>::SPT, SPTP = ThinStage<NT>::SPTP;
        // C offset of tile t of a slice: deposit(t * ROWS); the warp's lanes take one bit each
        auto tile_base = [&](uint32_t t) {
            uint64_t r = 0;
            for (int b = ThinStage<NT>::LR + lane; b < g.lm; b += 32)
                if ((t >> (b - ThinStage<NT>::LR)) & 1u) r |= 1ull << g.posC_m[b];
            const uint32_t lo = __reduce_or_sync(0xffffffffu, (uint32_t)r);
            const uint32_t hi = __reduce_or_sync(0xffffffffu, (uint32_t)(r >> 32));
            return ((uint64_t)hi << 32) | lo;
        };
        float cr[NT], ci[NT];
        float amx = 0.f;
        const int eo = g.planar_out ? planar_out_exponent(g.pout, s) : 0;
        if (g.planar_out && blockIdx.x == 0 && threadIdx.x == 0) g.pout.exps[s] = eo;
        int j = 0;  // tiles this group has drained
        for (uint32_t tile = blockIdx.x + grp * gridDim.x; tile < tps;
             tile += 2 * gridDim.x, ++j) {
            const int it = 2 * j + grp, buf = it % NB;
            bool ok = true;
            if (lane == 0)
                ok = mbar_wait(&tfull[buf], (uint32_t)(it / NB) & 1u, globaltimer() + limit) &&
                     !*(volatile int *)aborted;
            ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
            if (!named_and(1 + grp, ROWS, ok)) {
                if (gt == 0) *aborted = 1;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            uint32_t v[F::NR < 16 ? 8 : F::NR];
            tmem_ld_cols(tmem + lane_base + (uint32_t)(buf * F::NP), v);
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncwarp();
            if (lane == 0) mbar_arrive(&tempty[buf]);
#pragma unroll
            for (int n = 0; n < NT; ++n) {
                cr[n] = __uint_as_float(v[2 * n]);
                ci[n] = __uint_as_float(v[2 * n + 1]);
            }
            // the group's stage j & 1 was last read two of its tiles ago, before every thread
            // of the group passed the barrier of its previous tile
            float2 *stage = estage + (size_t)(2 * grp + (j & 1)) * ROWS * NT;
            stg.put(stage, gt, cr, ci);
            named_sync(3 + grp, ROWS);
            const uint64_t cbase = tile_base(tile);
            if (g.planar_out) {
#pragma unroll
                for (int q = 0; q < SPTP; ++q) {
                    if (TASKS % ROWS != 0 && gt + ROWS * q >= TASKS) break;
                    float2 w[8];
#pragma unroll
                    for (int e = 0; e < 8; ++e) {
                        w[e] = stg.at(stage, q, e);
                        amx = fmaxf(amx, fmaxf(fabsf(w[e].x), fabsf(w[e].y)));
                    }
                    planar_out_store8(g.pout, s, cbase | stg.os[q], w, eo);
                }
            } else {
                float2 *C = g.C + (int64_t)s * g.sC + cbase;
#pragma unroll
                for (int q = 0; q < SPT; ++q) {
                    if (SUBS % ROWS != 0 && gt + ROWS * q >= SUBS) break;
#pragma unroll
                    for (int e = 0; e < 2; ++e) {
                        const float2 v0 = stg.at(stage, q, e ? 4 : 0);
                        const float2 v1 = stg.at(stage, q, e ? 5 : 1);
                        amx = fmaxf(amx, fmaxf(fmaxf(fabsf(v0.x), fabsf(v0.y)),
                                               fmaxf(fabsf(v1.x), fabsf(v1.y))));
                        *reinterpret_cast<float4 *>(C + (stg.os[q] + 4 * e)) =
                            make_float4(v0.x, v0.y, v1.x, v1.y);
                    }
                }
            }
        }
        if (g.amax_out) amax_publish(g.amax_out + s, amx);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(F::TMEM_COLS));
}

typedef CUresult (*PFN_encodeTiled)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                    const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                    const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                    CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

PFN_encodeTiled get_encode() {
    static PFN_encodeTiled fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000,
                                             cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_encodeTiled>(p);
    }
    return fn;
}

}  // namespace

bool tc_available() {
    int dev = 0, major = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return false;
    if (cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev) != cudaSuccess)
        return false;
    if (major != 10) return false;
    cudaFuncAttributes fa;
    if (cudaFuncGetAttributes(&fa, k_gemm_tc<2, 64, 128, 3, 1, 2>) != cudaSuccess) return false;
    return get_encode() != nullptr;
}

int encode_tmap_planar(void *tmap_host, const void *base, int64_t K, int64_t rows,
                       int64_t depth, int dtype, int bk, int box_rows) {
    PFN_encodeTiled enc = get_encode();
    if (!enc) return -1;
    const int esz = dtype == 2 ? 4 : 2;
    const int row_bytes = bk * esz;
    // K must fill whole 16-byte rows; a K below the tile is zero-filled by the tensor map
    if ((reinterpret_cast<uintptr_t>(base) & 15) != 0 ||
        (row_bytes != 16 && row_bytes != 32 && row_bytes != 64 && row_bytes != 128) ||
        (K * esz) % 16 != 0 || (K > bk && K % bk != 0) || dtype < 0 || dtype > 2)
        return -2;
    cuuint64_t dims[3] = {(cuuint64_t)K, (cuuint64_t)rows, (cuuint64_t)depth};
    cuuint64_t strides[2] = {(cuuint64_t)(K * esz), (cuuint64_t)(K * rows * esz)};
    if (box_rows != 32 && box_rows != 64 && box_rows != 128 && box_rows != 256) return -2;
    cuuint32_t box[3] = {(cuuint32_t)bk, (cuuint32_t)box_rows, 1};
    cuuint32_t estr[3] = {1, 1, 1};
    const CUtensorMapDataType ty = dtype == 2   ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                   : dtype == 1 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16
                                                : CU_TENSOR_MAP_DATA_TYPE_FLOAT16;
    CUresult r = enc(reinterpret_cast<CUtensorMap *>(tmap_host), ty, 3, const_cast<void *>(base),
                     dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                     row_bytes == 128  ? CU_TENSOR_MAP_SWIZZLE_128B
                     : row_bytes == 64 ? CU_TENSOR_MAP_SWIZZLE_64B
                     : row_bytes == 32 ? CU_TENSOR_MAP_SWIZZLE_32B
                                       : CU_TENSOR_MAP_SWIZZLE_NONE,
                     CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? 0 : -3;
}

namespace {

// The kernel variants, indexed by TcGemmDesc::variant: (id, planes, 16-bit elements per
// shared-memory row, N tile, stages, CTAs per SM, operand bytes).
#define TN_TC_VARIANTS(X)          \
    X(0, 2, 64, 128, 3, 1, 2)  /* 4M, long K (default)                  */ \
    X(1, 2, 32, 256, 4, 1, 2)  /* 4M, N tile 256                         */ \
    X(2, 2, 32, 128, 2, 2, 2)  /* 4M, short K: small ring, 2 CTAs per SM */ \
    X(3, 3, 32, 128, 4, 1, 2)  /* 3M                                     */ \
    X(4, 3, 64, 128, 2, 1, 2)  /* 3M, 128-byte swizzle                   */ \
    X(5, 2, 32, 128, 6, 1, 2)  /* 4M, 64-byte swizzle, 6 stages          */ \
    X(6, 4, 32, 128, 3, 1, 2)  /* split 4M (hi/lo planes), promoted      */ \
    X(7, 2, 32, 256, 4, 1, 4)  /* TF32 4M, N tile 256, K 16 per stage    */ \
    X(8, 2, 32, 128, 2, 2, 4)  /* TF32 4M, short K, 2 CTAs per SM        */ \
    X(9, 2, 64, 128, 3, 1, 4)  /* TF32 4M, 128-byte swizzle, K 32        */ \
    X(10, 3, 32, 128, 4, 1, 4) /* TF32 3M                                */ \
    X(11, 4, 32, 128, 3, 1, 4) /* split TF32 (3xTF32), promoted          */ \
    X(17, 2, 32, 64, 4, 2, 2)  /* 4M, N tile 64, 2 CTAs per SM           */ \
    X(18, 2, 32, 64, 4, 2, 4)  /* TF32 4M, N tile 64                     */ \
    X(19, 4, 32, 64, 2, 2, 2)  /* split 4M, N tile 64                    */ \
    X(20, 4, 32, 64, 2, 2, 4)  /* split TF32, N tile 64                  */ \
    X(21, 3, 32, 64, 2, 2, 2)  /* 3M, N tile 64                          */ \
    X(22, 3, 32, 64, 2, 2, 4)  /* TF32 3M, N tile 64                     */ \
    X(23, 2, 32, 32, 4, 2, 2)  /* 4M, N tile 32, 2 CTAs per SM           */ \
    X(24, 2, 32, 32, 4, 2, 4)  /* TF32 4M, N tile 32                     */ \
    X(25, 4, 32, 32, 2, 2, 2)  /* split 4M, N tile 32                    */ \
    X(26, 4, 32, 32, 2, 2, 4)  /* split TF32, N tile 32                  */ \
    X(27, 3, 32, 32, 2, 2, 2)  /* 3M, N tile 32                          */ \
    X(28, 3, 32, 32, 2, 2, 4)  /* TF32 3M, N tile 32                     */

template <int NPL, int BKT, int BNT, int STG, int MINB, int ESZ>
cudaError_t configure_variant() {
    return cudaFuncSetAttribute(k_gemm_tc<NPL, BKT, BNT, STG, MINB, ESZ>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize,
                                Cfg<NPL, BKT, BNT, STG, MINB, ESZ>::SMEM_BYTES);
}

template <int NPL, int BKT, int BNT, int STG, int MINB, int ESZ>
cudaError_t launch_variant(const TcGemmDesc &d, int64_t slices, cudaStream_t st) {
    constexpr int KEL = Cfg<NPL, BKT, BNT, STG, MINB, ESZ>::KEL;
    if (d.ln < (BNT == 256 ? 8 : (BNT == 64 ? 6 : (BNT == 32 ? 5 : 7))) || d.lk < 3 ||
        (KEL == 64 && d.lk < 6) ||
        (d.dtype == 2) != (ESZ == 4))
        return cudaErrorInvalidValue;
    const int64_t tiles_n = (1ll << d.ln) / BNT;
    const int64_t tiles = ((1ll << d.lm) / BM) * tiles_n;
    if (tiles > 0x7fffffffll) return cudaErrorInvalidConfiguration;
    k_gemm_tc<NPL, BKT, BNT, STG, MINB, ESZ>
        <<<dim3((unsigned)tiles, (unsigned)slices), NPL == 4 ? 192 : 128,
           Cfg<NPL, BKT, BNT, STG, MINB, ESZ>::SMEM_BYTES, st>>>(d, tiles_n);
    return cudaGetLastError();
}

}  // namespace

template <int ESZ, int RB, int BNP, int NPL>
cudaError_t configure_pers() {
    using F = PersCfg<ESZ, RB, BNP, NPL>;
    cudaError_t e = cudaFuncSetAttribute(k_gemm_tc_pers<ESZ, RB, false, BNP, NPL>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         F::SMEM_BYTES);
    if (e == cudaSuccess && ESZ == 2)
        e = cudaFuncSetAttribute(k_gemm_tc_pers<ESZ, RB, ESZ == 2, BNP, NPL>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, F::SMEM_BYTES);
    return e;
}

int sm_count() {
    static int n = 0;
    if (n == 0) {
        int dev = 0, v = 0;
        if (cudaGetDevice(&dev) == cudaSuccess &&
            cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess)
            n = v;
        if (n <= 0) n = 152;
    }
    return n;
}

template <int ESZ, int RB, int BNP, int NPL>
cudaError_t launch_pers(const TcGemmDesc &d, int64_t slices, cudaStream_t st) {
    using F = PersCfg<ESZ, RB, BNP, NPL>;
    // tile rows and columns index the deposit tables with 24 bits each; tiles count in 32 bits
    if (d.ln < F::LBN || d.lk < 3 || d.lk > (NPL == 4 ? 9 : 12) || d.lm > 31 || d.ln > 31 ||
        (d.dtype == 2) != (ESZ == 4))
        return cudaErrorInvalidValue;
    const int64_t tiles_n = (1ll << d.ln) / BNP;
    const int64_t total = ((1ll << d.lm) / BM) * tiles_n * slices;
    if (total > 0x7fffffffll) return cudaErrorInvalidConfiguration;
    int64_t grid = sm_count();
    if (grid > total) grid = total;
    // planar two-plane results (16-bit only) use the packed staging
    if (ESZ == 2 && d.planar_out && d.pout.planes == 2)
        k_gemm_tc_pers<ESZ, RB, ESZ == 2, BNP, NPL>
            <<<(unsigned)grid, PERS_THREADS, F::SMEM_BYTES, st>>>(d, tiles_n, slices);
    else
        k_gemm_tc_pers<ESZ, RB, false, BNP, NPL>
            <<<(unsigned)grid, PERS_THREADS, F::SMEM_BYTES, st>>>(d, tiles_n, slices);
    return cudaGetLastError();
}

template <int NT, int KC>
cudaError_t configure_thin_tc() {
    return cudaFuncSetAttribute(k_gemm_thin_tc<NT, KC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                ThinTcCfg<NT, KC>::SMEM_BYTES);
}

template <int NT, int KC>
cudaError_t launch_thin_tc_t(const ThinTcDesc &d, int64_t slices, cudaStream_t st) {
    using F = ThinTcCfg<NT, KC>;
    // one CTA per SM in all, spread over the slices (grid row y = slice), at most one per tile
    const int64_t tps = (1ll << d.g.lm) / 128;
    int64_t per_slice = sm_count() / slices;
    if (per_slice < 1) per_slice = 1;
    if (per_slice > tps) per_slice = tps;
    k_gemm_thin_tc<NT, KC><<<dim3((unsigned)per_slice, (unsigned)slices), F::THREADS,
                             F::SMEM_BYTES, st>>>(d, slices);
    return cudaGetLastError();
}

// Variants 12-16 are the persistent short-K kernel with 128-column tiles: 16-bit with rows of
// 64, 16 and 32 bytes (12, 14, 15), TF32 with rows of 64 and 32 bytes (13, 16); 29-33 the same
// five with 64-column tiles, 34-38 with 32-column tiles; 39-53 the compensated (hi / lo planes)
// counterparts of 12-16, 29-33 and 34-38 in that order.
constexpr int kPersFp16 = 12, kPersTf32 = 13, kPersFp16R16 = 14, kPersFp16R32 = 15,
              kPersTf32R32 = 16, kPers64 = 29, kPers32 = 34, kPersSplit = 39, kPersEnd = 54;

bool is_pers(int v) {
    return (v >= kPersFp16 && v <= kPersTf32R32) || (v >= kPers64 && v < kPersEnd);
}

bool pers_split(int v) { return v >= kPersSplit && v < kPersEnd; }

// the 4M 128-column variant (12-16) of the same row width and operand type, and the N tile
int pers_base(int v) { return v < kPers64 ? v : 12 + (v - kPers64) % 5; }
int pers_bn(int v) {
    if (v < kPers64) return PERS_BN;
    const int g = ((v - kPers64) / 5) % 3;  // 29-33 / 44-48: 64; 34-38 / 49-53: 32; 39-43: 128
    return g == 0 ? 64 : (g == 1 ? 32 : PERS_BN);
}

// the persistent variant for an N tile, compensated or not, on the row width of base (12-16)
int pers_variant(int base, int bn, bool split) {
    if (!split) return bn == 128 ? base : (bn == 64 ? kPers64 : kPers32) + base - 12;
    return kPersSplit + (bn == 128 ? 0 : (bn == 64 ? 5 : 10)) + base - 12;
}

int pers_kel(int v) {
    switch (pers_base(v)) {
        case kPersFp16: return PersCfg<2, 64>::KEL;
        case kPersTf32: return PersCfg<4, 64>::KEL;
        case kPersFp16R16: return PersCfg<2, 16>::KEL;
        case kPersFp16R32: return PersCfg<2, 32>::KEL;
        case kPersTf32R32: return PersCfg<4, 32>::KEL;
    }
    return 0;
}

template <int BNP, int NPL>
cudaError_t launch_pers_bn(int base, const TcGemmDesc &d, int64_t slices, cudaStream_t st) {
    switch (base) {
        case kPersFp16: return launch_pers<2, 64, BNP, NPL>(d, slices, st);
        case kPersTf32: return launch_pers<4, 64, BNP, NPL>(d, slices, st);
        case kPersFp16R16: return launch_pers<2, 16, BNP, NPL>(d, slices, st);
        case kPersFp16R32: return launch_pers<2, 32, BNP, NPL>(d, slices, st);
        case kPersTf32R32: return launch_pers<4, 32, BNP, NPL>(d, slices, st);
    }
    return cudaErrorInvalidValue;
}

template <int BNP, int NPL>
cudaError_t configure_pers_bn() {
    cudaError_t e = configure_pers<2, 64, BNP, NPL>();
    if (e == cudaSuccess) e = configure_pers<4, 64, BNP, NPL>();
    if (e == cudaSuccess) e = configure_pers<2, 16, BNP, NPL>();
    if (e == cudaSuccess) e = configure_pers<2, 32, BNP, NPL>();
    if (e == cudaSuccess) e = configure_pers<4, 32, BNP, NPL>();
    return e;
}

cudaError_t tc_prepare() {
    cudaError_t e = configure_pers_bn<128, 2>();
    if (e == cudaSuccess) e = configure_pers_bn<64, 2>();
    if (e == cudaSuccess) e = configure_pers_bn<32, 2>();
    if (e == cudaSuccess) e = configure_pers_bn<128, 4>();
    if (e == cudaSuccess) e = configure_pers_bn<64, 4>();
    if (e == cudaSuccess) e = configure_pers_bn<32, 4>();
    if (e == cudaSuccess) e = configure_thin_tc<4, 4>();
    if (e == cudaSuccess) e = configure_thin_tc<4, 8>();
    if (e == cudaSuccess) e = configure_thin_tc<4, 16>();
    if (e == cudaSuccess) e = configure_thin_tc<8, 4>();
    if (e == cudaSuccess) e = configure_thin_tc<8, 8>();
    if (e == cudaSuccess) e = configure_thin_tc<8, 16>();
    if (e == cudaSuccess) e = configure_thin_tc<16, 4>();
    if (e == cudaSuccess) e = configure_thin_tc<16, 8>();
    if (e == cudaSuccess) e = configure_thin_tc<16, 16>();
#define TN_TC_CONFIGURE(id, npl, bk, bn, stg, minb, esz) \
    if (e == cudaSuccess) e = configure_variant<npl, bk, bn, stg, minb, esz>();
    TN_TC_VARIANTS(TN_TC_CONFIGURE)
#undef TN_TC_CONFIGURE
    return e;
}

// K elements per pipeline stage of a variant (the tensor map's box width)
int tc_variant_bk(int variant) {
    if (is_pers(variant)) return pers_kel(variant);
    switch (variant) {
#define TN_TC_BK(id, npl, bk, bn, stg, minb, esz) \
    case id: return 2 * bk / esz;
        TN_TC_VARIANTS(TN_TC_BK)
#undef TN_TC_BK
    }
    return 0;
}

int tc_variant_bn(int variant) {
    if (is_pers(variant)) return pers_bn(variant);
    switch (variant) {
#define TN_TC_BN(id, npl, bk, bn, stg, minb, esz) \
    case id: return bn;
        TN_TC_VARIANTS(TN_TC_BN)
#undef TN_TC_BN
    }
    return 0;
}

bool tc_variant_is_pers(int variant) { return is_pers(variant); }

bool tc_variant_tf32(int variant) {
    if (is_pers(variant)) return pers_base(variant) == kPersTf32 || pers_base(variant) == kPersTf32R32;
    switch (variant) {
#define TN_TC_ESZ(id, npl, bk, bn, stg, minb, esz) \
    case id: return esz == 4;
        TN_TC_VARIANTS(TN_TC_ESZ)
#undef TN_TC_ESZ
    }
    return false;
}

// Variant choice (measured on GB300): short contractions (K <= 512) are epilogue-bound and run
// two CTAs per SM; long ones use the 128 x 256 tile (1.98 PFLOP/s on m=2^13, n=2^14, k=2^14
// against 1.79 for 128 x 128), or 128 x 128 when N < 256.
int tc_variant_form(int variant) {
    if (is_pers(variant)) return pers_split(variant) ? 3 : 1;
    switch (variant) {
#define TN_TC_FORM(id, npl, bk, bn, stg, minb, esz) \
    case id: return npl == 3 ? 2 : (npl == 4 ? 3 : 1);
        TN_TC_VARIANTS(TN_TC_FORM)
#undef TN_TC_FORM
    }
    return 0;
}

int tc_num_variants() { return kPersEnd; }

namespace {
int gf2_rank(std::vector<int> v) {
    int r = 0;
    for (int bit = 4; bit >= 0; --bit) {
        int piv = -1;
        for (size_t i = r; i < v.size(); ++i)
            if ((v[i] >> bit) & 1) {
                piv = (int)i;
                break;
            }
        if (piv < 0) continue;
        std::swap(v[r], v[piv]);
        for (size_t i = 0; i < v.size(); ++i)
            if ((int)i != r && ((v[i] >> bit) & 1)) v[i] ^= v[r];
        ++r;
    }
    return r;
}
}  // namespace

void tc_choose_swizzle(const int8_t *tb_src, int8_t *phi, int bits) {
    // bank index of a chunk element: its column's low `bits` bits XOR phi(row); a chunk bit
    // contributes its own bit when it is a column bit below `bits`, phi[i] for row bit i
    auto contrib = [&](int sq, const int *ph) {
        return (sq & 128) ? ph[sq & 127] : ((sq & 127) < bits ? 1 << (sq & 127) : 0);
    };
    // rows 0..4 (the lanes of a drain write) take a permutation of the unit masks (with 0 when
    // bits = 4), so a drain write spreads over all banks; rows 5, 6 take any unit mask or 0
    std::vector<int> units = {0};
    for (int b = 0; b < bits; ++b) units.push_back(1 << b);
    std::vector<int> perm = bits == 5 ? std::vector<int>{1, 2, 4, 8, 16}
                                      : std::vector<int>{0, 1, 2, 4, 8};
    std::sort(perm.begin(), perm.end());
    int best[7] = {perm[0], perm[1], perm[2], perm[3], perm[4], 0, 0};
    int best_rank = -1;
    do {
        int ph[7] = {perm[0], perm[1], perm[2], perm[3], perm[4], 0, 0};
        for (int f : units)
            for (int g : units) {
                ph[5] = f;
                ph[6] = g;
                std::vector<int> lanes;
                for (int q = 3; q < 8; ++q) lanes.push_back(contrib(tb_src[q], ph));
                const int r = gf2_rank(lanes);
                if (r > best_rank) {
                    best_rank = r;
                    for (int i = 0; i < 7; ++i) best[i] = ph[i];
                }
            }
    } while (best_rank < bits && std::next_permutation(perm.begin(), perm.end()));
    for (int i = 0; i < 7; ++i) phi[i] = (int8_t)best[i];
    phi[7] = 0;
}

bool tc_variant_fits(int variant, int lk, int ln) {
    if (is_pers(variant)) {
        // K up to 512 in every form; the 4M forms with 64-byte rows also take K up to 4096
        // (candidates of the autotuner: with K of 1024 the one-tile kernel's epilogue, not
        // overlapped with the next tile's products, costs ~20% of a 128 x 256 tile)
        const int bn = pers_bn(variant), base = pers_base(variant);
        const int kmax = (!pers_split(variant) && (base == kPersFp16 || base == kPersTf32)) ? 12 : 9;
        return lk >= 3 && lk <= kmax && (bn == 128 ? ln >= 7 : (bn == 64 ? ln == 6 : ln == 5));
    }
    const int bk = tc_variant_bk(variant), bn = tc_variant_bn(variant);
    if (bk == 0) return false;
    if (bk == 64 && lk < 6) return false;
    if (lk < 3) return false;
    // the 64-column tile is for narrow results (n = 64 .. 512); wider ones fill 128 or 256;
    // the 32-column tile for n = 32 only
    if (bn == 64) return ln >= 6 && ln <= 9;
    if (bn == 32) return ln == 5;
    return ln >= (bn == 256 ? 8 : 7);
}

// bk_pref / bn_pref: 0 or the K / N tile the caller asks for (K tile in 16-bit elements of a
// shared-memory row: 32 = 64-byte rows, 64 = 128-byte rows, for both operand types).
int tc_pick_variant(int form, int lk, int ln, int bk_pref, int bn_pref, bool tf32) {
    // short 4M or compensated contractions: the persistent kernel with a 128-, 64- or 32-column
    // tile, unless a tile shape was asked for
    if ((form == 1 || form == 3) && lk >= 3 && lk <= 9 && bk_pref == 0 && bn_pref == 0 &&
        ln >= 5) {
        const int base = tf32 ? (lk == 3 ? kPersTf32R32 : kPersTf32)
                              : (lk == 3 ? kPersFp16R16 : (lk == 4 ? kPersFp16R32 : kPersFp16));
        return pers_variant(base, ln >= 7 ? 128 : (ln == 6 ? 64 : 32), form == 3);
    }
    // n = 32 or 64: otherwise the 32- or 64-column one-tile kernel (2 CTAs per SM), every form
    if (ln == 5) {
        if (form == 3) return tf32 ? 26 : 25;
        if (form == 2) return tf32 ? 28 : 27;
        return tf32 ? 24 : 23;
    }
    if (ln < 7) {
        if (form == 3) return tf32 ? 20 : 19;
        if (form == 2) return tf32 ? 22 : 21;
        return tf32 ? 18 : 17;
    }
    if (tf32) {
        if (form == 3) return 11;
        if (form == 2) return 10;
        if (bn_pref == 256 && ln >= 8) return 7;
        if (bk_pref == 64) return 9;
        if (lk <= 9) return 8;
        return ln >= 8 && bn_pref != 128 ? 7 : 9;
    }
    if (form == 3) return 6;
    if (form == 2) return bk_pref == 64 ? 4 : 3;
    if (bn_pref == 256 && ln >= 8) return 1;
    if (bk_pref == 32) return lk <= 9 ? 2 : 5;
    if (bk_pref == 64 || bn_pref == 128) return lk <= 9 && bk_pref != 64 ? 2 : 0;
    if (lk <= 9) return 2;
    return ln >= 8 ? 1 : 0;
}

cudaError_t launch_gemm_tc(const TcGemmDesc &d, int64_t slices, cudaStream_t st) {
    if (d.lm < 7 || slices > 65535) return cudaErrorInvalidValue;
    if (is_pers(d.variant)) {
        const int bn = pers_bn(d.variant), base = pers_base(d.variant);
        if (pers_split(d.variant)) {
            if (bn == 64) return launch_pers_bn<64, 4>(base, d, slices, st);
            if (bn == 32) return launch_pers_bn<32, 4>(base, d, slices, st);
            return launch_pers_bn<128, 4>(base, d, slices, st);
        }
        if (bn == 64) return launch_pers_bn<64, 2>(base, d, slices, st);
        if (bn == 32) return launch_pers_bn<32, 2>(base, d, slices, st);
        return launch_pers_bn<128, 2>(base, d, slices, st);
    }
    switch (d.variant) {
#define TN_TC_LAUNCH(id, npl, bk, bn, stg, minb, esz) \
    case id: return launch_variant<npl, bk, bn, stg, minb, esz>(d, slices, st);
        TN_TC_VARIANTS(TN_TC_LAUNCH)
#undef TN_TC_LAUNCH
    }
    return cudaErrorInvalidValue;
}


bool thin_tc_fits(int lm, int ln, int lk) {
    return lm >= 8 && lm <= 30 && ln >= 2 && ln <= 4 && lk >= 2 && lk <= 4;
}

int encode_tmap_thin(void *tmap_host, const void *A, int lm, int lk, int64_t depth) {
    // A as [depth][2^lm rows][2 KC floats], one 128-row half per box
    return encode_tmap_planar(tmap_host, A, 2ll << lk, 1ll << lm, depth, 2, 2 << lk, 128);
}

cudaError_t launch_gemm_thin_tc(const ThinTcDesc &d, int64_t slices, cudaStream_t st) {
    const GemmDesc &g = d.g;
    if (!thin_tc_fits(g.lm, g.ln, g.lk) || g.tile_bits != 7 + g.ln || slices < 1)
        return cudaErrorInvalidValue;
    switch (g.ln * 8 + g.lk) {
        case 2 * 8 + 2: return launch_thin_tc_t<4, 4>(d, slices, st);
        case 2 * 8 + 3: return launch_thin_tc_t<4, 8>(d, slices, st);
        case 2 * 8 + 4: return launch_thin_tc_t<4, 16>(d, slices, st);
        case 3 * 8 + 2: return launch_thin_tc_t<8, 4>(d, slices, st);
        case 3 * 8 + 3: return launch_thin_tc_t<8, 8>(d, slices, st);
        case 3 * 8 + 4: return launch_thin_tc_t<8, 16>(d, slices, st);
        case 4 * 8 + 2: return launch_thin_tc_t<16, 4>(d, slices, st);
        case 4 * 8 + 3: return launch_thin_tc_t<16, 8>(d, slices, st);
        case 4 * 8 + 4: return launch_thin_tc_t<16, 16>(d, slices, st);
    }
    return cudaErrorInvalidValue;
}

// One CTA whose producer issues no loads: the MMA warp's wait on the first stage runs out after
// limit_ms, the CTA records the timeout in the status word, skips its epilogue, frees its tensor
// memory and exits.  Returns TN_ERR_TIMEOUT when that happened, TN_OK when the wait did not run out.
tn_status tc_selftest_wait_timeout(int32_t limit_ms, cudaStream_t st) {
    if (limit_ms < 1 || limit_ms > 10000) return report(TN_ERR_INVALID_ARG, "limit_ms out of range");
    if (!tc_available()) return report(TN_ERR_UNSUPPORTED, "no tcgen05 device");
    tc_status_read_and_clear();
    float2 *buf = nullptr;  // a valid tile-sized target; the self-test never writes it
    if (cudaMalloc(&buf, sizeof(float2) * 128 * 128 + 64) != cudaSuccess)
        return report(TN_ERR_OOM, "self-test buffer");
    TcGemmDesc d;
    memset(&d, 0, sizeof d);
    int32_t *exps = reinterpret_cast<int32_t *>(buf + 128 * 128);
    if (encode_tmap_planar(&d.tmA, buf, 64, 128, 2, 0, 64, 128) != 0 ||
        encode_tmap_planar(&d.tmB, buf, 64, 128, 2, 0, 64, 128) != 0) {
        cudaFree(buf);
        return report(TN_ERR_CUDA, "self-test tensor maps");
    }
    d.C = buf;
    d.lm = 7;
    d.ln = 7;
    d.lk = 6;
    d.slices_a = d.slices_b = 1;
    d.expA = d.expB = exps;
    d.form = 1;
    d.bk = 64;
    d.variant = 0;
    d.wait_limit_ns = (uint64_t)limit_ms * 1000000ull;
    d.selftest_no_loads = 1;
    cudaError_t e = launch_gemm_tc(d, 1, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFree(buf);
    if (e != cudaSuccess) return report(TN_ERR_CUDA, "self-test launch failed");
    return tc_status_read_and_clear() & 1u ? report(TN_ERR_TIMEOUT, "bounded wait ran out")
                                           : TN_OK;
}

unsigned int tc_status_read_and_clear() {
    unsigned int v = 0, z = 0;
    if (cudaMemcpyFromSymbol(&v, g_tc_status, sizeof v) != cudaSuccess) return 0xffffffffu;
    if (v) cudaMemcpyToSymbol(g_tc_status, &z, sizeof z);
    return v;
}

}  // namespace tn
