// Complex64 GEMM on the CUDA cores (FP32 FMA, 4 real products per complex multiply-add):
// C[m, n] = sum_k A[m, k] * B[n, k] per slice, A = [M][K] and B = [N][K] row-major, the result
// scattered into the consumer's memory order (the index reordering of Sec. 4.1 applied at the
// producer's store, so no separate transpose pass is needed).
//
// Accumulation is blocked: each 16-wide K tile is summed in fresh registers and then added to the
// running sum, which keeps the FP32 rounding error of a length-K sum near sqrt(K/16 + 16) units
// instead of sqrt(K).  The finished 64 x 64 tile is staged in shared memory and written out in
// the order of the consumer's memory index (tile bits sorted by their position in C), so the
// stores are contiguous whenever C's low bits fall inside the tile.
//
// Steps with few outputs and a long contraction (e.g. the last step of a circuit, which sums two
// large halves into the amplitudes) are split along K: CTA z sums its K range into a partial
// tile, and a second kernel adds the partials in increasing z (a fixed order, so results do not
// depend on scheduling) and scatters the sums.
#include "tn_internal.h"
#include "tn_planar_out.cuh"

namespace tn {

namespace {

constexpr int BM = 64, BN = 64, TM = 4, TN = 4;

__device__ __forceinline__ uint64_t deposit(uint64_t x, int n, const int8_t *pos) {
    uint64_t r = 0;
    for (int i = 0; i < n; ++i)
        if ((x >> i) & 1ull) r |= 1ull << pos[i];
    return r;
}

// 256 threads as 16 x 16; each thread owns rows ty + 16*i and columns tx + 16*j (i, j < 4).
// BK is the K tile (16, or 8 for contractions of at most 8 elements, which would otherwise
// multiply half a tile of zero padding).
template <int BK>
__global__ void __launch_bounds__(256) k_gemm_simt(GemmDesc d, int64_t tiles_n) {
    constexpr int AS = 2 * 16 * (BM + 1), BS = 2 * 16 * (BN + 1);
    static_assert(AS + BS >= BM * BN, "staging tile must fit in the operand buffers");
    __shared__ __align__(16) float2 sbuf[AS + BS];
    auto As = reinterpret_cast<float2(*)[BK][BM + 1]>(sbuf);
    auto Bs = reinterpret_cast<float2(*)[BK][BN + 1]>(sbuf + AS);
    const int64_t s = blockIdx.y;
    const int64_t tile = blockIdx.x;
    const int64_t m0 = (tile / tiles_n) * BM, n0 = (tile % tiles_n) * BN;
    const int64_t M = 1ll << d.lm, N = 1ll << d.ln;
    const int64_t Kfull = 1ll << d.lk;
    const int64_t K = Kfull / d.splits;  // this CTA's K range: [z * K, (z + 1) * K)
    const int64_t kz = (int64_t)blockIdx.z * K;
    const float2 *A = d.A + s * d.sA + kz;
    const float2 *B = d.B + s * d.sB + kz;
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;

    // global -> shared mapping: 64 rows x BK k; thread loads row (tid >> 2), k lk..lk+BK/4-1
    constexpr int KQ = BK / 4;
    const int lr = tid >> 2, lk = (tid & 3) * KQ;
    float2 ra[KQ], rb[KQ];
    auto load = [&](int64_t k0) {
        const int64_t gm = m0 + lr, gn = n0 + lr;
#pragma unroll
        for (int q = 0; q < KQ; ++q) {
            const int64_t gk = k0 + lk + q;
            ra[q] = (gm < M && gk < K) ? A[gm * Kfull + gk] : make_float2(0.f, 0.f);
            rb[q] = (gn < N && gk < K) ? B[gn * Kfull + gk] : make_float2(0.f, 0.f);
        }
    };
    auto store = [&](int buf) {
#pragma unroll
        for (int q = 0; q < KQ; ++q) {
            As[buf][lk + q][lr] = ra[q];
            Bs[buf][lk + q][lr] = rb[q];
        }
    };

    float cr[TM][TN], ci[TM][TN];
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) cr[i][j] = ci[i][j] = 0.f;

    load(0);
    store(0);
    __syncthreads();
    const int64_t ktiles = (K + BK - 1) / BK;
    for (int64_t kt = 0; kt < ktiles; ++kt) {
        const int buf = kt & 1;
        if (kt + 1 < ktiles) load((kt + 1) * BK);
        float tr[TM][TN], ti[TM][TN];
#pragma unroll
        for (int i = 0; i < TM; ++i)
#pragma unroll
            for (int j = 0; j < TN; ++j) tr[i][j] = ti[i][j] = 0.f;
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
            float2 a[TM], b[TN];
#pragma unroll
            for (int i = 0; i < TM; ++i) a[i] = As[buf][kk][ty + 16 * i];
#pragma unroll
            for (int j = 0; j < TN; ++j) b[j] = Bs[buf][kk][tx + 16 * j];
#pragma unroll
            for (int i = 0; i < TM; ++i)
#pragma unroll
                for (int j = 0; j < TN; ++j) {
                    tr[i][j] = fmaf(a[i].x, b[j].x, tr[i][j]);
                    tr[i][j] = fmaf(-a[i].y, b[j].y, tr[i][j]);
                    ti[i][j] = fmaf(a[i].x, b[j].y, ti[i][j]);
                    ti[i][j] = fmaf(a[i].y, b[j].x, ti[i][j]);
                }
        }
#pragma unroll
        for (int i = 0; i < TM; ++i)
#pragma unroll
            for (int j = 0; j < TN; ++j) {
                cr[i][j] += tr[i][j];
                ci[i][j] += ti[i][j];
            }
        if (kt + 1 < ktiles) store(buf ^ 1);
        __syncthreads();
    }

    if (d.splits > 1) {
        float2 *P = d.partial + ((int64_t)blockIdx.z * gridDim.y + s) * M * N;
#pragma unroll
        for (int i = 0; i < TM; ++i) {
            const int64_t gm = m0 + ty + 16 * i;
            if (gm >= M) continue;
#pragma unroll
            for (int j = 0; j < TN; ++j) {
                const int64_t gn = n0 + tx + 16 * j;
                if (gn < N) P[gm * N + gn] = make_float2(cr[i][j], ci[i][j]);
            }
        }
        return;
    }
    // stage the tile (row-major 64 x 64) and write it out in C's memory order
    float2 *stage = sbuf;
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j)
            stage[(ty + 16 * i) * BN + tx + 16 * j] = make_float2(cr[i][j], ci[i][j]);
    // element pairs of the tile in C order: sorted tile bit 0 is C's position 0 (the pair),
    // bits 1..8 come from the thread index and the rest from the iteration; the sorted tile bits
    // were computed on the host
    const int nb = d.tile_bits;
    __syncthreads();
    const int dpair = 1 << d.tb_src[0];
    int wlo = 0;
    uint64_t olo = 0;
    for (int q = 1; q < 9 && q < nb; ++q)
        if ((threadIdx.x >> (q - 1)) & 1) {
            wlo |= 1 << d.tb_src[q];
            olo |= 1ull << d.tb_pos[q];
        }
    const uint64_t cbase =
        deposit((uint64_t)m0, d.lm, d.posC_m) | deposit((uint64_t)n0, d.ln, d.posC_n);
    float2 *C = d.C + s * d.sC + cbase;
    const int eo = d.planar_out ? planar_out_exponent(d.pout, s) : 0;
    if (d.planar_out && blockIdx.x == 0 && blockIdx.z == 0 && threadIdx.x == 0)
        d.pout.exps[s] = eo;
    float amx = 0.f;
    auto put = [&](uint64_t off, int w) {
        const float2 v0 = stage[w], v1 = stage[w + dpair];
        if (d.planar_out) {
            planar_out_store2(d.pout, s, cbase | off, v0, v1, eo);
        } else {
            *reinterpret_cast<float4 *>(C + off) = make_float4(v0.x, v0.y, v1.x, v1.y);
        }
        amx = fmaxf(amx, fmaxf(fmaxf(fabsf(v0.x), fabsf(v0.y)), fmaxf(fabsf(v1.x), fabsf(v1.y))));
    };
    if (nb - 1 <= 8) {
        if ((int)threadIdx.x < (1 << (nb - 1))) put(olo, wlo);
    } else {
        for (int it = 0; it < (1 << (nb - 9)); ++it) {
            int w = wlo;
            uint64_t off = olo;
            for (int q = 9; q < nb; ++q)
                if ((it >> (q - 9)) & 1) {
                    w |= 1 << d.tb_src[q];
                    off |= 1ull << d.tb_pos[q];
                }
            put(off, w);
        }
    }
    if (d.amax_out) amax_publish(d.amax_out + s, amx);
}

// Split-K partial of a skinny step (the whole output fits one SW x LW tile of 1024 elements,
// 16 x 64 or 32 x 32: the side with at most SW free elements is "S", the other, at most LW, is
// "L"; K is long, e.g. the last step of a circuit).  Four groups of 64 threads each own a quarter
// of every 64-wide K tile; a thread accumulates a 4 x 4 block of outputs (S rows sg, sg + SW/4,
// .., L columns lg, lg + LW/4, ..), so every pair of shared-memory loads feeds 4 complex
// products.  The groups' sums are added in group order and CTA z writes partial[z][s] (row-major
// M x N) for k_splitk_reduce.
constexpr int kSkBK = 64;
// one buffer: S [k][SW + 1], L [k][LW + 1]; double-buffered (the 16 x 64 form is the larger)
constexpr int sk_buf(int sw) { return kSkBK * (sw + 1) + kSkBK * (1024 / sw + 1); }
constexpr int kSkSmem = 2 * sk_buf(16) * 8;            // bytes
static_assert(sk_buf(32) <= sk_buf(16), "shared-memory size of the skinny forms");

__device__ __forceinline__ void cp_async8(float2 *dst, const float2 *src, bool valid) {
    const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(d), "l"(src),
                 "r"(valid ? 8 : 0)
                 : "memory");
}

template <int SW>
__global__ void __launch_bounds__(256) k_gemm_skinny(GemmDesc d) {
    constexpr int LW = 1024 / SW, CS = LW / 4, RS = SW / 4;
    constexpr int kSkS = kSkBK * (SW + 1), kSkL = kSkBK * (LW + 1);
    extern __shared__ __align__(16) float2 skmem[];
    const int64_t s = blockIdx.y;
    const bool swap = d.lm > d.ln;               // S is B when M > N
    const int ls = swap ? d.ln : d.lm, ll = swap ? d.lm : d.ln;
    const int S = 1 << ls, L = 1 << ll;
    const int64_t Kfull = 1ll << d.lk;
    const int64_t K = Kfull / d.splits;
    const int64_t kz = (int64_t)blockIdx.z * K;
    const float2 *PS = (swap ? d.B + s * d.sB : d.A + s * d.sA) + kz;
    const float2 *PL = (swap ? d.A + s * d.sA : d.B + s * d.sB) + kz;
    const int tid = threadIdx.x, g = tid >> 6, t64 = tid & 63;
    const int sg = t64 / CS, lg = t64 % CS;
    auto bufS = [&](int b) {
        return reinterpret_cast<float2(*)[SW + 1]>(skmem + b * (kSkS + kSkL));
    };
    auto bufL = [&](int b) {
        return reinterpret_cast<float2(*)[LW + 1]>(skmem + b * (kSkS + kSkL) + kSkS);
    };
    // asynchronous copy of the K tile starting at k0 into buffer b (zero past this CTA's range)
    auto prefetch = [&](int b, int64_t k0) {
        float2(*sS)[SW + 1] = bufS(b);
        float2(*sL)[LW + 1] = bufL(b);
        for (int e = tid; e < S * kSkBK; e += 256) {
            const int r = e / kSkBK, k = e % kSkBK;
            const bool ok = k0 + k < K;
            cp_async8(&sS[k][r], PS + (ok ? (int64_t)r * Kfull + k0 + k : 0), ok);
        }
        for (int e = tid; e < L * kSkBK; e += 256) {
            const int r = e / kSkBK, k = e % kSkBK;
            const bool ok = k0 + k < K;
            cp_async8(&sL[k][r], PL + (ok ? (int64_t)r * Kfull + k0 + k : 0), ok);
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
    };
    float cr[4][4], ci[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) cr[i][j] = ci[i][j] = 0.f;
    const int64_t ntiles = (K + kSkBK - 1) / kSkBK;
    prefetch(0, 0);
    for (int64_t t = 0; t < ntiles; ++t) {
        const int b = (int)(t & 1);
        if (t + 1 < ntiles) {
            prefetch(b ^ 1, (t + 1) * kSkBK);
            asm volatile("cp.async.wait_group 1;" ::: "memory");  // tile t has landed
        } else {
            asm volatile("cp.async.wait_group 0;" ::: "memory");
        }
        __syncthreads();
        const float2(*sS)[SW + 1] = bufS(b);
        const float2(*sL)[LW + 1] = bufL(b);
        float tr[4][4], ti[4][4];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) tr[i][j] = ti[i][j] = 0.f;
#pragma unroll 4
        for (int kk = g * 16; kk < g * 16 + 16; ++kk) {
            float2 a[4], bb[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = sS[kk][sg + RS * i];
#pragma unroll
            for (int j = 0; j < 4; ++j) bb[j] = sL[kk][lg + CS * j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    tr[i][j] = fmaf(a[i].x, bb[j].x, tr[i][j]);
                    tr[i][j] = fmaf(-a[i].y, bb[j].y, tr[i][j]);
                    ti[i][j] = fmaf(a[i].x, bb[j].y, ti[i][j]);
                    ti[i][j] = fmaf(a[i].y, bb[j].x, ti[i][j]);
                }
        }
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                cr[i][j] += tr[i][j];
                ci[i][j] += ti[i][j];
            }
        __syncthreads();  // buffer b is refilled by the prefetch of tile t + 2
    }
    // add the four groups' sums in group order (through the buffers, idle after the last
    // barrier: 4 x 1024 float2 <= 2 buffers)
    float2 *red = skmem;
    static_assert(4 * 1024 <= 2 * (kSkS + kSkL), "reduction space");
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
            red[(g * SW + sg + RS * i) * LW + lg + CS * j] = make_float2(cr[i][j], ci[i][j]);
    __syncthreads();
    const int64_t MN = (int64_t)S * L;
    float2 *P = d.partial + ((int64_t)blockIdx.z * gridDim.y + s) * MN;
    for (int e = tid; e < SW * LW; e += 256) {
        const int si = e / LW, li = e % LW;
        if (si >= S || li >= L) continue;
        float re = 0.f, im = 0.f;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const float2 v = red[(q * SW + si) * LW + li];
            re += v.x;
            im += v.y;
        }
        // row-major M x N: (m, n) = (si, li), or (li, si) when the roles were swapped
        P[swap ? (int64_t)li * S + si : (int64_t)si * L + li] = make_float2(re, im);
    }
}

// Sum of the split-K partials in increasing split order, scattered into C's order.
__global__ void k_splitk_reduce(GemmDesc d, int64_t slices) {
    const int64_t MN = 1ll << (d.lm + d.ln);
    const int64_t total = slices * MN;
    const uint64_t nmask = (1ull << d.ln) - 1;
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int64_t s = idx / MN, e = idx % MN;
        float re = 0.f, im = 0.f;
        for (int z = 0; z < d.splits; ++z) {
            const float2 v = d.partial[((int64_t)z * slices + s) * MN + e];
            re += v.x;
            im += v.y;
        }
        const uint64_t m = (uint64_t)e >> d.ln, n = (uint64_t)e & nmask;
        d.C[s * d.sC + (int64_t)(deposit(m, d.lm, d.posC_m) | deposit(n, d.ln, d.posC_n))] =
            make_float2(re, im);
        if (d.amax_out) atomicMax(d.amax_out + s, __float_as_uint(fmaxf(fabsf(re), fabsf(im))));
    }
}

// Thin steps (the low-intensity contractions of App. A.2): C[m, n] = sum_k A[m, k] B[n, k] with
// few columns (N = NT <= 16) and a contraction of K <= 1024 (summed in one FP32 chain per
// output).  One thread owns one row m of A and all NT outputs of that row; a
// tile is 256 rows.  B is held in shared memory as [K][NT] and read as broadcast 16-byte pairs,
// or, in the walking form with NT * K <= 16, in every thread's registers (those steps would
// otherwise spend most of the L1 / shared-memory pipe on the broadcasts).
// For K <= 8 and NT <= 8, or K <= 16 and NT = 16 (KS = K; 2 blocks per SM, the two output
// stages in dynamic shared memory), the grid holds as many blocks as fit on the GPU, each walking its slice's
// tiles with a stride: a thread loads its own row of A straight into registers (K * 8 contiguous
// bytes; a warp reads one contiguous span) and fetches its row of the next tile before it stores
// the current one, so loads stay in flight during the store phase; two output stages taken in
// turn leave one block barrier per tile.  For longer K (KS = 0) a block
// takes one tile and stages its rows through shared memory in chunks of 16 of K with coalesced
// 16-byte loads.  A step whose small operand is A runs with the roles swapped (the complex
// product commutes).  Each tile (256 x NT) is staged and written in C's order with 8 consecutive
// elements per thread, as in the other epilogues.
constexpr int kThinRows = 256, kThinKC = 16, kThinLd = kThinKC + 1;
// blocks per SM the launch bounds guarantee: the walking form keeps its rows of A in registers
// (two tiles' worth), so 16 columns with it fit 2 blocks
constexpr int thin_min_blocks(int nt, int ks) {
    return ks && nt == 16 ? 2 : ((ks && nt < 8) ? 4 : 3);
}
// the walking form holds a small operand of at most 16 complex values in registers (every
// thread the same values), so the inner loop reads no shared memory at all; larger ones stay
// in shared memory, read as broadcast 16-byte pairs
constexpr bool thin_b_in_regs(int nt, int ks) { return ks != 0 && nt * ks <= 16; }
// the walking form with 16 columns stages its two output tiles in dynamic shared memory
constexpr bool thin_dyn_smem(int nt, int ks) { return ks != 0 && nt == 16; }
constexpr int thin_dyn_bytes(int nt) { return 2 * kThinRows * (nt + 1) * 8; }

template <int NT, int KS, bool PL>
__global__ void __launch_bounds__(256, thin_min_blocks(NT, KS)) k_gemm_thin(GemmDesc d) {
    constexpr int NB = NT < 2 ? 2 : NT;  // row stride of sB (pairs stay 16-byte aligned)
    constexpr int LD = NT + 1;           // row stride of the output stage
    // KS > 0: two output stages used in turn (one barrier per tile); KS = 0: rows of A, then
    // the stage
    constexpr bool DYN = thin_dyn_smem(NT, KS);
    __shared__ __align__(16) float2 sA_st[DYN ? 2 : (KS ? 2 * kThinRows * LD : kThinRows * kThinLd)];
    extern __shared__ __align__(16) float2 sA_dyn[];
    float2 *sA = DYN ? sA_dyn : sA_st;
    constexpr bool BREG = thin_b_in_regs(NT, KS);
    __shared__ __align__(16) float2 sB[BREG ? 2 : (KS ? KS : 64) * NB];
    const int64_t s = blockIdx.y;
    const int K = KS ? KS : 1 << d.lk;
    const float2 *As = d.A + s * d.sA;
    const float2 *B = d.B + s * d.sB;
    const int tid = threadIdx.x;
    float cr[NT], ci[NT];
    auto mac = [&](const float2 a, const float2 *bk) {
#pragma unroll
        for (int n = 0; n < NT; n += 2) {
            float2 b0, b1;
            if (NT >= 2) {
                const float4 bb = *reinterpret_cast<const float4 *>(bk + n);
                b0 = make_float2(bb.x, bb.y);
                b1 = make_float2(bb.z, bb.w);
            } else {
                b0 = bk[0];
                b1 = b0;
            }
            cr[n] = fmaf(a.x, b0.x, cr[n]);
            cr[n] = fmaf(-a.y, b0.y, cr[n]);
            ci[n] = fmaf(a.x, b0.y, ci[n]);
            ci[n] = fmaf(a.y, b0.x, ci[n]);
            if (n + 1 < NT) {
                cr[n + 1] = fmaf(a.x, b1.x, cr[n + 1]);
                cr[n + 1] = fmaf(-a.y, b1.y, cr[n + 1]);
                ci[n + 1] = fmaf(a.x, b1.y, ci[n + 1]);
                ci[n + 1] = fmaf(a.y, b1.x, ci[n + 1]);
            }
        }
    };
    // output: stage rows with stride NT + 1, then write 8 consecutive elements of C per task
    auto soff = [&](int sq) { return (sq & 128) ? (LD << (sq & 127)) : (1 << sq); };
    int w8[8];
    {
        const int d0 = soff(d.tb_src[0]), d1 = soff(d.tb_src[1]), d2 = soff(d.tb_src[2]);
#pragma unroll
        for (int j = 0; j < 8; ++j)
            w8[j] = ((j & 1) ? d0 : 0) + ((j & 2) ? d1 : 0) + ((j & 4) ? d2 : 0);
    }
    // a tile has 256 * NT elements (tile_bits = 8 + log2 NT): 32 * NT runs of 8 consecutive
    // elements of C; their stage and C offsets are the same for every tile, so they are set once
    constexpr int TASKS = kThinRows * NT / 8;
    // two lanes share each run of 8, so every thread has stores to make: for complex64 results
    // lane half h writes elements 4j + 2h and 4j + 2h + 1 in its store j (each store instruction
    // fills whole 32-byte sectors); for planar 16-bit results (PL, a separate instantiation)
    // lane half h writes elements 4h .. 4h + 3, 8 bytes per plane (a warp's stores cover 256
    // contiguous bytes of each plane)
    constexpr int SUBS = TASKS * 2, SPT = (SUBS + 255) / 256;
    int ws[SPT];
    uint64_t os[SPT];
    const int d0 = w8[1], d1 = w8[2], d2 = w8[4];
#pragma unroll
    for (int i = 0; i < SPT; ++i) {
        const int u = tid + 256 * i, r = u >> 1, h = u & 1;
        ws[i] = h ? (PL ? d2 : d1) : 0;
        os[i] = h ? (PL ? 4 : 2) : 0;
        for (int q = 3; q < d.tile_bits; ++q)
            if ((r >> (q - 3)) & 1) {
                ws[i] += soff(d.tb_src[q]);
                os[i] |= 1ull << d.tb_pos[q];
            }
    }
    float amx = 0.f;
    // a result that feeds a tensor-core step is written as its scaled planar 16-bit copy, with
    // the exponent bounded from the inputs' max-abs (as in the other epilogues)
    const int eo = PL ? planar_out_exponent(d.pout, s) : 0;
    if (PL && blockIdx.x == 0 && tid == 0) d.pout.exps[s] = eo;
    // write the tile whose C offset (its rows' deposit) is cbase through `stage`; callers make
    // sure no thread still reads `stage` from an earlier tile
    auto emit = [&](float2 *stage, uint64_t cbase) {
#pragma unroll
        for (int n = 0; n < NT; ++n) stage[tid * LD + n] = make_float2(cr[n], ci[n]);
        __syncthreads();
        float2 *C = d.C + s * d.sC + cbase;
        if constexpr (PL) {
#pragma unroll
            for (int i = 0; i < SPT; ++i) {
                if (SUBS % 256 != 0 && tid + 256 * i >= SUBS) break;
                float2 v[4];
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    v[j] = stage[ws[i] + w8[j]];
                    amx = fmaxf(amx, fmaxf(fabsf(v[j].x), fabsf(v[j].y)));
                }
                planar_out_store4(d.pout, s, cbase | os[i], v, eo);
            }
        } else {
#pragma unroll
            for (int i = 0; i < SPT; ++i) {
                if (SUBS % 256 != 0 && tid + 256 * i >= SUBS) break;
#pragma unroll
                for (int j = 0; j < 2; ++j) {
                    const int w = ws[i] + (j ? d2 : 0);
                    const float2 v0 = stage[w], v1 = stage[w + d0];
                    amx = fmaxf(amx, fmaxf(fmaxf(fabsf(v0.x), fabsf(v0.y)),
                                           fmaxf(fabsf(v1.x), fabsf(v1.y))));
                    *reinterpret_cast<float4 *>(C + (os[i] + 4 * j)) =
                        make_float4(v0.x, v0.y, v1.x, v1.y);
                }
            }
        }
    };
    if constexpr (KS != 0) {
        const int64_t tiles = (1ll << d.lm) / kThinRows;
        float2 a[KS], an[KS];
        auto fetch = [&](float2 *dst, int64_t t) {
            const float4 *Ar =
                reinterpret_cast<const float4 *>(As + (t * kThinRows + tid) * KS);
#pragma unroll
            for (int q = 0; q < KS / 2; ++q) {
                const float4 v = Ar[q];
                dst[2 * q] = make_float2(v.x, v.y);
                dst[2 * q + 1] = make_float2(v.z, v.w);
            }
        };
        // C offset of tile t: deposit(t * 256), its 8 low bits zero; the warp's lanes take one
        // bit each and OR their contributions
        auto tile_base = [&](int64_t t) {
            uint64_t r = 0;
            for (int i = 8 + (tid & 31); i < d.lm; i += 32)
                if (((uint64_t)t >> (i - 8)) & 1ull) r |= 1ull << d.posC_m[i];
            const uint32_t lo = __reduce_or_sync(0xffffffffu, (uint32_t)r);
            const uint32_t hi = __reduce_or_sync(0xffffffffu, (uint32_t)(r >> 32));
            return ((uint64_t)hi << 32) | lo;
        };
        int64_t t = blockIdx.x;  // < tiles: the launch makes at most one block per tile
        fetch(a, t);
        float2 breg[BREG ? KS * NT : 1];
        if constexpr (BREG) {
#pragma unroll
            for (int e = 0; e < NT * KS; ++e) breg[(e % KS) * NT + e / KS] = B[e];
        } else {
            for (int e = tid; e < NT * KS; e += 256) {
                const int n = e / KS, k = e % KS;
                sB[k * NB + n] = B[e];
            }
            __syncthreads();
        }
        int buf = 0;
        for (; t < tiles; t += gridDim.x) {
            if (t + gridDim.x < tiles) fetch(an, t + gridDim.x);
#pragma unroll
            for (int n = 0; n < NT; ++n) cr[n] = ci[n] = 0.f;
            if constexpr (BREG) {
#pragma unroll
                for (int k = 0; k < KS; ++k)
#pragma unroll
                    for (int n = 0; n < NT; ++n) {
                        const float2 b = breg[k * NT + n];
                        cr[n] = fmaf(a[k].x, b.x, cr[n]);
                        cr[n] = fmaf(-a[k].y, b.y, cr[n]);
                        ci[n] = fmaf(a[k].x, b.y, ci[n]);
                        ci[n] = fmaf(a[k].y, b.x, ci[n]);
                    }
            } else {
#pragma unroll
                for (int k = 0; k < KS; ++k) mac(a[k], sB + k * NB);
            }
            // stage `buf` was last read two tiles ago, before every thread passed the barrier
            // inside the previous tile's emit
            emit(sA + buf * kThinRows * LD, tile_base(t));
            buf ^= 1;
#pragma unroll
            for (int k = 0; k < KS; ++k) a[k] = an[k];
        }
    } else {
        const int64_t m0 = (int64_t)blockIdx.x * kThinRows;
        const float2 *A = As + m0 * K;
#pragma unroll
        for (int n = 0; n < NT; ++n) cr[n] = ci[n] = 0.f;
        // the small operand 64 of K at a time (K up to 1024), the rows of A 16 of K at a time
        for (int kb = 0; kb < K; kb += 64) {
            const int kbw = K - kb < 64 ? K - kb : 64;
            __syncthreads();  // every thread is done with the previous part of sB
            for (int e = tid; e < NT * kbw; e += 256) {
                const int n = e / kbw, k = e % kbw;
                sB[k * NB + n] = B[(int64_t)n * K + kb + k];
            }
            for (int kc = kb; kc < kb + kbw; kc += kThinKC) {
                const int kw = kb + kbw - kc < kThinKC ? kb + kbw - kc : kThinKC;  // 2^j >= 2
                const int hp = kw >> 1;  // 16-byte pairs per row
                __syncthreads();
                for (int e = tid; e < kThinRows * hp; e += 256) {
                    const int r = e / hp, q = e % hp;
                    const float4 v =
                        *reinterpret_cast<const float4 *>(A + (int64_t)r * K + kc + 2 * q);
                    sA[r * kThinLd + 2 * q] = make_float2(v.x, v.y);
                    sA[r * kThinLd + 2 * q + 1] = make_float2(v.z, v.w);
                }
                __syncthreads();
                for (int k = 0; k < kw; ++k)
                    mac(sA[tid * kThinLd + k], sB + (kc - kb + k) * NB);
            }
        }
        __syncthreads();  // the stage reuses sA
        emit(sA, deposit((uint64_t)m0, d.lm, d.posC_m));
    }
    if (d.amax_out) amax_publish(d.amax_out + s, amx);
}

// Thin sparse-state step (at most 16 columns): thread per (configuration c, row m) holding all
// NN outputs of its row; B[gB[c]] is staged in shared memory 64 values of k at a time, so each
// element of A is read once.  Block = 256 rows of one configuration.
template <int NN>
__global__ void __launch_bounds__(256) k_sparse_thin(GenericDesc d, const int32_t *gA,
                                                     const int32_t *gB, int64_t mblocks) {
    constexpr int KC = 64;
    __shared__ float2 Bs[KC][NN];
    __shared__ uint64_t offak[KC], offbk[KC];
    constexpr int ln = NN == 1 ? 0 : NN == 2 ? 1 : NN == 4 ? 2 : NN == 8 ? 3 : 4;  // NN = 2^ln
    const int lm = d.rank_c - ln, nk = d.nk;
    const int64_t c = (int64_t)blockIdx.x / mblocks;
    const int64_t m = ((int64_t)blockIdx.x % mblocks) * 256 + threadIdx.x;
    const int64_t M = 1ll << lm, K = 1ll << nk;
    const float2 *A = d.A + (int64_t)gA[c] * d.sA;
    const float2 *B = d.B + (int64_t)gB[c] * d.sB;
    const bool row_ok = m < M;
    const uint64_t offm = row_ok ? deposit((uint64_t)m, lm, d.posA_c + ln) : 0;
    float cr[NN], ci[NN];
#pragma unroll
    for (int n = 0; n < NN; ++n) cr[n] = ci[n] = 0.f;
    for (int64_t k0 = 0; k0 < K; k0 += KC) {
        const int kc = (int)(K - k0 < KC ? K - k0 : KC);
        __syncthreads();  // the previous chunk is consumed
        if (threadIdx.x < kc) {
            offak[threadIdx.x] = deposit((uint64_t)(k0 + threadIdx.x), nk, d.posA_k);
            offbk[threadIdx.x] = deposit((uint64_t)(k0 + threadIdx.x), nk, d.posB_k);
        }
        __syncthreads();
        for (int e = threadIdx.x; e < kc * NN; e += blockDim.x) {
            const int kk = e / NN, n = e % NN;
            Bs[kk][n] = B[deposit((uint64_t)n, ln, d.posB_c) | offbk[kk]];
        }
        __syncthreads();
        if (row_ok)
            for (int kk = 0; kk < kc; ++kk) {
                const float2 a = A[offm | offak[kk]];
#pragma unroll
                for (int n = 0; n < NN; ++n) {
                    const float2 b = Bs[kk][n];
                    cr[n] = fmaf(a.x, b.x, cr[n]);
                    cr[n] = fmaf(-a.y, b.y, cr[n]);
                    ci[n] = fmaf(a.x, b.y, ci[n]);
                    ci[n] = fmaf(a.y, b.x, ci[n]);
                }
            }
    }
    if (row_ok) {
        float2 *Cc = d.C + c * d.sC + m * NN;
#pragma unroll
        for (int n = 0; n < NN; ++n) Cc[n] = make_float2(cr[n], ci[n]);
    }
}

// Grouped sparse-state step (see SparseGroupDesc): one 64 x 64 tile of one group's GEMM per CTA.
// Row r / column q of the tile resolve to an operand element offset (without k) and a part of
// the result offset, so C[(row part) + (column part)] = sum_k A[rowA + offA(k)] B[colB + offB(k)].
template <int BK>
__global__ void __launch_bounds__(256) k_sparse_group(GenericDesc d, int32_t ln,
                                                      SparseGroupDesc g) {
    __shared__ __align__(16) float2 As[2][BK][BM + 1];
    __shared__ __align__(16) float2 Bs[2][BK][BN + 1];
    __shared__ int64_t rowA[BM], colB[BN], outR[BM], outC[BN];
    __shared__ uint64_t kofA[2][BK], kofB[2][BK];  // operand offsets of the K chunk's elements
    const int lm = d.rank_c - ln, nk = d.nk;
    const int64_t M = 1ll << lm, N = 1ll << ln, K = 1ll << nk;
    const int32_t *t = g.tiles + 3 * (int64_t)blockIdx.x;
    const int grp = t[0];
    const int64_t r0 = (int64_t)t[1] * BM, q0 = (int64_t)t[2] * BN;
    const int64_t off = g.grp_off[grp], len = g.grp_len[grp];
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    // rows: m of A (grouped by A) or (member, m) (grouped by B); columns likewise for n of B
    const int64_t rows = g.by_a ? M : len * M, cols = g.by_a ? len * N : N;
    if (tid < BM) {
        const int64_t r = r0 + tid;
        int64_t ra = -1, orow = 0;
        if (r < rows) {
            const int64_t m = g.by_a ? r : (r & (M - 1));
            const int64_t c = g.by_a ? g.members[off] : g.members[off + (r >> lm)];
            ra = (int64_t)g.gA[c] * d.sA + (int64_t)deposit((uint64_t)m, lm, d.posA_c + ln);
            orow = (g.by_a ? 0 : c * d.sC) + m * N;
        }
        rowA[tid] = ra;
        outR[tid] = orow;
    } else if (tid < BM + BN) {
        const int j = tid - BM;
        const int64_t q = q0 + j;
        int64_t cb = -1, ocol = 0;
        if (q < cols) {
            const int64_t n = g.by_a ? (q & (N - 1)) : q;
            const int64_t c = g.by_a ? g.members[off + (q >> ln)] : g.members[off];
            cb = (int64_t)g.gB[c] * d.sB + (int64_t)deposit((uint64_t)n, ln, d.posB_c);
            ocol = (g.by_a ? c * d.sC : 0) + n;
        }
        colB[j] = cb;
        outC[j] = ocol;
    }
    // K-chunk offset tables (deposits of k into A's and B's contracted bits): chunk kt uses
    // buffer kt & 1; threads 128.. fill a chunk's table before the barrier that precedes its
    // loads, two chunks ahead of its use
    auto koffs = [&](int64_t k0, int buf) {
        const int e = tid - 128;
        if (e >= 0 && e < BK) {
            const int64_t gk = k0 + e;
            kofA[buf][e] = gk < K ? deposit((uint64_t)gk, nk, d.posA_k) : 0;
            kofB[buf][e] = gk < K ? deposit((uint64_t)gk, nk, d.posB_k) : 0;
        }
    };
    koffs(0, 0);
    __syncthreads();
    constexpr int KQ = BK / 4;
    const int lr = tid >> 2, lk = (tid & 3) * KQ;
    float2 ra[KQ], rb[KQ];
    auto load = [&](int64_t k0, int buf) {
#pragma unroll
        for (int q = 0; q < KQ; ++q) {
            const bool kin = k0 + lk + q < K;
            ra[q] = (rowA[lr] >= 0 && kin) ? d.A[rowA[lr] + (int64_t)kofA[buf][lk + q]]
                                           : make_float2(0.f, 0.f);
            rb[q] = (colB[lr] >= 0 && kin) ? d.B[colB[lr] + (int64_t)kofB[buf][lk + q]]
                                           : make_float2(0.f, 0.f);
        }
    };
    auto store = [&](int buf) {
#pragma unroll
        for (int q = 0; q < KQ; ++q) {
            As[buf][lk + q][lr] = ra[q];
            Bs[buf][lk + q][lr] = rb[q];
        }
    };
    float cr[TM][TN], ci[TM][TN];
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) cr[i][j] = ci[i][j] = 0.f;
    load(0, 0);
    store(0);
    const int64_t ktiles = (K + BK - 1) / BK;
    if (ktiles > 1) koffs(BK, 1);
    __syncthreads();
    for (int64_t kt = 0; kt < ktiles; ++kt) {
        const int buf = kt & 1;
        if (kt + 1 < ktiles) load((kt + 1) * BK, buf ^ 1);
        // the table of chunk kt + 2 reuses buffer buf (its last reads were chunk kt's loads, in
        // the previous iteration); the barrier below publishes it before chunk kt + 2 loads
        if (kt + 2 < ktiles) koffs((kt + 2) * BK, buf);
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
            float2 a[TM], b[TN];
#pragma unroll
            for (int i = 0; i < TM; ++i) a[i] = As[buf][kk][ty + 16 * i];
#pragma unroll
            for (int j = 0; j < TN; ++j) b[j] = Bs[buf][kk][tx + 16 * j];
#pragma unroll
            for (int i = 0; i < TM; ++i)
#pragma unroll
                for (int j = 0; j < TN; ++j) {
                    cr[i][j] = fmaf(a[i].x, b[j].x, cr[i][j]);
                    cr[i][j] = fmaf(-a[i].y, b[j].y, cr[i][j]);
                    ci[i][j] = fmaf(a[i].x, b[j].y, ci[i][j]);
                    ci[i][j] = fmaf(a[i].y, b[j].x, ci[i][j]);
                }
        }
        if (kt + 1 < ktiles) store(buf ^ 1);
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < TM; ++i) {
        const int r = ty + 16 * i;
        if (rowA[r] < 0) continue;
#pragma unroll
        for (int j = 0; j < TN; ++j) {
            const int q = tx + 16 * j;
            if (colB[q] >= 0) d.C[outR[r] + outC[q]] = make_float2(cr[i][j], ci[i][j]);
        }
    }
}

// Sparse-state step with a dense GEMM inside each configuration (Sec. 3.3): for configuration c
// of the result, C[c][m][n] = sum_k A[gA[c]][m, k] B[gB[c]][n, k], where the operands' labels sit
// at arbitrary bit positions (offsets by deposit) and C is row-major over (A-only labels,
// B-only labels).  Same 64 x 64 tile and double-buffered shared-memory K loop as k_gemm_simt;
// grid x = tiles x configurations.
template <int BK>
__global__ void __launch_bounds__(256) k_sparse_gemm(GenericDesc d, int32_t ln, const int32_t *gA,
                                                     const int32_t *gB, int64_t tiles_m,
                                                     int64_t tiles_n) {
    __shared__ __align__(16) float2 As[2][BK][BM + 1];
    __shared__ __align__(16) float2 Bs[2][BK][BN + 1];
    __shared__ uint64_t offm[BM], offn[BN];
    const int lm = d.rank_c - ln, nk = d.nk;
    const int64_t tiles = tiles_m * tiles_n;
    const int64_t c = (int64_t)blockIdx.x / tiles;
    const int64_t tile = (int64_t)blockIdx.x % tiles;
    const int64_t m0 = (tile / tiles_n) * BM, n0 = (tile % tiles_n) * BN;
    const int64_t M = 1ll << lm, N = 1ll << ln, K = 1ll << nk;
    const float2 *A = d.A + (int64_t)gA[c] * d.sA;
    const float2 *B = d.B + (int64_t)gB[c] * d.sB;
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    if (tid < BM) offm[tid] = m0 + tid < M ? deposit((uint64_t)(m0 + tid), lm, d.posA_c + ln) : 0;
    else if (tid < BM + BN) {
        const int j = tid - BM;
        offn[j] = n0 + j < N ? deposit((uint64_t)(n0 + j), ln, d.posB_c) : 0;
    }
    __syncthreads();
    constexpr int KQ = BK / 4;
    const int lr = tid >> 2, lk = (tid & 3) * KQ;
    float2 ra[KQ], rb[KQ];
    auto load = [&](int64_t k0) {
        const int64_t gm = m0 + lr, gn = n0 + lr;
#pragma unroll
        for (int q = 0; q < KQ; ++q) {
            const int64_t gk = k0 + lk + q;
            const bool kin = gk < K;
            const uint64_t oka = kin ? deposit((uint64_t)gk, nk, d.posA_k) : 0;
            const uint64_t okb = kin ? deposit((uint64_t)gk, nk, d.posB_k) : 0;
            ra[q] = (gm < M && kin) ? A[offm[lr] | oka] : make_float2(0.f, 0.f);
            rb[q] = (gn < N && kin) ? B[offn[lr] | okb] : make_float2(0.f, 0.f);
        }
    };
    auto store = [&](int buf) {
#pragma unroll
        for (int q = 0; q < KQ; ++q) {
            As[buf][lk + q][lr] = ra[q];
            Bs[buf][lk + q][lr] = rb[q];
        }
    };
    float cr[TM][TN], ci[TM][TN];
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) cr[i][j] = ci[i][j] = 0.f;
    load(0);
    store(0);
    __syncthreads();
    const int64_t ktiles = (K + BK - 1) / BK;
    for (int64_t kt = 0; kt < ktiles; ++kt) {
        const int buf = kt & 1;
        if (kt + 1 < ktiles) load((kt + 1) * BK);
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
            float2 a[TM], b[TN];
#pragma unroll
            for (int i = 0; i < TM; ++i) a[i] = As[buf][kk][ty + 16 * i];
#pragma unroll
            for (int j = 0; j < TN; ++j) b[j] = Bs[buf][kk][tx + 16 * j];
#pragma unroll
            for (int i = 0; i < TM; ++i)
#pragma unroll
                for (int j = 0; j < TN; ++j) {
                    cr[i][j] = fmaf(a[i].x, b[j].x, cr[i][j]);
                    cr[i][j] = fmaf(-a[i].y, b[j].y, cr[i][j]);
                    ci[i][j] = fmaf(a[i].x, b[j].y, ci[i][j]);
                    ci[i][j] = fmaf(a[i].y, b[j].x, ci[i][j]);
                }
        }
        if (kt + 1 < ktiles) store(buf ^ 1);
        __syncthreads();
    }
    float2 *Cc = d.C + c * d.sC;
#pragma unroll
    for (int i = 0; i < TM; ++i) {
        const int64_t gm = m0 + ty + 16 * i;
        if (gm >= M) continue;
#pragma unroll
        for (int j = 0; j < TN; ++j) {
            const int64_t gn = n0 + tx + 16 * j;
            if (gn < N) Cc[gm * N + gn] = make_float2(cr[i][j], ci[i][j]);
        }
    }
}

}  // namespace

cudaError_t simt_prepare() {
    cudaError_t e = cudaSuccess;
    for (auto f : {k_gemm_thin<16, 2, false>, k_gemm_thin<16, 4, false>, k_gemm_thin<16, 8, false>,
                   k_gemm_thin<16, 16, false>, k_gemm_thin<16, 2, true>, k_gemm_thin<16, 4, true>,
                   k_gemm_thin<16, 8, true>, k_gemm_thin<16, 16, true>})
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     thin_dyn_bytes(16));
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_gemm_skinny<16>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, kSkSmem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_gemm_skinny<32>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 kSkSmem);
    return e;
}

cudaError_t launch_sparse_group(const GenericDesc &d, int32_t ln, const SparseGroupDesc &g,
                                cudaStream_t st) {
    if (g.ntiles <= 0) return cudaSuccess;
    if (g.ntiles > 0x7fffffffll || d.rank_c - ln < 0 || ln < 0) return cudaErrorInvalidValue;
    if (d.nk >= 4)
        k_sparse_group<16><<<(unsigned)g.ntiles, 256, 0, st>>>(d, ln, g);
    else
        k_sparse_group<8><<<(unsigned)g.ntiles, 256, 0, st>>>(d, ln, g);
    return cudaGetLastError();
}

cudaError_t launch_sparse_thin(const GenericDesc &d, int32_t ln, const int32_t *gA,
                               const int32_t *gB, int64_t nconf, cudaStream_t st) {
    if (nconf <= 0) return cudaSuccess;
    const int lm = d.rank_c - ln;
    if (lm < 0 || ln < 0 || ln > 4) return cudaErrorInvalidValue;
    const int64_t mblocks = ((1ll << lm) + 255) / 256;
    const int64_t blocks = mblocks * nconf;
    if (blocks > 0x7fffffffll) return cudaErrorInvalidValue;
    switch (ln) {
    case 0: k_sparse_thin<1><<<(unsigned)blocks, 256, 0, st>>>(d, gA, gB, mblocks); break;
    case 1: k_sparse_thin<2><<<(unsigned)blocks, 256, 0, st>>>(d, gA, gB, mblocks); break;
    case 2: k_sparse_thin<4><<<(unsigned)blocks, 256, 0, st>>>(d, gA, gB, mblocks); break;
    case 3: k_sparse_thin<8><<<(unsigned)blocks, 256, 0, st>>>(d, gA, gB, mblocks); break;
    default: k_sparse_thin<16><<<(unsigned)blocks, 256, 0, st>>>(d, gA, gB, mblocks); break;
    }
    return cudaGetLastError();
}

cudaError_t launch_sparse_gemm(const GenericDesc &d, int32_t ln, const int32_t *gA,
                               const int32_t *gB, int64_t nconf, cudaStream_t st) {
    if (nconf <= 0) return cudaSuccess;
    const int lm = d.rank_c - ln;
    if (lm < 0 || ln < 0 || d.nk < 1) return cudaErrorInvalidValue;
    const int64_t tiles_m = ((1ll << lm) + BM - 1) / BM, tiles_n = ((1ll << ln) + BN - 1) / BN;
    const int64_t blocks = tiles_m * tiles_n * nconf;
    if (blocks > 0x7fffffffll) return cudaErrorInvalidValue;
    if (d.nk >= 4)
        k_sparse_gemm<16><<<(unsigned)blocks, 256, 0, st>>>(d, ln, gA, gB, tiles_m, tiles_n);
    else
        k_sparse_gemm<8><<<(unsigned)blocks, 256, 0, st>>>(d, ln, gA, gB, tiles_m, tiles_n);
    return cudaGetLastError();
}

cudaError_t launch_gemm_simt(const GemmDesc &d, int64_t slices, cudaStream_t st) {
    const int64_t M = 1ll << d.lm, N = 1ll << d.ln;
    const int64_t tm = (M + BM - 1) / BM, tn_ = (N + BN - 1) / BN;
    if (tm * tn_ > 0x7fffffffll || slices > 65535 || d.splits < 1 || d.splits > 65535 ||
        ((1ll << d.lk) % d.splits) != 0 || (d.splits > 1 && !d.partial))
        return cudaErrorInvalidConfiguration;
    const dim3 grid((unsigned)(tm * tn_), (unsigned)slices, (unsigned)d.splits);
    const int lmin = d.lm < d.ln ? d.lm : d.ln, lmax = d.lm < d.ln ? d.ln : d.lm;
    const bool sk16 = lmin <= 4 && lmax <= 6, sk32 = lmin == 5 && lmax == 5;
    const bool skinny = d.splits > 1 && (sk16 || sk32) && (1ll << d.lk) / d.splits >= kSkBK;
    if (skinny && sk16)
        k_gemm_skinny<16><<<dim3(1, (unsigned)slices, (unsigned)d.splits), 256, kSkSmem, st>>>(d);
    else if (skinny)
        k_gemm_skinny<32><<<dim3(1, (unsigned)slices, (unsigned)d.splits), 256, kSkSmem, st>>>(d);
    else if (d.lk - (d.splits > 1 ? __builtin_ctz((unsigned)d.splits) : 0) <= 3)
        k_gemm_simt<8><<<grid, 256, 0, st>>>(d, tn_);
    else
        k_gemm_simt<16><<<grid, 256, 0, st>>>(d, tn_);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || d.splits == 1) return e;
    const int64_t total = slices << (d.lm + d.ln);
    int64_t blocks = (total + 255) / 256;
    if (blocks > 152 * 32) blocks = 152 * 32;
    k_splitk_reduce<<<(unsigned)blocks, 256, 0, st>>>(d, slices);
    return cudaGetLastError();
}

void sort_tile_bits(int tm, int tn, const int8_t *posC_m, const int8_t *posC_n, int row_tag,
                    int8_t *src, int8_t *pos) {
    int s_[32], p_[32], n = 0;
    for (int j = 0; j < tn; ++j) { s_[n] = j; p_[n] = posC_n[j]; ++n; }
    for (int i = 0; i < tm; ++i) { s_[n] = row_tag | i; p_[n] = posC_m[i]; ++n; }
    for (int a = 1; a < n; ++a)
        for (int b = a; b > 0 && p_[b - 1] > p_[b]; --b) {
            int t = p_[b]; p_[b] = p_[b - 1]; p_[b - 1] = t;
            t = s_[b]; s_[b] = s_[b - 1]; s_[b - 1] = t;
        }
    for (int q = 0; q < n; ++q) {
        src[q] = (int8_t)s_[q];
        pos[q] = (int8_t)p_[q];
    }
}

namespace {
// rank over GF(2) of n 4-bit vectors
int rank4(const int *v, int n) {
    int b[4] = {0, 0, 0, 0};  // b[i]: a reduced vector with leading bit i
    int r = 0;
    for (int k = 0; k < n; ++k) {
        int x = v[k] & 15;
        for (int i = 3; i >= 0 && x; --i)
            if ((x >> i) & 1) {
                if (!b[i]) {
                    b[i] = x;
                    ++r;
                    x = 0;
                } else {
                    x ^= b[i];
                }
            }
    }
    return r;
}
}  // namespace

int thin_choose_swizzle(const int8_t *tb_src, int lnt, bool planar, int8_t *phi) {
    // the 8-byte bank pair (0..15) of element (r, c) is ((r << lnt) & 15) | (c ^ phi(r)): a row
    // bit i adds bit lnt + i (when below 4) and phi[i]; a column bit k adds bit k
    const int nt = 1 << lnt;
    int ph[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int k = 0; k < lnt; ++k) ph[4 - lnt + k] = 1 << k;  // rows 0-3 spread over the banks
    auto vec = [&](int sq, const int *f) {
        if (sq & 128) {
            const int i = sq & 127;
            return (lnt + i < 4 ? 1 << (lnt + i) : 0) | (i < 8 ? f[i] : 0);
        }
        return 1 << sq;
    };
    const int rbits[4] = {128, 129, 130, 131};
    const int rd[4] = {planar ? tb_src[3] : tb_src[1], tb_src[planar ? 4 : 3],
                       tb_src[planar ? 5 : 4], tb_src[planar ? 6 : 5]};
    auto score = [&](const int *f) {
        int w[4], r[4];
        for (int q = 0; q < 4; ++q) {
            w[q] = vec(rbits[q], f);
            r[q] = vec(rd[q], f);
        }
        return (rank4(w, 4) == 4 ? 1 : 0) + (rank4(r, 4) == 4 ? 1 : 0);
    };
    int best = score(ph), best_ph[8];
    for (int i = 0; i < 8; ++i) best_ph[i] = ph[i];
    if (best < 2 && lnt > 0) {
        // try every phi on the row bits the reads span (at most 4 of them, 16^4 cases)
        int rows[4], nr = 0;
        for (int q = 0; q < 4; ++q)
            if ((rd[q] & 128) && (rd[q] & 127) < 8) rows[nr++] = rd[q] & 127;
        int total = 1;
        for (int q = 0; q < nr; ++q) total *= nt;
        for (int code = 0; code < total && best < 2; ++code) {
            int f[8];
            for (int i = 0; i < 8; ++i) f[i] = ph[i];
            int c = code;
            for (int q = 0; q < nr; ++q) {
                f[rows[q]] = c % nt;
                c /= nt;
            }
            const int sc = score(f);
            if (sc > best) {
                best = sc;
                for (int i = 0; i < 8; ++i) best_ph[i] = f[i];
            }
        }
    }
    for (int i = 0; i < 8; ++i) phi[i] = (int8_t)best_ph[i];
    return best;
}

// Number of K splits for a CUDA-core GEMM step: enough CTAs to fill the GPU a few times when
// the output tiles alone cannot, with at least 256 contracted elements per split.
int gemm_simt_splits(int lm, int ln, int lk, int64_t slices) {
    const int lmin = lm < ln ? lm : ln, lmax = lm < ln ? ln : lm;
    if (((lmin <= 4 && lmax <= 6) || (lmin == 5 && lmax == 5)) && lk >= 11) {
        // skinny (the whole output is one CTA's tile): about 16 CTAs per SM in total, each with
        // at least 1024 contracted elements
        const int64_t want = (16 * 152 + slices - 1) / slices;
        int sp = 1;
        while (sp < want && (1ll << lk) / (sp * 2) >= 1024 && sp < 4096) sp *= 2;
        return sp;
    }
    const int64_t tiles = ((1ll << lm) + BM - 1) / BM * (((1ll << ln) + BN - 1) / BN) * slices;
    int splits = 1;
    while (tiles * splits < 4 * 152 && (lk - 8) > 0 && (1ll << lk) / (splits * 2) >= 256 &&
           splits < 4096)
        splits *= 2;
    return splits;
}

// Blocks per slice for the tile-walking variant: the blocks its launch bounds guarantee on every
// SM, spread over the slices, at most one per tile.  (Only attribute queries here: the launch may
// be under stream capture.)
template <int NT, int KS>
void launch_thin_walk(const GemmDesc &d, dim3 grid, cudaStream_t st) {
    static int sms = 0;
    if (sms == 0) {
        int dev = 0, v = 0;
        if (cudaGetDevice(&dev) == cudaSuccess &&
            cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess)
            sms = v;
        if (sms <= 0) sms = 152;
    }
    const int64_t resident = (int64_t)sms * thin_min_blocks(NT, KS);
    const int64_t per_slice = (resident + grid.y - 1) / grid.y;
    if (per_slice < (int64_t)grid.x) grid.x = (unsigned)per_slice;
    const int dyn = thin_dyn_smem(NT, KS) ? thin_dyn_bytes(NT) : 0;
    if (d.planar_out) k_gemm_thin<NT, KS, true><<<grid, 256, dyn, st>>>(d);
    else k_gemm_thin<NT, KS, false><<<grid, 256, dyn, st>>>(d);
}

template <int NT>
void launch_thin_long(const GemmDesc &d, dim3 grid, cudaStream_t st) {
    if (d.planar_out) k_gemm_thin<NT, 0, true><<<grid, 256, 0, st>>>(d);
    else k_gemm_thin<NT, 0, false><<<grid, 256, 0, st>>>(d);
}

template <int NT>
void launch_thin_n(const GemmDesc &d, dim3 grid, cudaStream_t st) {
    if constexpr (NT == 16) {  // 16 columns: the walking form up to K = 16, 2 blocks per SM
        switch (d.lk) {
            case 1: launch_thin_walk<NT, 2>(d, grid, st); break;
            case 2: launch_thin_walk<NT, 4>(d, grid, st); break;
            case 3: launch_thin_walk<NT, 8>(d, grid, st); break;
            case 4: launch_thin_walk<NT, 16>(d, grid, st); break;
            default: launch_thin_long<NT>(d, grid, st); break;
        }
    } else {
        switch (d.lk) {
            case 1: launch_thin_walk<NT, 2>(d, grid, st); break;
            case 2: launch_thin_walk<NT, 4>(d, grid, st); break;
            case 3: launch_thin_walk<NT, 8>(d, grid, st); break;
            default: launch_thin_long<NT>(d, grid, st); break;
        }
    }
}

cudaError_t launch_gemm_thin(const GemmDesc &d, int64_t slices, cudaStream_t st) {
    if (d.lm < 8 || d.ln < 0 || d.ln > 4 || d.lk < 1 || d.lk > 10 || slices > 65535 ||
        d.tile_bits != 8 + d.ln || d.tile_bits < 3)
        return cudaErrorInvalidConfiguration;
    const dim3 grid((unsigned)((1ll << d.lm) / kThinRows), (unsigned)slices);
    switch (d.ln) {
        case 0: launch_thin_n<1>(d, grid, st); break;
        case 1: launch_thin_n<2>(d, grid, st); break;
        case 2: launch_thin_n<4>(d, grid, st); break;
        case 3: launch_thin_n<8>(d, grid, st); break;
        default: launch_thin_n<16>(d, grid, st); break;
    }
    return cudaGetLastError();
}

}  // namespace tn
