// Complex64 GEMM on the CUDA cores (FP32 FMA, 4 real products per complex multiply-add):
// C[m, n] = sum_k A[m, k] * B[n, k] per slice, A = [M][K] and B = [N][K] row-major, the result
// scattered into the consumer's memory order (the index reordering of Sec. 4.1 applied at the
// producer's store, so no separate transpose pass is needed).
#include "tn_internal.h"

namespace tn {

namespace {

constexpr int BM = 64, BN = 64, BK = 16, TM = 4, TN = 4;

__device__ __forceinline__ uint64_t deposit(uint64_t x, int n, const int8_t *pos) {
    uint64_t r = 0;
    for (int i = 0; i < n; ++i)
        if ((x >> i) & 1ull) r |= 1ull << pos[i];
    return r;
}

// 256 threads as 16 x 16; each thread owns rows ty + 16*i and columns tx + 16*j (i, j < 4).
__global__ void __launch_bounds__(256) k_gemm_simt(GemmDesc d, int64_t tiles_n) {
    __shared__ float2 As[2][BK][BM + 1];
    __shared__ float2 Bs[2][BK][BN + 1];
    const int64_t s = blockIdx.y;
    const int64_t tile = blockIdx.x;
    const int64_t m0 = (tile / tiles_n) * BM, n0 = (tile % tiles_n) * BN;
    const int64_t M = 1ll << d.lm, N = 1ll << d.ln, K = 1ll << d.lk;
    const float2 *A = d.A + s * d.sA;
    const float2 *B = d.B + s * d.sB;
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;

    // global -> shared mapping: 64 rows x 16 k; thread loads row (tid >> 2), k (tid & 3) * 4..+3
    const int lr = tid >> 2, lk = (tid & 3) * 4;
    float2 ra[4], rb[4];
    auto load = [&](int64_t k0) {
        const int64_t gm = m0 + lr, gn = n0 + lr;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int64_t gk = k0 + lk + q;
            ra[q] = (gm < M && gk < K) ? A[gm * K + gk] : make_float2(0.f, 0.f);
            rb[q] = (gn < N && gk < K) ? B[gn * K + gk] : make_float2(0.f, 0.f);
        }
    };
    auto store = [&](int buf) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
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

    float2 *C = d.C + s * d.sC;
    uint64_t coff[TN];
#pragma unroll
    for (int j = 0; j < TN; ++j) coff[j] = deposit((uint64_t)(n0 + tx + 16 * j), d.ln, d.posC_n);
#pragma unroll
    for (int i = 0; i < TM; ++i) {
        const int64_t gm = m0 + ty + 16 * i;
        if (gm >= M) continue;
        const uint64_t roff = deposit((uint64_t)gm, d.lm, d.posC_m);
#pragma unroll
        for (int j = 0; j < TN; ++j) {
            const int64_t gn = n0 + tx + 16 * j;
            if (gn < N) C[roff | coff[j]] = make_float2(cr[i][j], ci[i][j]);
        }
    }
}

}  // namespace

cudaError_t launch_gemm_simt(const GemmDesc &d, int64_t slices, cudaStream_t st) {
    const int64_t M = 1ll << d.lm, N = 1ll << d.ln;
    const int64_t tm = (M + BM - 1) / BM, tn_ = (N + BN - 1) / BN;
    if (tm * tn_ > 0x7fffffffll || slices > 65535) return cudaErrorInvalidConfiguration;
    k_gemm_simt<<<dim3((unsigned)(tm * tn_), (unsigned)slices), 256, 0, st>>>(d, tn_);
    return cudaGetLastError();
}

}  // namespace tn
