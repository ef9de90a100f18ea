// CUDA-core kernels of the contraction engine: element-wise contraction of small steps, slice
// binding of the leaves (Sec. 3.2), FP64 cross-slice accumulation and readout (Eq. lxeb_2), and
// the per-tensor power-of-two scaling into planar 16-bit storage (Sec. 4.2, dynamic scaling).
#include <cuda_fp16.h>
#include <cuda_bf16.h>

#include "tn_internal.h"

namespace tn {

namespace {

__device__ __forceinline__ uint64_t deposit(uint64_t x, int n, const int8_t *pos) {
    uint64_t r = 0;
    for (int i = 0; i < n; ++i)
        if (((x >> i) & 1ull) && pos[i] >= 0) r |= 1ull << pos[i];
    return r;
}

// One thread per output element of C (in C's own memory order, so stores are coalesced),
// summing over the contracted bits in increasing order.  A block walks chunks of 2^LB
// consecutive outputs; the operand offsets of the chunk's low LB bits come from shared-memory
// tables built once per block, those of the high bits are computed once per chunk.
__global__ void __launch_bounds__(256) k_generic(GenericDesc d, int64_t total) {
    __shared__ uint64_t koffA[1024], koffB[1024];
    __shared__ uint64_t loA[1024], loB[1024];
    const int nk = d.nk;
    const bool table = nk <= 10;
    const int lb = d.rank_c < 10 ? d.rank_c : 10;
    for (int j = threadIdx.x; j < (1 << lb); j += blockDim.x) {
        loA[j] = deposit((uint64_t)j, lb, d.posA_c);
        loB[j] = deposit((uint64_t)j, lb, d.posB_c);
    }
    if (table) {
        for (int k = threadIdx.x; k < (1 << nk); k += blockDim.x) {
            koffA[k] = deposit((uint64_t)k, nk, d.posA_k);
            koffB[k] = deposit((uint64_t)k, nk, d.posB_k);
        }
    }
    __syncthreads();
    const uint64_t cmask = (d.rank_c >= 63) ? ~0ull : ((1ull << d.rank_c) - 1);
    const int64_t nchunks = total >> lb;
    const int64_t K = 1ll << nk;
    for (int64_t ch = blockIdx.x; ch < nchunks; ch += gridDim.x) {
        const int64_t base = ch << lb;
        const int64_t s = base >> d.rank_c;
        const uint64_t c0 = (uint64_t)base & cmask;
        const uint64_t hA = deposit(c0 >> lb, d.rank_c - lb, d.posA_c + lb);
        const uint64_t hB = deposit(c0 >> lb, d.rank_c - lb, d.posB_c + lb);
        const float2 *Ab = d.A + s * d.sA + hA;
        const float2 *Bb = d.B + s * d.sB + hB;
        float2 *Cb = d.C + s * d.sC + (int64_t)c0;
        float amx = 0.f;
        for (int j = threadIdx.x; j < (1 << lb); j += blockDim.x) {
            const float2 *A = Ab + loA[j];
            const float2 *B = Bb + loB[j];
            float re = 0.f, im = 0.f;
            for (int64_t k = 0; k < K; ++k) {
                uint64_t oa, ob;
                if (table) {
                    oa = koffA[k];
                    ob = koffB[k];
                } else {
                    oa = deposit((uint64_t)k, nk, d.posA_k);
                    ob = deposit((uint64_t)k, nk, d.posB_k);
                }
                const float2 a = A[oa], b = B[ob];
                re = fmaf(a.x, b.x, re);
                re = fmaf(-a.y, b.y, re);
                im = fmaf(a.x, b.y, im);
                im = fmaf(a.y, b.x, im);
            }
            Cb[j] = make_float2(re, im);
            amx = fmaxf(amx, fmaxf(fabsf(re), fabsf(im)));
        }
        if (d.amax_out) amax_publish(d.amax_out + s, amx);
    }
}

// Steps with nothing contracted (outer products, with or without batch labels): C[c] = A[a(c)]
// B[b(c)].  Pure streams of stores, so the per-output work is cut to the bone: a thread keeps
// the operand offsets of its 4 outputs in each 1024-output chunk in registers (the same in every
// chunk), the chunk's high-bit offsets come from a warp-parallel deposit (lane i takes output
// bit 10 + i), and the max-abs is published once per slice a block touches rather than per
// chunk.
__global__ void __launch_bounds__(256) k_generic_k1(GenericDesc d, int64_t total) {
    constexpr int LB = 10, PER = (1 << LB) / 256;
    const int lane = threadIdx.x & 31;
    uint64_t oa[PER], ob[PER];
#pragma unroll
    for (int t = 0; t < PER; ++t) {
        const uint64_t j = (uint64_t)threadIdx.x + 256 * t;
        oa[t] = deposit(j, LB, d.posA_c);
        ob[t] = deposit(j, LB, d.posB_c);
    }
    const uint64_t cmask = (d.rank_c >= 63) ? ~0ull : ((1ull << d.rank_c) - 1);
    const int64_t nchunks = total >> LB;
    int64_t cur_s = -1;
    float amx = 0.f;
    for (int64_t ch = blockIdx.x; ch < nchunks; ch += gridDim.x) {
        const int64_t base = ch << LB;
        const int64_t s = base >> d.rank_c;
        const uint64_t c0 = (uint64_t)base & cmask;
        if (s != cur_s) {
            if (cur_s >= 0 && d.amax_out) amax_publish(d.amax_out + cur_s, amx);
            amx = 0.f;
            cur_s = s;
        }
        uint64_t ha = 0, hb = 0;
        for (int i = LB + lane; i < d.rank_c; i += 32)
            if ((c0 >> i) & 1ull) {
                if (d.posA_c[i] >= 0) ha |= 1ull << d.posA_c[i];
                if (d.posB_c[i] >= 0) hb |= 1ull << d.posB_c[i];
            }
        ha = ((uint64_t)__reduce_or_sync(0xffffffffu, (uint32_t)(ha >> 32)) << 32) |
             __reduce_or_sync(0xffffffffu, (uint32_t)ha);
        hb = ((uint64_t)__reduce_or_sync(0xffffffffu, (uint32_t)(hb >> 32)) << 32) |
             __reduce_or_sync(0xffffffffu, (uint32_t)hb);
        const float2 *Ab = d.A + s * d.sA + ha;
        const float2 *Bb = d.B + s * d.sB + hb;
        float2 *Cb = d.C + s * d.sC + (int64_t)c0;
#pragma unroll
        for (int t = 0; t < PER; ++t) {
            const float2 a = Ab[oa[t]], b = Bb[ob[t]];
            const float re = fmaf(a.x, b.x, -a.y * b.y), im = fmaf(a.x, b.y, a.y * b.x);
            Cb[threadIdx.x + 256 * t] = make_float2(re, im);
            amx = fmaxf(amx, fmaxf(fabsf(re), fabsf(im)));
        }
    }
    if (cur_s >= 0 && d.amax_out) amax_publish(d.amax_out + cur_s, amx);
}

// A run of consecutive small element-wise steps in one launch: block s executes every step of
// the run for slice s in order, one thread per output element as in k_generic, with a block
// barrier between steps (a step's outputs are read by later steps of the same block only).  The
// plan gives all tensors a run touches pairwise disjoint memory, so blocks never race.
__global__ void __launch_bounds__(256) k_generic_chain(const GenericDesc *steps, int32_t nsteps) {
    __shared__ uint64_t koffA[1024], koffB[1024];
    __shared__ uint64_t loA[1024], loB[1024];
    const int64_t s = blockIdx.x;
    for (int i = 0; i < nsteps; ++i) {
        const GenericDesc &d = steps[i];
        const int nk = d.nk, rc = d.rank_c;
        const int lb = rc < 10 ? rc : 10;
        for (int j = threadIdx.x; j < (1 << lb); j += blockDim.x) {
            loA[j] = deposit((uint64_t)j, lb, d.posA_c);
            loB[j] = deposit((uint64_t)j, lb, d.posB_c);
        }
        for (int k = threadIdx.x; k < (1 << nk); k += blockDim.x) {
            koffA[k] = deposit((uint64_t)k, nk, d.posA_k);
            koffB[k] = deposit((uint64_t)k, nk, d.posB_k);
        }
        __syncthreads();
        const int K = 1 << nk;
        for (int64_t ch = 0; ch < (1ll << (rc - lb)); ++ch) {
            const uint64_t c0 = (uint64_t)ch << lb;
            const uint64_t hA = deposit(c0 >> lb, rc - lb, d.posA_c + lb);
            const uint64_t hB = deposit(c0 >> lb, rc - lb, d.posB_c + lb);
            const float2 *Ab = d.A + s * d.sA + hA;
            const float2 *Bb = d.B + s * d.sB + hB;
            float2 *Cb = d.C + s * d.sC + (int64_t)c0;
            for (int j = threadIdx.x; j < (1 << lb); j += blockDim.x) {
                const float2 *A = Ab + loA[j];
                const float2 *B = Bb + loB[j];
                float re = 0.f, im = 0.f;
                for (int k = 0; k < K; ++k) {
                    const float2 a = A[koffA[k]], b = B[koffB[k]];
                    re = fmaf(a.x, b.x, re);
                    re = fmaf(-a.y, b.y, re);
                    im = fmaf(a.x, b.y, im);
                    im = fmaf(a.y, b.x, im);
                }
                Cb[j] = make_float2(re, im);
            }
        }
        __syncthreads();  // outputs visible to the next step; tables free
    }
}

// Sparse-state leaves (Sec. 3.3): grid (leaf, chunk); block (leaf, chunk) writes a strided part
// of that leaf's configurations x dense elements.
__global__ void k_sparse_leaves(const SparseLeafDesc *leaves) {
    const SparseLeafDesc &d = leaves[blockIdx.x];
    const int64_t nd = 1ll << d.rank_d;
    const int64_t total = d.nconf * nd;
    for (int64_t i = blockIdx.y * (int64_t)blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.y * blockDim.x) {
        const int64_t c = i >> d.rank_d;
        const uint64_t j = (uint64_t)(i & (nd - 1));
        const double2 v = d.src[d.cfg_off[c] | (int64_t)deposit(j, d.rank_d, d.pos_d)];
        d.dst[i] = make_float2((float)v.x, (float)v.y);
    }
}

// One sparse-state step: thread per (configuration c, dense output j), summing over the
// contracted dense bits in increasing order; the operand entries are the configurations gA[c],
// gB[c] (the projections of c onto each operand's open labels).
__global__ void __launch_bounds__(256) k_sparse_step(GenericDesc d, const int32_t *gA,
                                                     const int32_t *gB, int64_t nconf) {
    __shared__ uint64_t koffA[1024], koffB[1024];
    const int nk = d.nk;
    const bool table = nk <= 10;
    if (table) {
        for (int k = threadIdx.x; k < (1 << nk); k += blockDim.x) {
            koffA[k] = deposit((uint64_t)k, nk, d.posA_k);
            koffB[k] = deposit((uint64_t)k, nk, d.posB_k);
        }
    }
    __syncthreads();
    const int64_t total = nconf << d.rank_c;
    const int64_t K = 1ll << nk;
    const uint64_t jmask = (1ull << d.rank_c) - 1;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t c = i >> d.rank_c;
        const uint64_t j = (uint64_t)i & jmask;
        const float2 *A = d.A + (int64_t)gA[c] * d.sA + deposit(j, d.rank_c, d.posA_c);
        const float2 *B = d.B + (int64_t)gB[c] * d.sB + deposit(j, d.rank_c, d.posB_c);
        float re = 0.f, im = 0.f;
        for (int64_t k = 0; k < K; ++k) {
            const uint64_t oa = table ? koffA[k] : deposit((uint64_t)k, nk, d.posA_k);
            const uint64_t ob = table ? koffB[k] : deposit((uint64_t)k, nk, d.posB_k);
            const float2 a = A[oa], b = B[ob];
            re = fmaf(a.x, b.x, re);
            re = fmaf(-a.y, b.y, re);
            im = fmaf(a.x, b.y, im);
            im = fmaf(a.y, b.x, im);
        }
        d.C[c * d.sC + (int64_t)j] = make_float2(re, im);
    }
}

__global__ void k_sparse_amps(const float2 *root, const int32_t *idx, int64_t n, double2 *amps) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const float2 v = root[idx[i]];
        amps[i].x += (double)v.x;
        amps[i].y += (double)v.y;
    }
}

// Leaf binding: grid (item, slice, chunk); the blocks of one (item, slice) share its elements.
__global__ void k_bind(const BindItem *items, const double2 *src, float2 *arena,
                       int64_t slice_begin) {
    const BindItem it = items[blockIdx.x];
    const int64_t s = blockIdx.y;
    const uint64_t sigma = (uint64_t)(slice_begin + s);
    uint64_t soff = 0;
    for (int t = 0; t < it.nsl; ++t)
        if ((sigma >> it.sl_bit[t]) & 1ull) soff |= 1ull << it.sl_pos[t];
    const int64_t n = 1ll << it.rank;
    float2 *dst = arena + it.dst_off + s * it.dst_sstride;
    for (int64_t i = blockIdx.z * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.z * blockDim.x) {
        const uint64_t so = deposit((uint64_t)i, it.rank, it.pos_src) | soff;
        const double2 v = src[it.src_off + (int64_t)so];
        dst[i] = make_float2((float)v.x, (float)v.y);
    }
}

// Tiled leaf binding (see BindTiled).  Shared memory holds one tile of up to MAXN complex64
// (2^11, or 2^12 when the six lowest source bits all lie above destination bit 5); the element
// of tile index tau sits at tau ^ (((tau >> 6) & 31) << 1).  The XOR changes bits 1-5 only, so
// the two elements of a destination pair stay adjacent and 16-byte aligned, and when the
// source's low bits land on tile bits 6-10 the 32 lanes of a read still write 32 distinct
// 16-byte slots of one 512-byte row.
__device__ __forceinline__ int tile_slot(int tau) { return tau ^ (((tau >> 6) & 31) << 1); }

template <int MAXN>
__global__ void __launch_bounds__(256) k_bind_tiled(BindTiled b, const double2 *__restrict__ src,
                                                    float2 *__restrict__ arena,
                                                    int64_t slice_begin) {
    __shared__ __align__(16) float2 tile[MAXN];
    const int64_t s = blockIdx.y;
    const uint64_t sigma = (uint64_t)(slice_begin + s);
    uint64_t soff = 0;
    for (int j = 0; j < b.nsl; ++j)
        if ((sigma >> b.sl_bit[j]) & 1ull) soff |= 1ull << b.sl_pos[j];
    const double2 *S = src + b.src_off + soff;
    float2 *D = arena + b.dst_off + s * b.dst_sstride;
    const int n = 1 << b.t;
    const int tid = threadIdx.x;
    // read-order index e = tid + 256 k: its tile index and source offset are those of tid OR'ed
    // with those of 256 k (disjoint bits)
    int tau0 = 0;
    uint64_t so0 = 0;
    for (int q = 0; q < 8 && q < b.t; ++q)
        if ((tid >> q) & 1) {
            tau0 |= 1 << b.e2t[q];
            so0 |= 1ull << b.e2s[q];
        }
    // write-order pair j = tid + 256 k covers tile indices 2 j, 2 j + 1; destination bits of
    // tile bits 6-8 come from tid, those of tile bits 9 and up from k
    uint64_t dw0 = 0;
    for (int q = 6; q < 9 && q < b.t; ++q)
        if (((2 * tid) >> q) & 1) dw0 |= 1ull << b.t2d[q];
    for (int64_t w = blockIdx.x; w < b.ntiles; w += gridDim.x) {
        uint64_t dbase = 0, sbase = 0;
        for (int u = 0; u < b.nrest; ++u)
            if ((w >> u) & 1) {
                dbase |= 1ull << b.rest_d[u];
                sbase |= 1ull << b.rest_s[u];
            }
        for (int k = 0; (k << 8) + tid < n; ++k) {
            int tau = tau0;
            uint64_t so = so0;
            for (int q = 8; q < b.t; ++q)
                if ((k >> (q - 8)) & 1) {
                    tau |= 1 << b.e2t[q];
                    so |= 1ull << b.e2s[q];
                }
            const double2 v = S[sbase | so];
            tile[tile_slot(tau)] = make_float2((float)v.x, (float)v.y);
        }
        __syncthreads();
        for (int k = 0; (k << 8) + tid < (n >> 1); ++k) {
            const int tau = 2 * (tid + (k << 8));
            uint64_t doff = dbase | dw0 | (uint64_t)(tau & 63);
            for (int q = 9; q < b.t; ++q)
                if ((tau >> q) & 1) doff |= 1ull << b.t2d[q];
            *reinterpret_cast<float4 *>(D + doff) =
                *reinterpret_cast<const float4 *>(&tile[tile_slot(tau)]);
        }
        __syncthreads();
    }
}

// amps[x] += sum over slices s (in increasing order) of root[s][x], in FP64.
__global__ void k_accumulate(const float2 *root, int64_t sstride, int64_t n, int64_t slices,
                             double2 *amps) {
    for (int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; x < n;
         x += (int64_t)gridDim.x * blockDim.x) {
        double2 acc = amps[x];
        for (int64_t s = 0; s < slices; ++s) {
            const float2 v = root[s * sstride + x];
            acc.x += (double)v.x;
            acc.y += (double)v.y;
        }
        amps[x] = acc;
    }
}

// The same with sliced open labels (amplitude batches, Sec. 3.2 slicing applied to open
// bonds): slice s0 + s adds its root into the block of amps that its bits for those labels
// select.  A thread owns one root element and walks the slices in increasing order; different
// threads write different amplitudes, and slices of one block are summed in slice order.
__global__ void k_accumulate_batched(const float2 *root, int64_t sstride, int64_t n,
                                     int64_t slices, int64_t s0, const AccMap m,
                                     double2 *amps) {
    for (int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; x < n;
         x += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t xo = deposit((uint64_t)x, m.nroot, m.root_pos);
        for (int64_t s = 0; s < slices; ++s) {
            const uint64_t sig = (uint64_t)(s0 + s);
            uint64_t o = xo;
            for (int i = 0; i < m.nb; ++i)
                if ((sig >> m.bj[i]) & 1ull) o |= 1ull << m.bpos[i];
            const float2 v = root[s * sstride + x];
            double2 a = amps[o];
            a.x += (double)v.x;
            a.y += (double)v.y;
            amps[o] = a;
        }
    }
}

// FP64 readout, pass 1: block partial sums of p = |a|^2 and p^2 (fixed order per block).
__global__ void __launch_bounds__(256) k_readout_partial(const double2 *amps, int64_t n,
                                                         double *partial) {
    __shared__ double s1[256], s2[256];
    double a1 = 0.0, a2 = 0.0;
    for (int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; x < n;
         x += (int64_t)gridDim.x * blockDim.x) {
        const double2 v = amps[x];
        const double p = v.x * v.x + v.y * v.y;
        a1 += p;
        a2 += p * p;
    }
    s1[threadIdx.x] = a1;
    s2[threadIdx.x] = a2;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) {
            s1[threadIdx.x] += s1[threadIdx.x + w];
            s2[threadIdx.x] += s2[threadIdx.x + w];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        partial[2 * blockIdx.x] = s1[0];
        partial[2 * blockIdx.x + 1] = s2[0];
    }
}

// Pass 2: one thread sums the block partials in block order.
__global__ void k_readout_final(double *partial, int32_t n_partial) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double a1 = 0.0, a2 = 0.0;
    for (int i = 0; i < n_partial; ++i) {
        a1 += partial[2 * i];
        a2 += partial[2 * i + 1];
    }
    partial[0] = a1;
    partial[1] = a2;
}

__global__ void k_zero_f64(double2 *p, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        p[i] = make_double2(0.0, 0.0);
}

// max(|re|, |im|) per slice, as float bits (non-negative floats order like unsigned ints).
__global__ void __launch_bounds__(256) k_amax(ConvertDesc d) {
    const int64_t s = blockIdx.y;
    const float4 *src = reinterpret_cast<const float4 *>(d.src + s * d.src_sstride);
    const int64_t n2 = d.n >> 1;  // two complex numbers per float4
    float m = 0.f;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n2;
         i += (int64_t)gridDim.x * blockDim.x) {
        const float4 v = src[i];
        m = fmaxf(m, fmaxf(fmaxf(fabsf(v.x), fabsf(v.y)), fmaxf(fabsf(v.z), fabsf(v.w))));
    }
    if ((d.n & 1) && blockIdx.x == 0 && threadIdx.x == 0) {
        const float2 v = d.src[s * d.src_sstride + d.n - 1];
        m = fmaxf(m, fmaxf(fabsf(v.x), fabsf(v.y)));
    }
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(d.amax + s, __float_as_uint(m));
}

__device__ __forceinline__ int scale_exponent(unsigned int amax_bits) {
    const float a = __uint_as_float(amax_bits);
    if (!(a > 0.f) || !isfinite(a)) return 0;
    return ilogbf(a) - 14;  // stored max lands in [2^14, 2^15): inside FP16's range
}

// complex64 -> planar 16-bit: stored = value * 2^-e (exact power-of-two scaling).  With three
// planes the third holds re + im, summed in FP32 and rounded once; with four, planes 2 and 3 hold
// the residuals re - hi(re) and im - hi(im) (the "lo" halves of a compensated product).
template <typename T2>
__device__ __forceinline__ T2 pack2(float a, float b);
template <>
__device__ __forceinline__ __half2 pack2<__half2>(float a, float b) {
    return __floats2half2_rn(a, b);
}
template <>
__device__ __forceinline__ __nv_bfloat162 pack2<__nv_bfloat162>(float a, float b) {
    return __floats2bfloat162_rn(a, b);
}

// FP32 rounded to the nearest TF32 value (10 fraction bits, ties away from zero), kept in an
// FP32 container: the tensor core then reads it without further rounding.
__device__ __forceinline__ float round_tf32(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}
template <>
__device__ __forceinline__ float2 pack2<float2>(float a, float b) {
    return make_float2(round_tf32(a), round_tf32(b));
}

__device__ __forceinline__ float2 unpack2(__half2 h) { return __half22float2(h); }
__device__ __forceinline__ float2 unpack2(__nv_bfloat162 h) { return __bfloat1622float2(h); }
__device__ __forceinline__ float2 unpack2(float2 h) { return h; }

// T2 is a pair of stored elements (two 16-bit numbers, or two FP32 for TF32); the planes and
// strides of d count elements.
template <typename T2>
__device__ __forceinline__ void convert_body(const ConvertDesc &d, int64_t s, int e) {
    using T = decltype(T2().x);
    const Pow2 pe = pow2_of(-e);
    const float2 *src = d.src + s * d.src_sstride;
    T *base = reinterpret_cast<T *>(d.dst) + s * d.dst_sstride;
    T2 *re = reinterpret_cast<T2 *>(base);
    T2 *im = reinterpret_cast<T2 *>(base + d.plane_stride);
    T2 *sm = reinterpret_cast<T2 *>(base + 2 * d.plane_stride);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < (d.n >> 1);
         i += (int64_t)gridDim.x * blockDim.x) {
        const float4 v = reinterpret_cast<const float4 *>(src)[i];
        const float r0 = scale_pow2(v.x, pe), i0 = scale_pow2(v.y, pe);
        const float r1 = scale_pow2(v.z, pe), i1 = scale_pow2(v.w, pe);
        const T2 rh = pack2<T2>(r0, r1), ih = pack2<T2>(i0, i1);
        re[i] = rh;
        im[i] = ih;
        if (d.planes == 3) sm[i] = pack2<T2>(r0 + i0, r1 + i1);
        if (d.planes == 4) {
            // lo planes: the rounding residuals x - hi (exact in FP32), rounded again
            const float2 rf = unpack2(rh), jf = unpack2(ih);
            sm[i] = pack2<T2>(r0 - rf.x, r1 - rf.y);
            T2 *iml = reinterpret_cast<T2 *>(base + 3 * d.plane_stride);
            iml[i] = pack2<T2>(i0 - jf.x, i1 - jf.y);
        }
    }
}

__global__ void __launch_bounds__(256) k_convert16(ConvertDesc d) {
    const int64_t s = blockIdx.y;
    const int e = scale_exponent(d.amax[s]);
    if (blockIdx.x == 0 && threadIdx.x == 0) d.exps[s] = e;
    if (d.dtype == 2) convert_body<float2>(d, s, e);
    else if (d.dtype == 1) convert_body<__nv_bfloat162>(d, s, e);
    else convert_body<__half2>(d, s, e);
}

int grid_for(int64_t work, int threads) {
    int64_t b = (work + threads - 1) / threads;
    if (b < 1) b = 1;
    if (b > 152 * 64) b = 152 * 64;
    return (int)b;
}

}  // namespace

cudaError_t launch_generic(const GenericDesc &d, int64_t slices, cudaStream_t st) {
    const int64_t total = slices << d.rank_c;
    const int lb = d.rank_c < 10 ? d.rank_c : 10;
    int64_t blocks = total >> lb;
    if (blocks > 152 * 16) blocks = 152 * 16;
    if (d.nk == 0 && d.rank_c >= 10)
        k_generic_k1<<<(unsigned)blocks, 256, 0, st>>>(d, total);
    else
        k_generic<<<(unsigned)blocks, 256, 0, st>>>(d, total);
    return cudaGetLastError();
}

cudaError_t launch_generic_chain(const GenericDesc *steps_dev, int32_t nsteps, int64_t slices,
                                 cudaStream_t st) {
    if (nsteps <= 0 || slices <= 0) return cudaSuccess;
    if (slices > 0x7fffffff) return cudaErrorInvalidValue;
    k_generic_chain<<<(unsigned)slices, 256, 0, st>>>(steps_dev, nsteps);
    return cudaGetLastError();
}

cudaError_t launch_sparse_leaves(const SparseLeafDesc *leaves_dev, int32_t n, int32_t max_rank,
                                 cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    int64_t chunks = ((1ll << (max_rank < 24 ? max_rank : 24)) + 255) / 256;
    if (chunks > 1024) chunks = 1024;
    if (chunks < 1) chunks = 1;
    k_sparse_leaves<<<dim3((unsigned)n, (unsigned)chunks), 256, 0, st>>>(leaves_dev);
    return cudaGetLastError();
}

cudaError_t launch_sparse_step(const GenericDesc &d, const int32_t *gA, const int32_t *gB,
                               int64_t nconf, cudaStream_t st) {
    if (nconf <= 0) return cudaSuccess;
    k_sparse_step<<<grid_for(nconf << d.rank_c, 256), 256, 0, st>>>(d, gA, gB, nconf);
    return cudaGetLastError();
}

cudaError_t launch_sparse_amps(const float2 *root, const int32_t *idx, int64_t n, double2 *amps,
                               cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    k_sparse_amps<<<grid_for(n, 256), 256, 0, st>>>(root, idx, n, amps);
    return cudaGetLastError();
}

cudaError_t launch_bind(const BindItem *items_dev, int32_t n_items, const double2 *src,
                        float2 *arena, int64_t slice_begin, int64_t slices, int32_t max_rank,
                        cudaStream_t st) {
    if (n_items == 0 || slices == 0) return cudaSuccess;
    const int threads = max_rank >= 8 ? 256 : (max_rank >= 6 ? 64 : 32);
    int64_t chunks = ((1ll << max_rank) + threads * 8 - 1) / (threads * 8);
    if (chunks > 1024) chunks = 1024;
    if (chunks < 1) chunks = 1;
    k_bind<<<dim3((unsigned)n_items, (unsigned)slices, (unsigned)chunks), threads, 0, st>>>(
        items_dev, src, arena, slice_begin);
    return cudaGetLastError();
}

cudaError_t launch_bind_tiled(const BindTiled &b, const double2 *src, float2 *arena,
                              int64_t slice_begin, int64_t slices, cudaStream_t st) {
    if (slices <= 0) return cudaSuccess;
    if (b.t < 6 || b.t > 12 || slices > 65535 || b.ntiles < 1) return cudaErrorInvalidValue;
    const int per_sm = b.t <= 11 ? 8 : 6;  // resident blocks (16 or 32 KiB of shared memory)
    int64_t gx = (152 * per_sm + slices - 1) / slices;
    if (gx > b.ntiles) gx = b.ntiles;
    if (b.t <= 11)
        k_bind_tiled<2048><<<dim3((unsigned)gx, (unsigned)slices), 256, 0, st>>>(b, src, arena,
                                                                                 slice_begin);
    else
        k_bind_tiled<4096><<<dim3((unsigned)gx, (unsigned)slices), 256, 0, st>>>(b, src, arena,
                                                                                 slice_begin);
    return cudaGetLastError();
}

cudaError_t launch_accumulate(const float2 *root, int64_t root_sstride, int64_t n, int64_t slices,
                              double2 *amps, cudaStream_t st) {
    k_accumulate<<<grid_for(n, 256), 256, 0, st>>>(root, root_sstride, n, slices, amps);
    return cudaGetLastError();
}

cudaError_t launch_accumulate_batched(const float2 *root, int64_t root_sstride, int64_t n,
                                      int64_t slices, int64_t s0, const AccMap &m,
                                      double2 *amps, cudaStream_t st) {
    k_accumulate_batched<<<grid_for(n, 256), 256, 0, st>>>(root, root_sstride, n, slices, s0, m,
                                                          amps);
    return cudaGetLastError();
}

cudaError_t launch_readout(const double2 *amps, int64_t n, double *partial, int32_t n_partial,
                           cudaStream_t st) {
    k_readout_partial<<<n_partial, 256, 0, st>>>(amps, n, partial);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_readout_final<<<1, 32, 0, st>>>(partial, n_partial);
    return cudaGetLastError();
}

cudaError_t launch_zero_f64(double2 *p, int64_t n, cudaStream_t st) {
    k_zero_f64<<<grid_for(n, 256), 256, 0, st>>>(p, n);
    return cudaGetLastError();
}

cudaError_t launch_amax(const ConvertDesc &d, int64_t slices, cudaStream_t st) {
    const int gx = grid_for((d.n + 1) / 2, 256);
    const int g = gx > 1024 ? 1024 : gx;
    k_amax<<<dim3((unsigned)g, (unsigned)slices), 256, 0, st>>>(d);
    return cudaGetLastError();
}

cudaError_t launch_convert16(const ConvertDesc &d, int64_t slices, cudaStream_t st) {
    const int gx = grid_for(d.n / 2, 256);
    const int g = gx > 2048 ? 2048 : gx;
    k_convert16<<<dim3((unsigned)g, (unsigned)slices), 256, 0, st>>>(d);
    return cudaGetLastError();
}

}  // namespace tn
