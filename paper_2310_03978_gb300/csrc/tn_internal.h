// Internal declarations shared by the host runtime and the CUDA kernels of libtn.so.
//
// Every tensor is a "bit tensor": each label has dimension 2, so an element index is a word of
// bits and a label is a bit position.  Bit 0 of a tensor's memory index is its last label.
// A step C = sum_K A * B (Sec. 2.4, Eq. chap2_einsum) is described by where each bit of the
// output index and of the contracted index lands in the operands' memory indices.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#define TN_MAXR 48  // largest rank handled by a kernel descriptor

#include "../../include/tn.h"

namespace tn {

// Record `msg` as this thread's error detail (tn_last_error_detail) and return `s`.
tn_status report(tn_status s, const char *msg);
// The same with a printf format.
tn_status reportf(tn_status s, const char *fmt, ...);
// Clear this thread's error detail (every entry point does so on entry).
void clear_error();

constexpr uint32_t kNetMagic = 0x544e4e54u;     // "TNNT": a tn_network
constexpr uint32_t kSparseMagic = 0x544e5350u;  // "TNSP": a sparse-state plan
// Free a sparse-state plan (tn_destroy of a handle with kSparseMagic).
void sparse_destroy(void *handle);

// Direct planar 16-bit output of a GEMM whose result feeds a tensor-core step: the producer
// writes stored = value * 2^-e into the consumer's planar buffer (re, im, and for the 3M form
// re + im planes), with e chosen before the GEMM runs from the bound
//     max(|Re c|, |Im c|) <= 2 K max|a| max|b|,   max|x| = max over x of max(|Re x|, |Im x|),
// evaluated from the inputs' measured per-slice max-abs, so that |stored| < 2^15 (inside FP16's
// range) and no overflow is possible.  The exponent of slice s is written to exps[s].
struct PlanarOut {
    void *base;                     // plane p, slice s: base + p * plane_stride + s * sstride
    int64_t plane_stride;           // elements
    int64_t sstride;                // elements
    int32_t planes;                 // 2; 3 with the re + im plane; 4 with re_lo, im_lo planes
    int32_t bf16;
    int32_t *exps;                  // per slice exponent (written by the producer)
    const unsigned int *amax_a;     // inputs' per-slice max-abs, float bits, true scale
    const unsigned int *amax_b;
    int32_t a_sliced, b_sliced;     // 0: the input is shared by all slices (index 0)
    int32_t log2_k;
};

#ifdef __CUDACC__
// Exponent e of the direct planar output of slice s (see PlanarOut).
__device__ __forceinline__ int planar_out_exponent(const PlanarOut &o, int64_t s) {
    const float a = __uint_as_float(o.amax_a[o.a_sliced ? s : 0]);
    const float b = __uint_as_float(o.amax_b[o.b_sliced ? s : 0]);
    if (!(a > 0.f) || !(b > 0.f) || !isfinite(a) || !isfinite(b)) return 0;
    int ea, eb;
    frexpf(a, &ea);  // a < 2^ea
    frexpf(b, &eb);
    return ea + eb + 1 + o.log2_k - 15;  // 2 K a b < 2^(e + 15)
}
#endif

// Element-wise contraction: one thread per output element (any memory orders).
struct GenericDesc {
    const float2 *A;
    const float2 *B;
    float2 *C;
    int64_t sA, sB, sC;        // slice strides in elements (0 = shared by all slices)
    int32_t rank_c;            // output bits
    int32_t nk;                // contracted bits
    unsigned int *amax_out;    // optional: per slice max(|re|, |im|) of C (float bits, atomicMax)
    int8_t posA_c[TN_MAXR];    // output bit i -> bit of A's index (-1: label not in A)
    int8_t posB_c[TN_MAXR];
    int8_t posA_k[TN_MAXR];    // contracted bit j -> bit of A's index
    int8_t posB_k[TN_MAXR];
};

// Limits of a step run by k_generic_chain: output bits, contracted bits, and their sum.
constexpr int kChainMaxRankC = 12;
constexpr int kChainMaxNk = 10;
constexpr int kChainMaxWork = 14;

// Complex GEMM C[m, n] = sum_k A[m, k] * B[n, k] with A = [M][K] and B = [N][K] row-major per
// slice and C written at pdep(m -> posC_m) | pdep(n -> posC_n), i.e. in the consumer's order.
struct GemmDesc {
    const float2 *A;
    const float2 *B;
    float2 *C;
    int64_t sA, sB, sC;
    int32_t lm, ln, lk;        // log2 of M, N, K
    int32_t splits;            // > 1: split-K; CTA z sums K range z and writes partial[z][s]
    float2 *partial;           // split-K partial tiles, [splits][slices][M][N] row-major
    int32_t tile_bits;         // valid bits of a 64 x 64 tile (min(lm,6) + min(ln,6))
    unsigned int *amax_out;    // optional: per slice max(|re|, |im|) of C (float bits, atomicMax)
    int32_t planar_out;        // 1: write C as PlanarOut `pout` instead of complex64
    PlanarOut pout;
    int8_t tb_src[16];         // tile bits sorted by position in C: bit of the staging index
    int8_t tb_pos[16];         //   (n: 0..5, m: 6..11) and its position in C
    int8_t posC_m[TN_MAXR];    // bit i of m (0 = least significant) -> bit of C's index
    int8_t posC_n[TN_MAXR];
    int8_t phi[8];             // tensor-core thin kernel: XOR swizzle of the output stage by
                               //   row bit (thin_choose_swizzle)
};

// Slice binding and conversion of a leaf (Sec. 3.2): dst[s][i] (complex64, plan order) =
// src[sum_j bit_j(i) << posS[j] + sum_t bit_t(slice) << posSl[t]] (complex128, network order).
struct BindItem {
    int64_t dst_off;           // element offset of the destination (complex64) in the arena
    int64_t dst_sstride;       // slice stride of the destination (0 = invariant leaf)
    int64_t src_off;           // complex128 element offset in the network buffer
    int32_t rank;              // bits of the bound (destination) tensor
    int32_t nsl;               // sliced labels of this leaf
    int8_t pos_src[TN_MAXR];   // destination bit i -> source bit
    int8_t sl_bit[8];          // which bit of the slice id fixes sliced label t
    int8_t sl_pos[8];          // source bit of sliced label t
};

// Tiled slice binding of one large leaf (a stride-aware bit permutation, Sec. 2.4's
// permutation done once per leaf, with slicing, Sec. 3.2): the destination is cut into tiles of
// 2^t elements that hold destination bits 0-5 (contiguous in the destination) and the
// destination bits of the leaf's six lowest unsliced source bits (contiguous in the source).
// A block reads a tile in source order (a warp reads 32 consecutive complex128, 512 bytes,
// 16 bytes per lane), stages it in shared memory and writes it in destination order (16 bytes
// of two adjacent complex64 per lane).  The remaining destination bits number the tiles.
struct BindTiled {
    int64_t dst_off;            // element offset of the destination (complex64) in the arena
    int64_t dst_sstride;        // slice stride of the destination (0 = invariant leaf)
    int64_t src_off;            // complex128 element offset in the network buffer
    int64_t ntiles;             // 2^(rank - t)
    int32_t t;                  // tile bits (11..12, fewer only for ranks below 11)
    int32_t nrest;              // rank - t
    int32_t nsl;                // sliced labels of this leaf
    int32_t pad_;
    int8_t e2t[12];             // read-order bit q -> tile bit
    int8_t e2s[12];             // read-order bit q -> source bit
    int8_t t2d[12];             // tile bit -> destination bit (bits 0-5 map to themselves)
    int8_t rest_d[TN_MAXR];     // tile-number bit u -> destination bit
    int8_t rest_s[TN_MAXR];     // tile-number bit u -> source bit
    int8_t sl_bit[8];           // which bit of the slice id fixes sliced label j
    int8_t sl_pos[8];           // source bit of sliced label j
};

// Sort the bits of an output tile (tm row bits, tn column bits) by their position in C:
// src[q] = row_tag | i for row bit i, or j for column bit j; pos[q] = position in C.
// Output stage of the tensor-core thin kernel (128 rows x NT = 2^lnt columns of complex64): element
// (r, c) sits at r * NT + (c ^ phi(r)), phi(r) the XOR of phi[b] over the set bits b of r
// (each below NT).  Chosen so that the staging writes (a half-warp: 16 consecutive rows, one
// column) and the reads in C's order (tile bits sorted by position in C, tb_src as
// sort_tile_bits writes them with row tag 128; a half-warp spans tile bits 1, 3, 4, 5 for
// complex64 results, 3-6 for planar ones) each touch 16 distinct 8-byte bank pairs where the
// layout allows; returns how many of the two patterns are conflict-free.
int thin_choose_swizzle(const int8_t *tb_src, int lnt, bool planar, int8_t *phi);
void sort_tile_bits(int tm, int tn, const int8_t *posC_m, const int8_t *posC_n, int row_tag,
                    int8_t *src, int8_t *pos);


// Power-of-two scaling without a branch: x * 2^e as x * f1 * f2 with f1 = 2^clamp(e, -126, 127)
// and f2 = 2^(e - that) (clamped to the representable range).  For -126 <= e <= 127, f2 = 1 and
// the result is x * 2^e rounded once, exactly like ldexpf; beyond, it can round twice, but only
// for results below FP32's normal range.  The scaling's exponents stay far inside that range.
struct Pow2 {
    float f1, f2;
};
__device__ __forceinline__ float pow2_bits(int e) {  // 2^e for -149 <= e <= 127
    return e >= -126 ? __int_as_float((e + 127) << 23) : __int_as_float(1 << (e + 149));
}
__device__ __forceinline__ Pow2 pow2_of(int e) {
    const int e1 = max(-126, min(e, 127));
    const int e2 = max(-149, min(e - e1, 127));
    return Pow2{pow2_bits(e1), pow2_bits(e2)};
}
__device__ __forceinline__ float scale_pow2(float x, const Pow2 &p) { return x * p.f1 * p.f2; }

// Warp-reduced atomicMax of a non-negative float into *slot (float bits order like unsigned).
__device__ __forceinline__ void amax_publish(unsigned int *slot, float m) {
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(slot, __float_as_uint(m));
}

// Kernel launchers (stream-ordered; return the launch error).
cudaError_t launch_generic(const GenericDesc &d, int64_t slices, cudaStream_t st);
// Sparse-state contraction (Sec. 3.3).  A leaf's sparse form: for each sampled configuration c
// of its open labels, the complex64 array over its other (dense) labels, dst[c * 2^rank_d + j] =
// src[cfg_off[c] | deposit(j -> pos_d)].
struct SparseLeafDesc {
    const double2 *src;        // the leaf's complex128 data (row-major over all its labels)
    float2 *dst;
    const int64_t *cfg_off;    // per configuration: the element offset its open-label values select
    int64_t nconf;
    int32_t rank_d;            // dense labels
    int8_t pos_d[TN_MAXR];     // dense bit i (0 = least significant) -> bit of the leaf's index
};
// all leaves in one launch (descriptors in device memory)
cudaError_t launch_sparse_leaves(const SparseLeafDesc *leaves_dev, int32_t n, int32_t max_rank,
                                 cudaStream_t st);
// one step: for each configuration c of the result, C[c] = einsum(A[gA[c]], B[gB[c]]) over the
// dense labels described by d (d.sA, d.sB, d.sC = per-configuration strides)
cudaError_t launch_sparse_step(const GenericDesc &d, const int32_t *gA, const int32_t *gB,
                               int64_t nconf, cudaStream_t st);
// the same step as a 64 x 64-tiled GEMM per configuration: C's dense index is (A-only labels,
// then the ln B-only labels), row-major; for steps with enough m, n and k
cudaError_t launch_sparse_gemm(const GenericDesc &d, int32_t ln, const int32_t *gA,
                               const int32_t *gB, int64_t nconf, cudaStream_t st);
// Grouped form of a sparse-state step (the gather-indexed grouped GEMM): the result
// configurations are grouped by the configuration of one operand (by_a: A's), so each group is
// one GEMM whose other operand is the stack of its members' entries (columns (member, n) when
// grouped by A, rows (member, m) when grouped by B).  Tiles of 64 x 64 are listed on the host.
struct SparseGroupDesc {
    const int32_t *gA, *gB;    // per result configuration: operand configurations
    const int32_t *members;    // result configurations, group by group
    const int32_t *grp_off;    // per group: first member
    const int32_t *grp_len;    // per group: members
    const int32_t *tiles;      // per tile: group, row tile, column tile
    int64_t ntiles;
    int32_t by_a;
};
cudaError_t launch_sparse_group(const GenericDesc &d, int32_t ln, const SparseGroupDesc &g,
                                cudaStream_t st);
// the same step for at most 16 columns (ln <= 4): thread per (configuration, row)
cudaError_t launch_sparse_thin(const GenericDesc &d, int32_t ln, const int32_t *gA,
                               const int32_t *gB, int64_t nconf, cudaStream_t st);
// amps[i] += root[idx[i]] for the n samples (complex128 accumulation)
cudaError_t launch_sparse_amps(const float2 *root, const int32_t *idx, int64_t n, double2 *amps,
                               cudaStream_t st);
// nsteps descriptors in device memory, one block per slice (see k_generic_chain)
cudaError_t launch_generic_chain(const GenericDesc *steps_dev, int32_t nsteps, int64_t slices,
                                 cudaStream_t st);
// Set the CUDA-core kernels' shared-memory limits (once per device, outside any stream capture).
cudaError_t simt_prepare();
cudaError_t launch_gemm_simt(const GemmDesc &d, int64_t slices, cudaStream_t st);
int gemm_simt_splits(int lm, int ln, int lk, int64_t slices);
// Thin steps on the CUDA cores: A is the operand with 2^lm >= 256 rows, B has 2^ln <= 16 rows,
// 2 <= K <= 64; tile_bits = 8 + ln with tb_src / tb_pos sorted as for the tensor-core epilogue
// (row bits tagged 128 | bit); complex64 output only.
cudaError_t launch_gemm_thin(const GemmDesc &d, int64_t slices, cudaStream_t st);
cudaError_t launch_bind(const BindItem *items_dev, int32_t n_items, const double2 *src,
                        float2 *arena, int64_t slice_begin, int64_t slices, int32_t max_rank,
                        cudaStream_t st);
cudaError_t launch_bind_tiled(const BindTiled &b, const double2 *src, float2 *arena,
                              int64_t slice_begin, int64_t slices, cudaStream_t st);
cudaError_t launch_accumulate(const float2 *root, int64_t root_sstride, int64_t n, int64_t slices,
                              double2 *amps, cudaStream_t st);
// Where the root's elements go when open labels are sliced (amplitude batches): root bit r is
// amplitude-index bit root_pos[r]; bit bj[i] of the slice id is amplitude-index bit bpos[i].
struct AccMap {
    int32_t nroot = 0, nb = 0;
    int8_t root_pos[TN_MAXR];
    int8_t bj[TN_MAXR];
    int8_t bpos[TN_MAXR];
};
// amps[root element mapped by m, slice s0 + s] += root[s][x], slices in increasing order
cudaError_t launch_accumulate_batched(const float2 *root, int64_t root_sstride, int64_t n,
                                      int64_t slices, int64_t s0, const AccMap &m,
                                      double2 *amps, cudaStream_t st);
cudaError_t launch_readout(const double2 *amps, int64_t n, double *partial, int32_t n_partial,
                           cudaStream_t st);
cudaError_t launch_zero_f64(double2 *p, int64_t n, cudaStream_t st);

// Tensor-core path: planar 16-bit operands with one power-of-two exponent per slice.
struct ConvertDesc {
    const float2 *src;         // complex64 source, [slices][n]
    void *dst;                 // planar: re plane [slices][n] then im plane at +plane_stride
    int64_t n;                 // elements per slice
    int64_t src_sstride;
    int64_t plane_stride;      // elements between the re and the im plane
    int64_t dst_sstride;       // elements between slices inside one plane
    unsigned int *amax;        // per slice, float bits of max(|re|, |im|)
    int32_t *exps;             // per slice exponent e: stored = value * 2^-e
    int32_t dtype;             // 0 = fp16, 1 = bf16, 2 = FP32 rounded to TF32
    int32_t planes;            // 2: re, im; 3: re, im, re + im (3M); 4: re, im, re_lo, im_lo
};
cudaError_t launch_amax(const ConvertDesc &d, int64_t slices, cudaStream_t st);
cudaError_t launch_convert16(const ConvertDesc &d, int64_t slices, cudaStream_t st);

struct TcGemmDesc {
    CUtensorMap tmA;           // planar A: [planes * slices_a][M][K]: re, im (, re+im | lo)
    CUtensorMap tmB;           // planar B: [planes * slices_b][N][K]
    float2 *C;
    int64_t sC;
    int32_t lm, ln, lk;
    int32_t a_sliced, b_sliced;  // 0: operand shared by all slices
    int64_t slices_a, slices_b;  // slices stored per plane (1 when shared)
    const int32_t *expA;       // per slice exponents of A and B (index 0 if shared)
    const int32_t *expB;
    int32_t form;              // 1 = 4M, 2 = 3M, 3 = split 4M
    int32_t dtype;             // operands: 0 = fp16, 1 = bf16 (kind::f16), 2 = TF32 (kind::tf32)
    int32_t bk;                // K elements per stage (rows of 64 or 128 bytes)
    int32_t variant;           // kernel variant (tile shape, stages, CTAs per SM)
    unsigned int *amax_out;    // optional: per slice max(|re|, |im|) of C (float bits, atomicMax)
    int32_t planar_out;        // 1: write C as PlanarOut `pout` instead of complex64
    PlanarOut pout;
    uint64_t wait_limit_ns;    // bound of every mbarrier wait (0 = 4 s)
    int32_t selftest_no_loads; // self-test of the bounded waits: the producer issues no loads
    int8_t tb_src[16];         // the 13 bits of a 128 x 64 epilogue chunk sorted by position in
    int8_t tb_pos[16];         //   C: (is_row << 7) | bit index, and its position in C
    int8_t posC_m[TN_MAXR];
    int8_t posC_n[TN_MAXR];
    int8_t phi[8];             // persistent short-K epilogue: XOR swizzle of the staging column
                               //   by row bit i (a bit mask below 16; see tc_choose_swizzle)
    int8_t phi5[8];            //   the same for 4-byte staged elements (masks below 32)
};
bool tc_available();
// Set the kernels' shared-memory limits (once per device, outside any stream capture).
cudaError_t tc_prepare();
cudaError_t launch_gemm_tc(const TcGemmDesc &d, int64_t slices, cudaStream_t st);
// Device status word of the tensor-core kernel (bit 0: a bounded wait timed out); cleared.
unsigned int tc_status_read_and_clear();
// Self-test of the bounded waits (see tn_selftest_wait_timeout in tn.h).
tn_status tc_selftest_wait_timeout(int32_t limit_ms, cudaStream_t st);
// Encode a 3-D tensor map over planar data [planes*slices][rows][K] (K contiguous; dtype 0
// fp16, 1 bf16, 2 fp32), box {bk, box_rows, 1}; the swizzle follows the row width bk * element
// size: 128-, 64- or 32-byte swizzle for rows of 128, 64 or 32 bytes, none for 16 bytes.
int encode_tmap_planar(void *tmap_host, const void *base, int64_t K, int64_t rows,
                       int64_t depth, int dtype, int bk, int box_rows);
// Tensor-core kernel variants: pick one for a step (form 1 = 4M, 2 = 3M, 3 = split; preferences
// 0 = any), and read its K tile (elements per stage), N tile and operand type.
int tc_pick_variant(int form, int lk, int ln, int bk_pref, int bn_pref, bool tf32);
bool tc_variant_tf32(int variant);
int tc_variant_bk(int variant);
int tc_variant_bn(int variant);
int tc_variant_form(int variant);  // 1 = 4M, 2 = 3M, 3 = split 4M (hi/lo planes)
int tc_num_variants();
bool tc_variant_fits(int variant, int lk, int ln);
bool tc_variant_is_pers(int variant);  // the persistent short-K kernel (one CTA per SM)
// Staging swizzle of the persistent kernel's 128 x 32 chunk: element (row r, column c) sits at
// r * 32 + (c ^ phi(r)), phi linear in the row bits (phi[i] for row bit i).  Chosen so that the
// drain warps' writes (lanes = row bits 0..4) and the store warps' reads (lanes = the chunk's
// sorted bits 3..7) each spread over all banks: 16 eight-byte bank pairs (bits = 4, complex64
// staging) or 32 four-byte banks (bits = 5, packed 16-bit re / im).
void tc_choose_swizzle(const int8_t *tb_src, int8_t *phi, int bits);

// Thin step on the tensor cores (k_gemm_thin_tc): the streaming step of GemmDesc g (A the large
// complex64 operand [slices][2^lm][2^lk], B the small one [slices][2^ln][2^lk], tiles of 128
// rows and 2^ln columns: tile_bits = 7 + ln, tb_src / tb_pos from sort_tile_bits(7, ...)) as
// one real TF32 product with compensated (hi / lo) operands.  tmA: A as [depth][2^lm rows][2^(lk+1) floats] with boxes of
// 128 rows (encode_tmap_thin; depth = slices when A depends on the slice, else 1).
struct ThinTcDesc {
    CUtensorMap tmA;
    GemmDesc g;
    uint64_t wait_limit_ns;    // bound of every mbarrier wait (0 = 4 s)
};
bool thin_tc_fits(int lm, int ln, int lk);  // 2^8 <= M <= 2^30 rows, 4-16 columns, 4-16 terms
int encode_tmap_thin(void *tmap_host, const void *A, int lm, int lk, int64_t depth);
cudaError_t launch_gemm_thin_tc(const ThinTcDesc &d, int64_t slices, cudaStream_t st);

}  // namespace tn

// A loaded network (tn_network_load): labels and offsets on the host, the complex128 data on the
// device.  Shared by the dense planner and the sparse-state planner.
struct tn_network {
    uint32_t magic = tn::kNetMagic;
    int device = 0;
    std::vector<std::vector<int>> labels;  // per tensor, row-major order
    std::vector<int64_t> offset;           // complex128 element offset of each tensor
    std::vector<int> open;
    int64_t total = 0;                     // complex128 elements
    double2 *data = nullptr;               // device copy
};
