// Device store of the direct planar 16-bit output (PlanarOut, declared in tn_internal.h).
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "tn_internal.h"

namespace tn {

__device__ __forceinline__ void planar_out_store(const PlanarOut &o, int64_t s, uint64_t off,
                                                 float re, float im, int e) {
    const Pow2 pe = pow2_of(-e);
    const float r = scale_pow2(re, pe), i = scale_pow2(im, pe);
    const int64_t base = s * o.sstride + (int64_t)off;
    if (o.bf16) {
        __nv_bfloat16 *p = static_cast<__nv_bfloat16 *>(o.base) + base;
        const __nv_bfloat16 rh = __float2bfloat16_rn(r), ih = __float2bfloat16_rn(i);
        p[0] = rh;
        p[o.plane_stride] = ih;
        if (o.planes == 3) p[2 * o.plane_stride] = __float2bfloat16_rn(r + i);
        if (o.planes == 4) {
            p[2 * o.plane_stride] = __float2bfloat16_rn(r - __bfloat162float(rh));
            p[3 * o.plane_stride] = __float2bfloat16_rn(i - __bfloat162float(ih));
        }
    } else {
        __half *p = static_cast<__half *>(o.base) + base;
        const __half rh = __float2half_rn(r), ih = __float2half_rn(i);
        p[0] = rh;
        p[o.plane_stride] = ih;
        if (o.planes == 3) p[2 * o.plane_stride] = __float2half_rn(r + i);
        if (o.planes == 4) {
            p[2 * o.plane_stride] = __float2half_rn(r - __half2float(rh));
            p[3 * o.plane_stride] = __float2half_rn(i - __half2float(ih));
        }
    }
}

// Store two adjacent complex values (offsets off and off + 1, off even) into the planar output
// as one 2 x 16-bit word per plane.
__device__ __forceinline__ void planar_out_store2(const PlanarOut &o, int64_t s, uint64_t off,
                                                  float2 v0, float2 v1, int e) {
    const Pow2 pe = pow2_of(-e);
    const float r0 = scale_pow2(v0.x, pe), i0 = scale_pow2(v0.y, pe);
    const float r1 = scale_pow2(v1.x, pe), i1 = scale_pow2(v1.y, pe);
    const int64_t base = s * o.sstride + (int64_t)off;
    const int64_t ps = o.plane_stride / 2;
    if (o.bf16) {
        __nv_bfloat162 *p =
            reinterpret_cast<__nv_bfloat162 *>(static_cast<__nv_bfloat16 *>(o.base) + base);
        const __nv_bfloat162 rh = __floats2bfloat162_rn(r0, r1), ih = __floats2bfloat162_rn(i0, i1);
        p[0] = rh;
        p[ps] = ih;
        if (o.planes == 3) p[2 * ps] = __floats2bfloat162_rn(r0 + i0, r1 + i1);
        if (o.planes == 4) {
            const float2 rf = __bfloat1622float2(rh), jf = __bfloat1622float2(ih);
            p[2 * ps] = __floats2bfloat162_rn(r0 - rf.x, r1 - rf.y);
            p[3 * ps] = __floats2bfloat162_rn(i0 - jf.x, i1 - jf.y);
        }
    } else {
        __half2 *p = reinterpret_cast<__half2 *>(static_cast<__half *>(o.base) + base);
        const __half2 rh = __floats2half2_rn(r0, r1), ih = __floats2half2_rn(i0, i1);
        p[0] = rh;
        p[ps] = ih;
        if (o.planes == 3) p[2 * ps] = __floats2half2_rn(r0 + i0, r1 + i1);
        if (o.planes == 4) {
            const float2 rf = __half22float2(rh), jf = __half22float2(ih);
            p[2 * ps] = __floats2half2_rn(r0 - rf.x, r1 - rf.y);
            p[3 * ps] = __floats2half2_rn(i0 - jf.x, i1 - jf.y);
        }
    }
}

// Store eight consecutive complex values (offsets off .. off + 7, off a multiple of 8) into the
// planar output as one 16-byte word (8 x 16 bits) per plane.
template <typename T2>
__device__ __forceinline__ T2 pack_pair(float a, float b);
template <>
__device__ __forceinline__ __half2 pack_pair<__half2>(float a, float b) {
    return __floats2half2_rn(a, b);
}
template <>
__device__ __forceinline__ __nv_bfloat162 pack_pair<__nv_bfloat162>(float a, float b) {
    return __floats2bfloat162_rn(a, b);
}
__device__ __forceinline__ float2 unpack_pair(__half2 h) { return __half22float2(h); }
__device__ __forceinline__ float2 unpack_pair(__nv_bfloat162 h) { return __bfloat1622float2(h); }

template <typename T2, bool SCALE>
__device__ __forceinline__ void planar_out_store8_t(const PlanarOut &o, int64_t s, uint64_t off,
                                                    const float2 (&v)[8], int e) {
    union Row {
        uint4 u;
        T2 h[4];
    } re, im, p2, p3;
    const Pow2 pe = pow2_of(-e);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const float r0 = SCALE ? scale_pow2(v[2 * j].x, pe) : v[2 * j].x;
        const float i0 = SCALE ? scale_pow2(v[2 * j].y, pe) : v[2 * j].y;
        const float r1 = SCALE ? scale_pow2(v[2 * j + 1].x, pe) : v[2 * j + 1].x;
        const float i1 = SCALE ? scale_pow2(v[2 * j + 1].y, pe) : v[2 * j + 1].y;
        re.h[j] = pack_pair<T2>(r0, r1);
        im.h[j] = pack_pair<T2>(i0, i1);
        if (o.planes == 3) p2.h[j] = pack_pair<T2>(r0 + i0, r1 + i1);
        if (o.planes == 4) {
            const float2 rf = unpack_pair(re.h[j]), jf = unpack_pair(im.h[j]);
            p2.h[j] = pack_pair<T2>(r0 - rf.x, r1 - rf.y);
            p3.h[j] = pack_pair<T2>(i0 - jf.x, i1 - jf.y);
        }
    }
    uint16_t *base = static_cast<uint16_t *>(o.base) + s * o.sstride + (int64_t)off;
    *reinterpret_cast<uint4 *>(base) = re.u;
    *reinterpret_cast<uint4 *>(base + o.plane_stride) = im.u;
    if (o.planes >= 3) *reinterpret_cast<uint4 *>(base + 2 * o.plane_stride) = p2.u;
    if (o.planes == 4) *reinterpret_cast<uint4 *>(base + 3 * o.plane_stride) = p3.u;
}

// Store four consecutive complex values (offsets off .. off + 3, off a multiple of 4) into the
// planar output as one 8-byte word (4 x 16 bits) per plane.
template <typename T2>
__device__ __forceinline__ void planar_out_store4_t(const PlanarOut &o, int64_t s, uint64_t off,
                                                    const float2 (&v)[4], int e) {
    union Half {
        uint2 u;
        T2 h[2];
    } re, im, p2, p3;
    const Pow2 pe = pow2_of(-e);
#pragma unroll
    for (int j = 0; j < 2; ++j) {
        const float r0 = scale_pow2(v[2 * j].x, pe), i0 = scale_pow2(v[2 * j].y, pe);
        const float r1 = scale_pow2(v[2 * j + 1].x, pe), i1 = scale_pow2(v[2 * j + 1].y, pe);
        re.h[j] = pack_pair<T2>(r0, r1);
        im.h[j] = pack_pair<T2>(i0, i1);
        if (o.planes == 3) p2.h[j] = pack_pair<T2>(r0 + i0, r1 + i1);
        if (o.planes == 4) {
            const float2 rf = unpack_pair(re.h[j]), jf = unpack_pair(im.h[j]);
            p2.h[j] = pack_pair<T2>(r0 - rf.x, r1 - rf.y);
            p3.h[j] = pack_pair<T2>(i0 - jf.x, i1 - jf.y);
        }
    }
    uint16_t *base = static_cast<uint16_t *>(o.base) + s * o.sstride + (int64_t)off;
    *reinterpret_cast<uint2 *>(base) = re.u;
    *reinterpret_cast<uint2 *>(base + o.plane_stride) = im.u;
    if (o.planes >= 3) *reinterpret_cast<uint2 *>(base + 2 * o.plane_stride) = p2.u;
    if (o.planes == 4) *reinterpret_cast<uint2 *>(base + 3 * o.plane_stride) = p3.u;
}

__device__ __forceinline__ void planar_out_store4(const PlanarOut &o, int64_t s, uint64_t off,
                                                  const float2 (&v)[4], int e) {
    if (o.bf16) planar_out_store4_t<__nv_bfloat162>(o, s, off, v, e);
    else planar_out_store4_t<__half2>(o, s, off, v, e);
}

__device__ __forceinline__ void planar_out_store8(const PlanarOut &o, int64_t s, uint64_t off,
                                                  const float2 (&v)[8], int e) {
    if (o.bf16) planar_out_store8_t<__nv_bfloat162, true>(o, s, off, v, e);
    else planar_out_store8_t<__half2, true>(o, s, off, v, e);
}

// The same for values already multiplied by 2^-e.
__device__ __forceinline__ void planar_out_store8_prescaled(const PlanarOut &o, int64_t s,
                                                            uint64_t off, const float2 (&v)[8]) {
    if (o.bf16) planar_out_store8_t<__nv_bfloat162, false>(o, s, off, v, 0);
    else planar_out_store8_t<__half2, false>(o, s, off, v, 0);
}

}  // namespace tn
