// Device store of the direct planar 16-bit output (PlanarOut, declared in tn_internal.h).
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "tn_internal.h"

namespace tn {

__device__ __forceinline__ void planar_out_store(const PlanarOut &o, int64_t s, uint64_t off,
                                                 float re, float im, int e) {
    const float r = ldexpf(re, -e), i = ldexpf(im, -e);
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
    const float r0 = ldexpf(v0.x, -e), i0 = ldexpf(v0.y, -e);
    const float r1 = ldexpf(v1.x, -e), i1 = ldexpf(v1.y, -e);
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

}  // namespace tn
