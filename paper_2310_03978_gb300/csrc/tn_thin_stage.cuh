// Output stage of the tensor-core thin kernel (k_gemm_thin_tc): a tile of 128 rows and NT columns
// of complex64, thread t of a drain group holding row t, is staged in shared memory and written
// in the order of C's memory index, 8 consecutive elements of C per task.  (The CUDA-core thin kernel keeps a
// padded stage, rows NT + 1 apart: the swizzle's extra address arithmetic and registers cost
// it more than the bank conflicts it removes.)
//
// Element (r, c) of the stage sits at r * NT + (c ^ phi(r)), phi(r) the XOR of d.phi[b] over the
// set bits b of r (host: thin_choose_swizzle), so both the staging writes and the reads in C's
// order spread over the shared-memory banks.  The tile bits sorted by their position in C
// (d.tb_src, row bits tagged 128) split every element index into the part of bits 0-2 (the
// element inside a run of 8) and the part of the bits above (the run); each part is a row part
// R and a column part C of disjoint bits, and since phi is linear the stage index is the sum of
// the parts' R * NT plus the XOR of their C ^ phi(R).  Bits 0-2 contribute per bit (r0-r2,
// x0-x2), the run part per task (qr, qx).
#pragma once

#include "tn_internal.h"

namespace tn {

template <int NT>
struct ThinStage {
    static constexpr int LR = 7, ROWS = 1 << LR;  // rows of a tile (= threads of a group)
    // a tile has ROWS * NT elements: ROWS * NT / 8 runs of 8.  Complex64 results: two lanes
    // share each run (lane half h writes elements 4j + 2h and 4j + 2h + 1 in its store j, so
    // each store fills whole 32-byte sectors); planar 16-bit results (16 bytes per plane and
    // run): a lane writes whole runs, consecutive lanes consecutive runs
    static constexpr int TASKS = ROWS * NT / 8, SUBS = 2 * TASKS;
    static constexpr int SPT = (SUBS + ROWS - 1) / ROWS, SPTP = (TASKS + ROWS - 1) / ROWS;
    int phr;                  // column XOR of this thread's own row
    int r0, r1, r2, x0, x1, x2;  // tile bits 0-2: row part * NT, column part ^ phi(row part)
    int qr[SPT], qx[SPT];     // task q of this thread: the same for its run bits
    uint64_t os[SPT];         // C offset of task q (its element 0)

    __device__ __forceinline__ static int phi_of(const GemmDesc &d, int r) {
        int p = 0;
#pragma unroll
        for (int b = 0; b < 8; ++b)
            if ((r >> b) & 1) p ^= d.phi[b];
        return p;
    }

    __device__ __forceinline__ void init(const GemmDesc &d, int tid) {
        phr = phi_of(d, tid);
        int rr[3], xx[3];
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            const int sq = d.tb_src[q];
            const int R = (sq & 128) ? 1 << (sq & 127) : 0, Cc = (sq & 128) ? 0 : 1 << sq;
            rr[q] = R * NT;
            xx[q] = Cc ^ phi_of(d, R);
        }
        r0 = rr[0], r1 = rr[1], r2 = rr[2];
        x0 = xx[0], x1 = xx[1], x2 = xx[2];
#pragma unroll
        for (int i = 0; i < SPT; ++i) {
            const int u = tid + ROWS * i;
            const int r = d.planar_out ? u : u >> 1, h = d.planar_out ? 0 : u & 1;
            int R = 0, Cc = 0;
            uint64_t o = h ? 2 : 0;
            for (int q = 3; q < d.tile_bits; ++q)
                if ((r >> (q - 3)) & 1) {
                    const int sq = d.tb_src[q];
                    if (sq & 128) R |= 1 << (sq & 127);
                    else Cc |= 1 << sq;
                    o |= 1ull << d.tb_pos[q];
                }
            qr[i] = R * NT + (h ? r1 : 0);
            qx[i] = (Cc ^ phi_of(d, R)) ^ (h ? x1 : 0);
            os[i] = o;
        }
    }
    // this thread's row into the stage
    __device__ __forceinline__ void put(float2 *stage, int tid, const float *cr,
                                        const float *ci) const {
#pragma unroll
        for (int n = 0; n < NT; ++n) stage[tid * NT + (n ^ phr)] = make_float2(cr[n], ci[n]);
    }
    // element j of this thread's task i (j a compile-time constant after unrolling)
    __device__ __forceinline__ float2 at(const float2 *stage, int i, int j) const {
        const int R = qr[i] + ((j & 1) ? r0 : 0) + ((j & 2) ? r1 : 0) + ((j & 4) ? r2 : 0);
        const int X = qx[i] ^ ((j & 1) ? x0 : 0) ^ ((j & 2) ? x1 : 0) ^ ((j & 4) ? x2 : 0);
        return stage[R + X];
    }
};

}  // namespace tn
