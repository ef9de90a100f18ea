// FP64 readout of an amplitude vector that allocates no device memory (tn_readout_noalloc).
//
// Some callers cannot let a library call cudaMalloc: a process whose device memory is held by
// another allocator (PyTorch's caching allocator keeps freed blocks reserved, so a cudaMalloc
// from this library can fail even though the caller has memory cached), or one that runs under a
// fixed device-memory budget in which every allocation must come from its own pool.  This entry
// point serves them: it needs no plan, and its scratch (the per-block partial sums) lives in a
// file-scope device array of fixed size instead of an allocation.
//
// The array is 2 * kMaxBlocks doubles (64 KiB) and exists on every GPU that loads libtn.so until
// the process exits.  Each block sums a fixed chunk of kChunk amplitudes, so a call handles at
// most kMaxBlocks * kChunk = 2^28 amplitudes and rejects larger vectors.  Host code cannot use
// the array's name as a device address: the first call on a device looks the address up with
// cudaGetSymbolAddress (with that device current) and caches it per device.  All calls share the
// array and it keeps the last call's partial sums; every call overwrites each slot it reads
// before reading it, so nothing needs clearing, but calls whose kernels overlap on the GPU (for
// instance on two streams) race on the array.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>

#include "../../include/tn.h"
#include "tn_internal.h"

namespace {

constexpr int kChunk = 65536;                               // amplitudes per block
constexpr int kMaxBlocks = 4096;                            // partial-sum slots
constexpr int64_t kMaxAmps = (int64_t)kChunk * kMaxBlocks;  // 2^28
constexpr int kThreads = 256;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) double g_noalloc_scratch[2 * kMaxBlocks];

// Block b sums p = |a|^2 and p^2 over amplitudes [b * kChunk, (b + 1) * kChunk), each thread
// in index order, then the threads in a fixed tree order.
__global__ void __launch_bounds__(kThreads) k_noalloc_partial(const double2 *amps, int64_t n,
                                                              double *scratch) {
    __shared__ double s1[kThreads], s2[kThreads];
    const int64_t begin = (int64_t)blockIdx.x * kChunk;
    int64_t end = begin + kChunk;
    if (end > n) end = n;
    double a1 = 0.0, a2 = 0.0;
    for (int64_t x = begin + threadIdx.x; x < end; x += kThreads) {
        const double2 v = amps[x];
        const double p = v.x * v.x + v.y * v.y;
        a1 += p;
        a2 += p * p;
    }
    s1[threadIdx.x] = a1;
    s2[threadIdx.x] = a2;
    __syncthreads();
    for (int w = kThreads / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) {
            s1[threadIdx.x] += s1[threadIdx.x + w];
            s2[threadIdx.x] += s2[threadIdx.x + w];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        scratch[2 * blockIdx.x] = s1[0];
        scratch[2 * blockIdx.x + 1] = s2[0];
    }
}

// One thread adds the block partials in block order into slots 0 and 1.
__global__ void k_noalloc_final(double *scratch, int nblocks) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double a1 = 0.0, a2 = 0.0;
    for (int b = 0; b < nblocks; ++b) {
        a1 += scratch[2 * b];
        a2 += scratch[2 * b + 1];
    }
    scratch[0] = a1;
    scratch[1] = a2;
}

std::mutex g_mu;
double *g_scratch_dev[kMaxDevices];  // device address of g_noalloc_scratch, per device

// Device address of the scratch array on `dev` (which is current), looked up once.
tn_status scratch_address(int dev, double **out) {
    if (dev < 0 || dev >= kMaxDevices)
        return tn::report(TN_ERR_UNSUPPORTED, "tn_readout_noalloc: device index out of range");
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_dev[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p)
            return tn::report(TN_ERR_CUDA, "tn_readout_noalloc: cudaGetSymbolAddress failed");
        g_scratch_dev[dev] = static_cast<double *>(p);
    }
    *out = g_scratch_dev[dev];
    return TN_OK;
}

}  // namespace

extern "C" tn_status tn_readout_noalloc(const void *amps_dev, int64_t num_amps, int32_t n_qubits,
                                        double out[4], void *stream_) {
    tn::clear_error();
    if (!amps_dev || !out || num_amps <= 0 || n_qubits < 0 || n_qubits > 1000)
        return tn::report(TN_ERR_INVALID_ARG, "tn_readout_noalloc: bad arguments");
    if (num_amps > kMaxAmps)
        return tn::report(TN_ERR_INVALID_ARG,
                          "tn_readout_noalloc: at most 2^28 amplitudes (its fixed scratch holds "
                          "4096 block sums of 65536 amplitudes each)");
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess)
        return tn::report(TN_ERR_CUDA, "tn_readout_noalloc: no current CUDA device");
    double *scratch = nullptr;
    tn_status st = scratch_address(dev, &scratch);
    if (st != TN_OK) return st;
    cudaStream_t stream = (cudaStream_t)stream_;
    const int nblocks = (int)((num_amps + kChunk - 1) / kChunk);
    k_noalloc_partial<<<nblocks, kThreads, 0, stream>>>(static_cast<const double2 *>(amps_dev),
                                                         num_amps, scratch);
    k_noalloc_final<<<1, 32, 0, stream>>>(scratch, nblocks);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess)
        return tn::report(TN_ERR_CUDA, "tn_readout_noalloc: launch failed");
    double h[2] = {0.0, 0.0};
    e = cudaMemcpyAsync(h, scratch, sizeof h, cudaMemcpyDeviceToHost, stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess)
        return tn::report(TN_ERR_CUDA, "tn_readout_noalloc: copy of the sums failed");
    const double D = std::ldexp(1.0, n_qubits);
    out[0] = h[0];
    out[1] = h[1];
    out[2] = D * h[0] / (double)num_amps - 1.0;
    out[3] = h[0] > 0.0 ? D * h[1] / h[0] - 1.0 : 0.0;
    return TN_OK;
}
