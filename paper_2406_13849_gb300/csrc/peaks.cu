// peaks.cu - microbenchmarks that measure the ceilings the tracking kernels
// are reported against: FP64 and FP32 fused multiply-add issue rate and the
// rate of 64-bit integer atomic adds into L2 (spread and contended).  The
// caller times the launch (CUDA events on `stream`) and divides the
// operation count this returns by the elapsed time.
#include <cstdint>

#include "trk.h"
#include "trk_internal.h"

namespace {

template <class T>
__global__ void __launch_bounds__(256) k_fma(T* out, int iters, T seed) {
    T a0 = seed + T(threadIdx.x), a1 = a0 + T(1), a2 = a0 + T(2), a3 = a0 + T(3);
    T a4 = a0 + T(4), a5 = a0 + T(5), a6 = a0 + T(6), a7 = a0 + T(7);
    const T m = T(0.999999), c = T(1e-7);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            a0 = fma(a0, m, c); a1 = fma(a1, m, c); a2 = fma(a2, m, c); a3 = fma(a3, m, c);
            a4 = fma(a4, m, c); a5 = fma(a5, m, c); a6 = fma(a6, m, c); a7 = fma(a7, m, c);
        }
    }
    const T s = ((a0 + a1) + (a2 + a3)) + ((a4 + a5) + (a6 + a7));
    if (s == T(-12345.0)) out[threadIdx.x] = s;   // keeps the chain live
}

__global__ void __launch_bounds__(256) k_atomic(unsigned long long* bins, int nbins, int iters) {
    const unsigned tid = blockIdx.x * blockDim.x + threadIdx.x;
    unsigned h = tid * 2654435761u;
    for (int i = 0; i < iters; ++i) {
        h = h * 1664525u + 1013904223u;
        atomicAdd(bins + (h >> 8) % unsigned(nbins), 1ULL);
    }
}

}  // namespace

extern "C" {

// Peak microbenchmark (no counterpart in the paper; measurement support).
// kind 0: FP64 FMA, 1: FP32 FMA (result = flops, 2 per FMA);
// kind 2: u64 atomicAdd over `nbins` counters in dev_scratch (result = atomics).
// Launches blocks x 256 threads on `stream`; dev_scratch needs 8 * max(nbins, 256) bytes.
trk_status trk_peak_kernel(int kind, int blocks, int iters, int nbins, void* dev_scratch, size_t scratch_bytes,
                           double* ops, void* stream) {
    if (blocks <= 0 || iters <= 0 || !ops || !dev_scratch)
        return trk_status(trk::set_error(TRK_E_INVALID, "trk_peak_kernel: bad arguments"));
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const double threads = double(blocks) * 256.0;
    if (kind == 0) {
        if (scratch_bytes < 256 * sizeof(double)) return trk_status(trk::set_error(TRK_E_NOMEM, "scratch too small"));
        k_fma<double><<<blocks, 256, 0, s>>>(static_cast<double*>(dev_scratch), iters, 1.0);
        *ops = threads * iters * 32.0 * 2.0;
    } else if (kind == 1) {
        if (scratch_bytes < 256 * sizeof(float)) return trk_status(trk::set_error(TRK_E_NOMEM, "scratch too small"));
        k_fma<float><<<blocks, 256, 0, s>>>(static_cast<float*>(dev_scratch), iters, 1.0f);
        *ops = threads * iters * 32.0 * 2.0;
    } else if (kind == 2) {
        if (nbins <= 0 || scratch_bytes < size_t(nbins) * 8) return trk_status(trk::set_error(TRK_E_NOMEM, "scratch too small"));
        k_atomic<<<blocks, 256, 0, s>>>(static_cast<unsigned long long*>(dev_scratch), nbins, iters);
        *ops = threads * iters;
    } else {
        return trk_status(trk::set_error(TRK_E_INVALID, "trk_peak_kernel: unknown kind %d", kind));
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return trk_status(trk::set_error(TRK_E_CUDA, "trk_peak_kernel: %s", cudaGetErrorString(e)));
    return TRK_OK;
}

}  // extern "C"
