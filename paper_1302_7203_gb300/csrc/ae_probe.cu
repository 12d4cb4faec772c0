// ae_probe.cu -- throughput of the arithmetic pipes this solver runs on, for
// the denominators of its roofline (no counterpart in the paper).
//
// k_fma_rate: every thread runs U independent fused multiply-add chains
// a <- a b + c (b = 1 - 2^-10, c = 2^-10: the chains stay near 1, no
// subnormals, no overflow), so the pipe is fed U independent instructions per
// thread; the grid fills every SM to full occupancy.  b and c are loaded from
// device memory into registers: with them as kernel parameters (constant-bank
// operands) the FP64 pipe sustains only 1.6 of its 2 FMA lanes per clock and
// SM, with register operands 1.9.  Rate = 2 flops per FMA over the launch's
// CUDA-event time, best of three launches after a warm-up.
#include <cuda_runtime.h>

#include "ae_internal.h"

namespace ae {

template <typename T, int U>
__global__ void __launch_bounds__(256) k_fma_rate(int iters, const T *bc, T *out) {
    const T b = bc[0], c = bc[1];
    T a[U];
#pragma unroll
    for (int u = 0; u < U; ++u) a[u] = (T)1 + (T)(threadIdx.x + 3 * u) * (T)0x1p-20;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < U; ++u) a[u] = fma(a[u], b, c);
    }
    T s = 0;
#pragma unroll
    for (int u = 0; u < U; ++u) s += a[u];
    out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <typename T>
static cudaError_t time_fma(int iters, double *tflops, cudaStream_t st) {
    constexpr int U = 8;
    int dev = 0, sms = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (!e) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (!e) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fma_rate<T, U>, 256, 0);
    if (e) return e;
    const int grid = sms * (per_sm > 0 ? per_sm : 1);
    T *out = nullptr;
    e = cudaMallocAsync((void **)&out, sizeof(T) * ((size_t)grid * 256 + 2), st);
    if (e) return e;
    T *bc = out + (size_t)grid * 256;
    const T hbc[2] = {(T)1 - (T)0x1p-10, (T)0x1p-10};
    e = cudaMemcpyAsync(bc, hbc, sizeof(hbc), cudaMemcpyHostToDevice, st);
    if (!e) e = cudaStreamSynchronize(st);    // hbc is on this stack frame
    cudaEvent_t a = nullptr, z = nullptr;
    if (!e) e = cudaEventCreate(&a);
    if (!e) e = cudaEventCreate(&z);
    float best = 0.f;
    for (int r = 0; r < 4 && !e; ++r) {
        cudaEventRecord(a, st);
        k_fma_rate<T, U><<<grid, 256, 0, st>>>(iters, bc, out);
        cudaEventRecord(z, st);
        e = cudaEventSynchronize(z);
        float ms = 0.f;
        if (!e) e = cudaEventElapsedTime(&ms, a, z);
        if (!e && r > 0 && (best == 0.f || ms < best)) best = ms;   // launch 0: warm-up
    }
    if (!e) {
        const double flops = 2.0 * U * (double)iters * (double)grid * 256.0;
        *tflops = flops / (best * 1e-3) / 1e12;
    }
    if (a) cudaEventDestroy(a);
    if (z) cudaEventDestroy(z);
    cudaFreeAsync(out, st);
    return e;
}

cudaError_t probe_fma_rates(double *fp64_tflops, double *fp32_tflops, cudaStream_t st) {
    cudaError_t e = cudaSuccess;
    // ~30 ms a launch at the FP64 rate, ~10 ms at the FP32 rate
    if (fp64_tflops) e = time_fma<double>(1 << 14, fp64_tflops, st);
    if (!e && fp32_tflops) e = time_fma<float>(1 << 18, fp32_tflops, st);
    return e;
}

}  // namespace ae
