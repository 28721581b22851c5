// Measurement helpers (no counterpart in the paper): the library's own copy kernel, to measure
// the bandwidth of a working set that stays in L2 (or one that streams from HBM), and its own
// FP64 fused-multiply-add kernel, to measure the FP64 rate.  They state the roofline
// denominators of the step kernels that are not bound by HBM: the L2-resident meshes and the
// FP64 form.
#include <cuda_runtime.h>

#include "../../include/fedfem.h"

namespace {

// dst <- src, 16-byte vectors, grid-stride, `reps` passes over the same buffers.
__global__ void __launch_bounds__(512) k_probe_copy(float4 *__restrict__ dst, const float4 *__restrict__ src,
                                                     int64_t n, int reps)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int r = 0; r < reps; ++r)
        for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) dst[i] = src[i];
}

// Eight independent FMA chains per thread, `iters` FMAs each; the result goes to sink so
// that nothing is optimised away.
__global__ void __launch_bounds__(256) k_probe_fp64(int64_t iters, double a, double b, double *sink)
{
    double x[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) x[k] = (double)(threadIdx.x + k) * 1e-3;
    for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < 8; ++k) x[k] = fma(x[k], a, b);
    }
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < 8; ++k) s += x[k];
    if (s == 12345.678) sink[0] = s;  // never true for the inputs used; keeps the chains live
}

fedfem_status time_launches(cudaStream_t st, cudaEvent_t e0, cudaEvent_t e1, double *ms)
{
    if (cudaEventRecord(e1, st) != cudaSuccess) return FEDFEM_ERR_CUDA;
    if (cudaEventSynchronize(e1) != cudaSuccess) return FEDFEM_ERR_CUDA;
    float f = 0.f;
    if (cudaEventElapsedTime(&f, e0, e1) != cudaSuccess) return FEDFEM_ERR_CUDA;
    *ms = f;
    return FEDFEM_OK;
}

}  // namespace

extern "C" fedfem_status fedfem_probe_copy(void *dst_dev, const void *src_dev, int64_t bytes, int32_t reps,
                                           int32_t blocks_per_sm, void *stream, double *ms_out)
{
    if (!dst_dev || !src_dev || !ms_out || bytes < 16 || bytes % 16 || reps < 1 || blocks_per_sm < 1)
        return FEDFEM_ERR_ARG;
    if (((uintptr_t)dst_dev | (uintptr_t)src_dev) & 15) return FEDFEM_ERR_ARG;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return FEDFEM_ERR_CUDA;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return FEDFEM_ERR_CUDA;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return FEDFEM_ERR_CUDA;
    }
    fedfem_status s = FEDFEM_OK;
    const int64_t n = bytes / 16;
    // one untimed pass (first touch), then the timed ones
    k_probe_copy<<<sms * blocks_per_sm, 512, 0, st>>>((float4 *)dst_dev, (const float4 *)src_dev, n, 1);
    if (cudaGetLastError() != cudaSuccess || cudaEventRecord(e0, st) != cudaSuccess) s = FEDFEM_ERR_CUDA;
    if (s == FEDFEM_OK) {
        k_probe_copy<<<sms * blocks_per_sm, 512, 0, st>>>((float4 *)dst_dev, (const float4 *)src_dev, n, reps);
        s = cudaGetLastError() == cudaSuccess ? time_launches(st, e0, e1, ms_out) : FEDFEM_ERR_CUDA;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return s;
}

extern "C" fedfem_status fedfem_probe_fp64(int64_t iters, int32_t blocks_per_sm, void *stream, double *ms_out,
                                           double *flops_out)
{
    if (!ms_out || !flops_out || iters < 1 || blocks_per_sm < 1) return FEDFEM_ERR_ARG;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return FEDFEM_ERR_CUDA;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    double *sink = nullptr;
    if (cudaMalloc(&sink, 8) != cudaSuccess) return FEDFEM_ERR_OOM;
    cudaEvent_t e0, e1;
    fedfem_status s = FEDFEM_OK;
    if (cudaEventCreate(&e0) != cudaSuccess) {
        cudaFree(sink);
        return FEDFEM_ERR_CUDA;
    }
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        cudaFree(sink);
        return FEDFEM_ERR_CUDA;
    }
    const int grid = sms * blocks_per_sm;
    k_probe_fp64<<<grid, 256, 0, st>>>(iters / 8 + 1, 0.999999, 1e-7, sink);  // warm-up
    if (cudaGetLastError() != cudaSuccess || cudaEventRecord(e0, st) != cudaSuccess) s = FEDFEM_ERR_CUDA;
    if (s == FEDFEM_OK) {
        k_probe_fp64<<<grid, 256, 0, st>>>(iters, 0.999999, 1e-7, sink);
        s = cudaGetLastError() == cudaSuccess ? time_launches(st, e0, e1, ms_out) : FEDFEM_ERR_CUDA;
    }
    *flops_out = 2.0 * 8.0 * (double)iters * (double)grid * 256.0;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(sink);
    return s;
}
