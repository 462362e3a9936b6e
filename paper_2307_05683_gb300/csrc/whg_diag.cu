// whg_diag.cu -- diagnostics of libwhg: FP64 pipe throughput and a test hook
// for the library's own reciprocal / reciprocal square root.
#include <cstdio>

#include "whg_device.cuh"

namespace {

constexpr int kChains = 8;     // independent FMA chains per thread

__global__ void __launch_bounds__(256) k_dfma_loop(double* out, int iters, double seed)
{
    const int tid = blockIdx.x * blockDim.x + threadIdx.x;
    double a[kChains];
#pragma unroll
    for (int j = 0; j < kChains; ++j) a[j] = seed + 1e-3 * (double)(tid + j);
    const double b = 0.999999, c = 1e-9;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int j = 0; j < kChains; ++j) a[j] = fma(a[j], b, c);
    }
    double s = 0.0;
#pragma unroll
    for (int j = 0; j < kChains; ++j) s += a[j];
    out[tid] = s;
}

__global__ void k_special(const double* x, int n, double* out)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double v = x[i];
    out[i] = whg::rcp(v);
    out[n + i] = 1.0 / v;
    out[2 * n + i] = v > 0.0 ? whg::rsqrt(v) : 0.0;
    out[3 * n + i] = v > 0.0 ? ::rsqrt(v) : 0.0;
}

}  // namespace

extern "C" {

int whg_measure_fp64_tflops(double seconds, double* tflops)
{
    if (!tflops || !(seconds > 0.0)) return WHG_EINVAL;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return WHG_ECUDA;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return WHG_ECUDA;
    const int threads = 256, blocks = sms * 8;
    double* out = nullptr;
    if (cudaMalloc(&out, sizeof(double) * threads * blocks) != cudaSuccess) return WHG_ENOMEM;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    int iters = 256;
    float ms = 0.0f;
    int rc = WHG_OK;
    for (int round = 0; round < 12; ++round) {        // grow until the run lasts `seconds`
        cudaEventRecord(e0, 0);
        k_dfma_loop<<<blocks, threads>>>(out, iters, 1.0);
        cudaEventRecord(e1, 0);
        if (cudaEventSynchronize(e1) != cudaSuccess || cudaGetLastError() != cudaSuccess) {
            rc = WHG_ECUDA;
            break;
        }
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms >= 1e3 * seconds || iters >= (1 << 26)) break;
        const double grow = ms > 0.5f ? (1e3 * seconds) / ms * 1.05 : 16.0;
        iters = (int)(iters * (grow > 16.0 ? 16.0 : grow)) + 1;
    }
    if (rc == WHG_OK)
        *tflops = 2.0 * kChains * (double)iters * threads * blocks / (ms * 1e-3) / 1e12;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(out);
    return rc;
}

int whg_test_special(const double* x, int n, double* out)
{
    if (!x || !out || n < 0) return WHG_EINVAL;
    if (n == 0) return WHG_OK;
    k_special<<<(n + 255) / 256, 256>>>(x, n, out);
    if (cudaGetLastError() != cudaSuccess) return WHG_ECUDA;
    if (cudaDeviceSynchronize() != cudaSuccess) return WHG_ECUDA;
    return WHG_OK;
}

}  // extern "C"
