// whg_diag.cu -- diagnostics of libwhg: FP64 pipe throughput and a test hook
// for the library's own reciprocal / reciprocal square root.
#include <cstdio>
#include <vector>

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

// The same loop with only the first `active` lanes of each warp working (the
// others skip it): shows whether masked lanes cost FP64 pipe time.
__global__ void k_dfma_lanes(double* out, int iters, int active)
{
    const int tid = blockIdx.x * blockDim.x + threadIdx.x;
    double a[kChains];
#pragma unroll
    for (int j = 0; j < kChains; ++j) a[j] = 1.0 + 1e-3 * (double)(tid + j);
    if ((int)(threadIdx.x & 31u) < active) {
        for (int i = 0; i < iters; ++i) {
#pragma unroll
            for (int j = 0; j < kChains; ++j) a[j] = fma(a[j], 0.999999, 1e-9);
        }
    }
    double s = 0.0;
#pragma unroll
    for (int j = 0; j < kChains; ++j) s += a[j];
    out[tid] = s;
}

// FP64 issue rate by instruction kind: 8 independent dependent chains per
// thread of DFMA (KIND 0), DMUL (1) or DADD (2), or DFMA with one integer
// multiply-add (3) or one FP32 FMA (4) on chains of their own after every
// DFMA.  Each block records its SM cycles (clock64) around the loop.
template <int KIND>
__global__ void k_fp64_kind(double* out, long long* cycles, int iters)
{
    const int tid = blockIdx.x * blockDim.x + threadIdx.x;
    double a[kChains];
    unsigned u[kChains];
    float f[kChains];
#pragma unroll
    for (int j = 0; j < kChains; ++j) {
        a[j] = 1.0 + 1e-3 * (double)(tid + j);
        u[j] = 7u * (unsigned)tid + (unsigned)j;
        f[j] = 1.0f + (float)j;
    }
    const long long t0 = clock64();
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int j = 0; j < kChains; ++j) {
            if (KIND == 1) a[j] = a[j] * 0.999999;
            else if (KIND == 2) a[j] = a[j] + 1e-9;
            else a[j] = fma(a[j], 0.999999, 1e-9);
            if (KIND == 3) u[j] = u[j] * 3u + 1u;
            if (KIND == 4) f[j] = fmaf(f[j], 0.999f, 1e-3f);
        }
    }
    const long long t1 = clock64();
    double s = 0.0;
#pragma unroll
    for (int j = 0; j < kChains; ++j) s += a[j] + (double)u[j] + (double)f[j];
    out[tid] = s;
    if (threadIdx.x == 0) cycles[blockIdx.x] = t1 - t0;
}

// Kepler drift with runtime iteration counts and series lengths, for the
// solver search of Appendix A: 1/k! for k = 0..31 in constant memory; the
// G_n after the last iteration are evaluated at the final X with the Newton
// series length (the definition the oracle uses).
__constant__ double c_invfact[32];

__device__ __forceinline__ void stumpff_rt(double z, int T, double& c2, double& c3)
{
    c2 = c_invfact[2 * T + 2];      // series through z^T, as the step kernels sum it
    c3 = c_invfact[2 * T + 3];
    for (int k = T - 1; k >= 0; --k) {
        c2 = fma(-z, c2, c_invfact[2 * k + 2]);
        c3 = fma(-z, c3, c_invfact[2 * k + 3]);
    }
}

__global__ void k_kepler_sweep(const double* q, const double* v, const int* cfg, int n, double mu, double h,
                               long long steps, double* qo, double* vo)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double qx = q[3 * i], qy = q[3 * i + 1], qz = q[3 * i + 2];
    double vx = v[3 * i], vy = v[3 * i + 1], vz = v[3 * i + 2];
    // clamped: series of 1..12 terms keep every table index below 32
    const int hi = min(max(cfg[4 * i], 0), 16), ht = min(max(cfg[4 * i + 1], 1), 12);
    const int ni = min(max(cfg[4 * i + 2], 0), 16), nt = min(max(cfg[4 * i + 3], 1), 12);
    for (long long s = 0; s < steps; ++s) {
        const double r0 = sqrt(qx * qx + qy * qy + qz * qz);
        const double eta0 = qx * vx + qy * vy + qz * vz;
        const double beta = 2.0 * mu / r0 - (vx * vx + vy * vy + vz * vz);
        const double zeta0 = mu - beta * r0;
        double X = h / r0;
        double c2, c3;
        for (int it = 0; it < hi + ni; ++it) {
            const int T = it < hi ? ht : nt;
            const double X2 = X * X;
            stumpff_rt(beta * X2, T, c2, c3);
            const double G2 = X2 * c2, G3 = X2 * X * c3;
            const double G0 = 1.0 - beta * G2, G1 = X - beta * G3;
            const double F = r0 * G1 + eta0 * G2 + mu * G3 - h;
            const double Fp = r0 * G0 + eta0 * G1 + mu * G2;
            if (it < hi) {
                const double Fpp = eta0 * G0 + zeta0 * G1;
                X = X - 2.0 * F * Fp / (2.0 * Fp * Fp - F * Fpp);
            } else {
                X = X - F / Fp;
            }
        }
        const double X2 = X * X;
        stumpff_rt(beta * X2, nt, c2, c3);
        const double G2 = X2 * c2, G3 = X2 * X * c3;
        const double G0 = 1.0 - beta * G2, G1 = X - beta * G3;
        const double r = r0 * G0 + eta0 * G1 + mu * G2;
        const double f = 1.0 - mu * G2 / r0, g = h - mu * G3;
        const double fd = -mu * G1 / (r * r0), gd = 1.0 - mu * G2 / r;
        const double nqx = f * qx + g * vx, nqy = f * qy + g * vy, nqz = f * qz + g * vz;
        vx = fd * qx + gd * vx;
        vy = fd * qy + gd * vy;
        vz = fd * qz + gd * vz;
        qx = nqx; qy = nqy; qz = nqz;
    }
    qo[3 * i] = qx; qo[3 * i + 1] = qy; qo[3 * i + 2] = qz;
    vo[3 * i] = vx; vo[3 * i + 1] = vy; vo[3 * i + 2] = vz;
}

// The same seeds refined with FP64 operations only (e = fma(-x, y, 1),
// y^2 = y*y, y^3 = y^2*y, the correction polynomial in FP64): references
// the integer-pipe forms in whg_device.cuh must match within one ulp.
__device__ double rcp_fp64_ref(double x)
{
    const unsigned hi = (unsigned)__double2hiint(x);
    const unsigned lo = (unsigned)__double2loint(x);
    const int ex = (int)((hi >> 20) & 0x7ffu);
    const float mant = __uint_as_float(0x3f800000u | ((hi & 0x000fffffu) << 3) | (lo >> 29));
    const unsigned rb = __float_as_uint(whg::approx_rcp_f32(mant));
    const int dex = (int)((rb >> 23) & 0xffu) - 127 + 2046 - ex;
    const unsigned yhi = (hi & 0x80000000u) | ((unsigned)dex << 20) | ((rb >> 3) & 0x000fffffu);
    const double y = __hiloint2double((int)yhi, (int)(rb << 29));
    const double e = fma(-x, y, 1.0);
    return fma(y, fma(e, e, e), y);
}

__device__ double rsqrt_seed_ref(double x)
{
    const unsigned hi = (unsigned)__double2hiint(x);
    const unsigned lo = (unsigned)__double2loint(x);
    const int ex = (int)((hi >> 20) & 0x7ffu) - 1023;
    const int odd = ex & 1;
    const int half = (ex - odd) / 2;
    const float mant = __uint_as_float(((unsigned)(127 + odd) << 23) | ((hi & 0x000fffffu) << 3) | (lo >> 29));
    const unsigned rb = __float_as_uint(whg::approx_rsqrt_f32(mant));
    const int dex = (int)((rb >> 23) & 0xffu) - 127 - half + 1023;
    return __hiloint2double((int)(((unsigned)dex << 20) | ((rb >> 3) & 0x000fffffu)), (int)(rb << 29));
}

__device__ double rsqrt_fp64_ref(double x)
{
    const double y = rsqrt_seed_ref(x);
    const double e = fma(-x, y * y, 1.0);
    return fma(y * e, fma(0.375, e, 0.5), y);
}

__device__ double rsqrt_cubed_fp64_ref(double x)
{
    const double y = rsqrt_seed_ref(x);
    const double y2 = y * y;
    const double e = fma(-x, y2, 1.0);
    const double y3 = y2 * y;
    return fma(y3 * e, fma(1.875, e, 1.5), y3);
}

__global__ void k_special(const double* x, int n, double* out)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double v = x[i];
    const bool pos = v > 0.0 && v < 4.0e307;          // the rsqrt routines' domain (below 2^1022)
    out[i] = whg::rcp(v);
    out[n + i] = 1.0 / v;
    out[2 * n + i] = pos ? whg::rsqrt(v) : 0.0;
    out[3 * n + i] = pos ? ::rsqrt(v) : 0.0;
    out[4 * n + i] = whg::to_f64(whg::to_f32(v));
    out[5 * n + i] = (double)__double2float_rz(v);
    out[6 * n + i] = rcp_fp64_ref(v);
    out[7 * n + i] = pos ? rsqrt_fp64_ref(v) : 0.0;
    const bool nonneg = v >= 0.0 && v < 4.0e307;      // also zero: a coincident pair's r^2
    out[8 * n + i] = nonneg ? whg::rsqrt_cubed(v) : 0.0;
    out[9 * n + i] = nonneg ? rsqrt_cubed_fp64_ref(v) : 0.0;
    const double inv = 1.0 / v;
    out[10 * n + i] = nonneg ? whg::rcp_sq(v) : 0.0;
    out[11 * n + i] = nonneg ? inv * inv : 0.0;
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

int whg_probe_fp64_lanes(int warps_per_sm, int active_lanes, int iters, float* ms)
{
    if (!ms || warps_per_sm < 1 || warps_per_sm > 64 || active_lanes < 1 || active_lanes > 32 ||
        iters < 1 || iters > (1 << 24))
        return WHG_EINVAL;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return WHG_ECUDA;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return WHG_ECUDA;
    const int blocks = sms * warps_per_sm;        // one warp per block
    double* out = nullptr;
    if (cudaMalloc(&out, sizeof(double) * 32 * (size_t)blocks) != cudaSuccess) return WHG_ENOMEM;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    k_dfma_lanes<<<blocks, 32>>>(out, 64, active_lanes);          // warm-up
    cudaEventRecord(e0, 0);
    k_dfma_lanes<<<blocks, 32>>>(out, iters, active_lanes);
    cudaEventRecord(e1, 0);
    int rc = WHG_OK;
    if (cudaEventSynchronize(e1) != cudaSuccess || cudaGetLastError() != cudaSuccess) rc = WHG_ECUDA;
    else cudaEventElapsedTime(ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(out);
    return rc;
}

int whg_probe_fp64_kind(int kind, int warps_per_sm, int iters, double* lanes_per_clk)
{
    if (!lanes_per_clk || kind < 0 || kind > 4 || warps_per_sm < 1 || warps_per_sm > 32 || iters < 1 ||
        iters > (1 << 24))
        return WHG_EINVAL;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return WHG_ECUDA;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return WHG_ECUDA;
    const int blocks = sms * warps_per_sm;        // one warp per block, at most 32 blocks per SM: all resident
    void* buf = nullptr;
    if (cudaMalloc(&buf, (sizeof(double) * 32 + sizeof(long long)) * (size_t)blocks) != cudaSuccess)
        return WHG_ENOMEM;
    double* out = (double*)buf;
    long long* cyc = (long long*)(out + 32 * (size_t)blocks);
    auto launch = [&](int n) {
        switch (kind) {
            case 0: k_fp64_kind<0><<<blocks, 32>>>(out, cyc, n); break;
            case 1: k_fp64_kind<1><<<blocks, 32>>>(out, cyc, n); break;
            case 2: k_fp64_kind<2><<<blocks, 32>>>(out, cyc, n); break;
            case 3: k_fp64_kind<3><<<blocks, 32>>>(out, cyc, n); break;
            default: k_fp64_kind<4><<<blocks, 32>>>(out, cyc, n); break;
        }
    };
    launch(64);                                   // warm-up
    launch(iters);
    std::vector<long long> h((size_t)blocks);
    int rc = WHG_OK;
    if (cudaDeviceSynchronize() != cudaSuccess || cudaGetLastError() != cudaSuccess ||
        cudaMemcpy(h.data(), cyc, sizeof(long long) * h.size(), cudaMemcpyDeviceToHost) != cudaSuccess) {
        rc = WHG_ECUDA;
    } else {
        long long mx = 1;
        for (long long c : h) mx = c > mx ? c : mx;
        *lanes_per_clk = (double)iters * kChains * 32.0 * warps_per_sm / (double)mx;
    }
    cudaFree(buf);
    return rc;
}

int whg_kepler_sweep(const double* q, const double* v, const int* cfg, int n, double mu, double h,
                     long long steps, double* q_out, double* v_out)
{
    if (!q || !v || !cfg || !q_out || !v_out || n < 0 || steps < 0 || !(mu > 0.0) || !(h > 0.0))
        return WHG_EINVAL;
    if (n == 0) return WHG_OK;
    static bool table_ready = false;      // 1/k!, k = 0..31, rounded once from the exact factorial
    if (!table_ready) {
        double t[32];
        long double f = 1.0L;
        for (int k = 0; k < 32; ++k) {
            if (k > 1) f *= (long double)k;
            t[k] = (double)(1.0L / f);
        }
        if (cudaMemcpyToSymbol(c_invfact, t, sizeof t) != cudaSuccess) return WHG_ECUDA;
        table_ready = true;
    }
    k_kepler_sweep<<<(n + 127) / 128, 128>>>(q, v, cfg, n, mu, h, steps, q_out, v_out);
    if (cudaGetLastError() != cudaSuccess) return WHG_ECUDA;
    if (cudaDeviceSynchronize() != cudaSuccess) return WHG_ECUDA;
    return WHG_OK;
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
