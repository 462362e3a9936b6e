// whg_kernels_nt6.cu -- step, read and energy kernels with 6-term Stumpff
// series in the Newton phase (all lane counts, all GR modes).
#include "whg_device.cuh"

cudaError_t whg_launch_step_nt6(const WhgState& st, const WhgBuckets& bk, long long n, int gr_mode,
                                  const WhgLaunch& l)
{
    if (gr_mode == 0)
        whg::k_step<6, 0><<<l.grid, l.block, 0, l.stream>>>(st, bk, n);
    else if (gr_mode == 1)
        whg::k_step<6, 1><<<l.grid, l.block, 0, l.stream>>>(st, bk, n);
    else
        whg::k_step<6, 2><<<l.grid, l.block, 0, l.stream>>>(st, bk, n);
    return cudaGetLastError();
}

namespace {

// One warp per block; as many blocks as can be resident at once (capped at
// the number of warp-groups), so every warp of the launch runs from the start.
template <typename Kernel>
cudaError_t launch_queue(Kernel kern, const WhgState& st, const WhgBuckets& bk, long long n,
                         const WhgQueue& q, cudaStream_t stream)
{
    int per_sm = 0, dev = 0, sms = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 32, 0);
    if (e != cudaSuccess) return e;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    long long grid = (long long)(per_sm > 0 ? per_sm : 1) * sms;
    if (grid > bk.warp0[bk.nb]) grid = bk.warp0[bk.nb];
    if (grid < 1) return cudaSuccess;
    kern<<<(int)grid, 32, 0, stream>>>(st, bk, n, q);
    return cudaGetLastError();
}

}  // namespace

cudaError_t whg_launch_step_queue_nt6(const WhgState& st, const WhgBuckets& bk, long long n, int gr_mode,
                                       const WhgQueue& q, cudaStream_t stream)
{
    if (gr_mode == 0) return launch_queue(whg::k_step_queue<6, 0>, st, bk, n, q, stream);
    if (gr_mode == 1) return launch_queue(whg::k_step_queue<6, 1>, st, bk, n, q, stream);
    return launch_queue(whg::k_step_queue<6, 2>, st, bk, n, q, stream);
}

cudaError_t whg_launch_read_nt6(const WhgState& st, const WhgBuckets& bk, const WhgOut& o,
                                  const WhgLaunch& l)
{
    whg::k_read<6><<<l.grid, l.block, 0, l.stream>>>(st, bk, o);
    return cudaGetLastError();
}

cudaError_t whg_launch_energy_nt6(const WhgState& st, const WhgBuckets& bk, const WhgOut& o,
                                    int gr_mode, const WhgLaunch& l)
{
    if (gr_mode == 0)
        whg::k_energy<6, 0><<<l.grid, l.block, 0, l.stream>>>(st, bk, o);
    else
        whg::k_energy<6, 1><<<l.grid, l.block, 0, l.stream>>>(st, bk, o);
    return cudaGetLastError();
}
