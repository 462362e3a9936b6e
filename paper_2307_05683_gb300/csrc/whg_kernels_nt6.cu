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
