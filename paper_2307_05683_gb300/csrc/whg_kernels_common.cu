// whg_kernels_common.cu -- init and raw-state kernels, and the launchers that
// pick the Newton-phase series length.
#include "whg_device.cuh"

namespace whg {

__global__ void __launch_bounds__(WHG_MAX_BLOCK) k_init(WhgState st, WhgBuckets bk, WhgIn in)
{
    const int w = warp_index();
    if (w >= bk.warp0[bk.nb]) return;
    const int b = bucket_of(bk, w);
    WHG_DISPATCH_L(bk.L[b], (init_body<L_>(st, bk, in, b, w)))
}

__global__ void __launch_bounds__(WHG_MAX_BLOCK) k_raw(WhgState st, WhgBuckets bk, WhgOut io, int set)
{
    const int w = warp_index();
    if (w >= bk.warp0[bk.nb]) return;
    const int b = bucket_of(bk, w);
    WHG_DISPATCH_L(bk.L[b], (raw_body<L_>(st, bk, io, set, b, w)))
}

}  // namespace whg

cudaError_t whg_launch_init(const WhgState& st, const WhgBuckets& bk, const WhgIn& in, const WhgLaunch& l)
{
    whg::k_init<<<l.grid, l.block, 0, l.stream>>>(st, bk, in);
    return cudaGetLastError();
}

cudaError_t whg_launch_raw(const WhgState& st, const WhgBuckets& bk, const WhgOut& o, int set,
                           const WhgLaunch& l)
{
    whg::k_raw<<<l.grid, l.block, 0, l.stream>>>(st, bk, o, set);
    return cudaGetLastError();
}

cudaError_t whg_launch_step(const WhgState& st, const WhgBuckets& bk, long long n, int newton_terms,
                            int gr_mode, const WhgLaunch& l)
{
    return newton_terms == 6 ? whg_launch_step_nt6(st, bk, n, gr_mode, l)
                             : whg_launch_step_nt8(st, bk, n, gr_mode, l);
}

cudaError_t whg_launch_read(const WhgState& st, const WhgBuckets& bk, const WhgOut& o, int newton_terms,
                            const WhgLaunch& l)
{
    return newton_terms == 6 ? whg_launch_read_nt6(st, bk, o, l) : whg_launch_read_nt8(st, bk, o, l);
}

cudaError_t whg_launch_energy(const WhgState& st, const WhgBuckets& bk, const WhgOut& o, int newton_terms,
                              int gr_mode, const WhgLaunch& l)
{
    return newton_terms == 6 ? whg_launch_energy_nt6(st, bk, o, gr_mode, l)
                             : whg_launch_energy_nt8(st, bk, o, gr_mode, l);
}
