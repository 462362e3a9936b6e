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

// Ensemble repacking (no counterpart in the paper).  Within every bucket the
// systems still running come first and the stopped ones last, each group in
// its previous order, so that warps whose systems have all stopped skip their
// steps.  Each system's arithmetic involves only its own lanes, so moving it
// to other lanes leaves its results bitwise unchanged.
//
// order[new internal index] = old internal index; one block per bucket: a
// count of running systems, then a stable partition chunk by chunk
// (ballot/popc scan within warps, warp totals in shared memory).
__global__ void __launch_bounds__(1024) k_repack_order(WhgState st, WhgBuckets bk, int* order)
{
    const int b = blockIdx.x;
    if (b >= bk.nb) return;                                  // whole block
    const int s0 = bk.sys0[b], s1 = bk.sys0[b + 1];
    const int lane = (int)(threadIdx.x & 31u), wid = (int)(threadIdx.x >> 5), nw = (int)(blockDim.x >> 5);
    __shared__ int part[32];
    __shared__ int total;
    int cnt = 0;
    for (int s = s0 + (int)threadIdx.x; s < s1; s += (int)blockDim.x) cnt += st.status[s] == 0;
#pragma unroll
    for (int o = 16; o; o >>= 1) cnt += __shfl_xor_sync(WHG_FULL_MASK, cnt, o);
    if (lane == 0) part[wid] = cnt;
    __syncthreads();
    if (threadIdx.x == 0) {
        int t = 0;
        for (int i = 0; i < nw; ++i) t += part[i];
        total = t;
    }
    __syncthreads();
    const int nlive = total;
    int base_live = 0, base_stopped = 0;
    for (int c0 = s0; c0 < s1; c0 += (int)blockDim.x) {     // same trip count in every thread
        const int s = c0 + (int)threadIdx.x;
        const bool valid = s < s1;
        const bool live = valid && st.status[s] == 0;
        const unsigned bal = __ballot_sync(WHG_FULL_MASK, live);
        const int in_warp = __popc(bal & ((1u << lane) - 1u));
        __syncthreads();                                     // previous readers of part[] are done
        if (lane == 0) part[wid] = __popc(bal);
        __syncthreads();
        int before = 0, chunk_live = 0;
        for (int i = 0; i < nw; ++i) {
            const int v = part[i];
            before += i < wid ? v : 0;
            chunk_live += v;
        }
        const int excl = before + in_warp;                   // running systems before s in the chunk
        if (valid) {
            const int pos = live ? base_live + excl : nlive + base_stopped + ((int)threadIdx.x - excl);
            order[s0 + pos] = s;
        }
        const int nvalid = s1 - c0 < (int)blockDim.x ? s1 - c0 : (int)blockDim.x;
        base_live += chunk_live;
        base_stopped += nvalid - chunk_live;
    }
}

// Gather the state into dst in the new order: lane arrays for every lane in
// use (lanes that hold no system keep their index), per-system arrays once
// per system.  dst has the layout of src.
__global__ void __launch_bounds__(256) k_repack_gather(WhgState src, WhgState dst, WhgBuckets bk,
                                                       const int* order)
{
    const long long li = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int w = (int)(li >> 5);
    if (w >= bk.warp0[bk.nb]) return;
    const int lane = (int)(li & 31);
    const int b = bucket_of(bk, w);
    const int L = bk.L[b], spw = 32 / L;
    const int slot = lane / L, p = lane - slot * L;
    const int local = (w - bk.warp0[b]) * spw + slot;
    size_t from = (size_t)li;
    int s_new = -1, s_old = -1;
    if (slot < spw && local < bk.sys0[b + 1] - bk.sys0[b]) {
        s_new = bk.sys0[b] + local;
        s_old = order[s_new];
        WHG_CHECK(src, s_old >= bk.sys0[b] && s_old < bk.sys0[b + 1], WHG_BOUND_REPACK);
        const int lo = s_old - bk.sys0[b];
        from = (size_t)(bk.warp0[b] + lo / spw) * 32 + (size_t)(lo % spw) * L + p;
    }
    WHG_CHECK(src, (long long)from < src.nl && li < src.nl, WHG_BOUND_LANE);
    dst.m[li] = src.m[from];
    dst.qx[li] = src.qx[from];
    dst.qy[li] = src.qy[from];
    dst.qz[li] = src.qz[from];
    dst.vx[li] = src.vx[from];
    dst.vy[li] = src.vy[from];
    dst.vz[li] = src.vz[from];
    dst.a0[li] = src.a0[from];
    if (s_new >= 0 && p == 0) {
        const size_t S = (size_t)src.S;
        dst.m0[s_new] = src.m0[s_old];
        dst.dt[s_new] = src.dt[s_old];
        dst.M[s_new] = src.M[s_old];
        dst.rej2[s_new] = src.rej2[s_old];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            dst.xcm[k * S + s_new] = src.xcm[k * S + s_old];
            dst.vcm[k * S + s_new] = src.vcm[k * S + s_old];
        }
        dst.nstep[s_new] = src.nstep[s_old];
        dst.nplan[s_new] = src.nplan[s_old];
        dst.status[s_new] = src.status[s_old];
        dst.perm[s_new] = src.perm ? src.perm[s_old] : s_old;
    }
}

}  // namespace whg

cudaError_t whg_launch_repack(const WhgState& st, const WhgState& scratch, const WhgBuckets& bk, int* order,
                              cudaStream_t stream)
{
    whg::k_repack_order<<<bk.nb, 1024, 0, stream>>>(st, bk, order);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const long long lanes = (long long)bk.warp0[bk.nb] * 32;
    const int grid = (int)((lanes + 255) / 256);
    if (grid > 0) whg::k_repack_gather<<<grid, 256, 0, stream>>>(st, scratch, bk, order);
    return cudaGetLastError();
}

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

cudaError_t whg_launch_step_queue(const WhgState& st, const WhgBuckets& bk, long long n, int newton_terms,
                                  int gr_mode, const WhgQueue& q, cudaStream_t stream)
{
    return newton_terms == 6 ? whg_launch_step_queue_nt6(st, bk, n, gr_mode, q, stream)
                             : whg_launch_step_queue_nt8(st, bk, n, gr_mode, q, stream);
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
