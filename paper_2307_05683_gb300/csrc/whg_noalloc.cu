// whg_noalloc.cu -- whg_integrate_noalloc: init + n steps + synchronized read
// of an ensemble in one call that allocates no memory.
//
// For callers that cannot allocate device memory themselves or let a library
// do it: frameworks that reserve the GPU's memory up front and only hand out
// buffers from their own pool, host applications or plugins whose policy
// forbids device allocation once they are running, and loops that cannot pay
// cudaMalloc's implicit device-wide synchronization.  The caller passes device
// inputs and outputs; the working state (democratic heliocentric coordinates
// between the init, step and read kernels) lives in the fixed array below.
#include <cstdio>

#include "whg_internal.h"

namespace {

// Layout of the working state for at most WHG_NOALLOC_MAX_LANES lanes (whole
// warps of floor(32 / L) systems each): 8 lane arrays, 10 per-system doubles,
// one per-system int64 and two per-system ints.
constexpr size_t kLanes = WHG_NOALLOC_MAX_LANES;
constexpr size_t kSystems = WHG_NOALLOC_MAX_LANES;   // at least one lane per system
constexpr size_t kBytes = (8 * kLanes + 10 * kSystems) * sizeof(double) + kSystems * sizeof(long long) +
                          2 * kSystems * sizeof(int);

// Device-side scratch.  In host code this name is only a host stand-in: its
// device address comes from cudaGetSymbolAddress (per device, below).
static __device__ __align__(256) unsigned char g_scratch[kBytes];
#ifdef WHG_DEBUG_BOUNDS
static __device__ unsigned g_noalloc_bounds;      // index-check flag of the debug build
#endif

int noalloc_fail(int code, const char* fmt, const char* detail)
{
    char msg[256];
    snprintf(msg, sizeof msg, fmt, detail);
    whg_record_error(msg);
    return code;
}

// Device address of g_scratch on the current device.  Looked up on every
// call (the lookup allocates nothing), so that no address outlives a reset
// of the device's primary context; the first lookup on a device may load the
// library's device image, which is why the first call must precede any
// stream capture.
int scratch_address(void** out)
{
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess || !p)
        return noalloc_fail(WHG_ECUDA, "cudaGetSymbolAddress(scratch): %s", cudaGetErrorString(e));
    *out = p;
    return WHG_OK;
}

}  // namespace

extern "C" int whg_integrate_noalloc(int n_systems, int max_planets, const whg_options* opt_in,
                                     const double* masses, const double* pos, const double* vel,
                                     const int* n_planets, const double* dt, long long n_steps,
                                     double* pos_out, double* vel_out, int* status_out, double* t_out,
                                     void* cuda_stream)
{
    whg_options opt;
    whg_default_options(&opt);
    if (opt_in) opt = *opt_in;
    if (n_systems < 1 || max_planets < 1 || max_planets > WHG_MAX_PLANETS)
        return noalloc_fail(WHG_EINVAL, "whg_integrate_noalloc: %s", "need n_systems >= 1 and max_planets in 1..8");
    if (!masses || !pos || !vel || !dt || !pos_out || !vel_out)
        return noalloc_fail(WHG_EINVAL, "whg_integrate_noalloc: %s", "null input or output array");
    if (n_steps < 0) return noalloc_fail(WHG_EINVAL, "whg_integrate_noalloc: %s", "n_steps must be >= 0");
    if (opt.gr_mode < 0 || opt.gr_mode > 2 || (opt.newton_terms != 6 && opt.newton_terms != 8) ||
        (opt.gr_mode && !(opt.c_light > 0.0)) || opt.steps_per_launch < 0)
        return noalloc_fail(WHG_EINVAL, "whg_integrate_noalloc: %s", "invalid options");
    if (opt.lanes_per_system < 0 || opt.lanes_per_system > 8 ||
        (opt.lanes_per_system && opt.lanes_per_system < max_planets))
        return noalloc_fail(WHG_EINVAL, "whg_integrate_noalloc: %s", "lanes_per_system must be 0 or in max_planets..8");
    if (opt.close_encounter_hill < 0.0 || opt.eject_factor < 0.0)
        return noalloc_fail(WHG_EINVAL, "whg_integrate_noalloc: %s", "stop rules must be >= 0");
    // One lane group size for every system (the planet counts stay on the
    // device): lanes_per_system, or the packed size for max_planets.
    const int L = opt.lanes_per_system ? opt.lanes_per_system : whg_lanes_for_planets(max_planets);
    const int block = opt.block_size ? opt.block_size : 32;
    if (block < 32 || block > WHG_MAX_BLOCK || block % 32)
        return noalloc_fail(WHG_EINVAL, "whg_integrate_noalloc: %s", "block_size must be a multiple of 32 in 32..256");
    const int spw = 32 / L;
    const long long warps = ((long long)n_systems + spw - 1) / spw;
    if (warps * 32 > (long long)kLanes) {
        char why[160];
        snprintf(why, sizeof why, "%d systems x %d lanes exceed the fixed scratch of %d lanes",
                 n_systems, L, WHG_NOALLOC_MAX_LANES);
        return noalloc_fail(WHG_EINVAL, "whg_integrate_noalloc: %s", why);
    }

    void* base = nullptr;
    int rc = scratch_address(&base);
    if (rc) return rc;

    // Carve the state out of the scratch array (same layout as a context).
    const size_t NL = (size_t)warps * 32, P = (size_t)n_systems;
    WhgState st;
    double* d = (double*)base;
    st.m = d; d += NL;
    st.qx = d; d += NL;
    st.qy = d; d += NL;
    st.qz = d; d += NL;
    st.vx = d; d += NL;
    st.vy = d; d += NL;
    st.vz = d; d += NL;
    st.a0 = d; d += NL;
    st.m0 = d; d += P;
    st.dt = d; d += P;
    st.M = d; d += P;
    st.xcm = d; d += 3 * P;
    st.vcm = d; d += 3 * P;
    st.rej2 = d; d += P;
    long long* ll = (long long*)d;
    st.nstep = ll; ll += P;
    int* ip = (int*)ll;
    st.nplan = ip; ip += P;
    st.status = ip;
    st.perm = nullptr;
    st.nl = (long long)NL;
    st.dbg = nullptr;
#ifdef WHG_DEBUG_BOUNDS
    {
        void* flagp = nullptr;
        if (cudaGetSymbolAddress(&flagp, g_noalloc_bounds) != cudaSuccess)
            return noalloc_fail(WHG_ECUDA, "cudaGetSymbolAddress(bounds flag): %s", "");
        st.dbg = (unsigned*)flagp;
    }
#endif
    st.S = n_systems;
    st.Nmax = max_planets;
    st.c_light = opt.c_light;
    st.hill = opt.close_encounter_hill;
    st.eject = opt.eject_factor;
    st.merge = (opt.merge_jumps && opt.gr_mode == 0) ? 1 : 0;
    st.halley32 = opt.halley_fp32 ? 1 : 0;
    st.full_rotation = opt.interaction_schedule == 1 ? 1 : 0;

    WhgBuckets bk{};
    bk.nb = 1;
    bk.L[0] = L;
    bk.warp0[1] = (int)warps;
    bk.sys0[1] = n_systems;
    WhgLaunch l;
    l.block = block;
    l.grid = (int)((NL + block - 1) / block);
    l.stream = (cudaStream_t)cuda_stream;

    // The init kernel writes every lane and per-system field read later
    // (status and step counters start at zero), so stale contents left by an
    // earlier call are never read.
    WhgIn in{masses, pos, vel, n_planets, dt};
    cudaError_t e = whg_launch_init(st, bk, in, l);
    if (e != cudaSuccess) return noalloc_fail(WHG_ECUDA, "init kernel: %s", cudaGetErrorString(e));
    long long chunk = opt.steps_per_launch > 0 ? opt.steps_per_launch : 50000000LL / (warps * 4 + 1);
    if (chunk < 1) chunk = 1;
    for (long long left = n_steps; left > 0;) {
        const long long k = left < chunk ? left : chunk;
        e = whg_launch_step(st, bk, k, opt.newton_terms, opt.gr_mode, l);
        if (e != cudaSuccess) return noalloc_fail(WHG_ECUDA, "step kernel: %s", cudaGetErrorString(e));
        left -= k;
    }
    WhgOut o{};
    o.pos = pos_out;
    o.vel = vel_out;
    o.status = status_out;
    o.t = t_out;
    e = whg_launch_read(st, bk, o, opt.newton_terms, l);
    if (e != cudaSuccess) return noalloc_fail(WHG_ECUDA, "read kernel: %s", cudaGetErrorString(e));
    return WHG_OK;
}

// Index-check flags of whg_integrate_noalloc in the debug build (see the
// declaration in whg.h).  No allocation: the flag word is a device symbol.
extern "C" int whg_noalloc_debug_bounds(unsigned* flag)
{
    if (!flag) return WHG_EINVAL;
#ifdef WHG_DEBUG_BOUNDS
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpyFromSymbol(flag, g_noalloc_bounds, sizeof(unsigned));
    const unsigned zero = 0;
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(g_noalloc_bounds, &zero, sizeof(unsigned));
    if (e != cudaSuccess) return noalloc_fail(WHG_ECUDA, "whg_noalloc_debug_bounds: %s", cudaGetErrorString(e));
    return WHG_OK;
#else
    *flag = 0;
    return noalloc_fail(WHG_EINVAL, "whg_noalloc_debug_bounds: %s", "index checks are not compiled in (build with debug=True)");
#endif
}
