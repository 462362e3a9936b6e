// whg_api.cu -- host side of libwhg: the C ABI declared in include/whg.h.
//
// A context owns the ensemble's device state (structure of arrays; systems
// grouped by planet count, see whg_internal.h) and staging buffers for host
// I/O.  Every operation is a kernel on
// the context's stream; host-pointer calls add one cudaMemcpyAsync each way and
// wait for it.  Inputs given as host arrays are validated on the host.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include <cuda.h>
#include <cudaTypedefs.h>

#include "whg_internal.h"

struct whg_ctx {
    int S, Nmax, block, Lfixed, warps_cap;
    whg_options opt;
    cudaStream_t stream;
    int device;
    bool initialized;
    long long launches;
    WhgState st;
    WhgBuckets bk;
    int* perm_d;              // [S] device copy of the internal -> caller permutation
    // staging for host I/O (device memory)
    double* stage_d;          // S * (7 * (1 + Nmax) + 1) doubles
    int* stage_i;             // 2 * S ints
    long long* stage_l;       // S int64
    long long host_nstep;     // steps since init (-1: unknown after set_raw)
    // adjoint buffers (allocated by whg_adjoint_forward, kept until destroy)
    double* adj_buf;
    size_t adj_bytes;
    WhgAdj adj;
    long long adj_n;
    int adj_K, adj_nseg;
    bool adj_ready;
    cudaStream_t side[2];     // side streams for tape recomputation (created on first use)
    cudaEvent_t ev_entry, ev_ckpt, ev_exit;
    std::vector<cudaEvent_t> ev_tape, ev_back;   // per tape buffer
    std::vector<int> tape_of; // segment whose tape each buffer holds (-1: none)
    int adj_nbuf;             // tape buffers of the current forward half
    // adjoint scheduling (whg_adjoint_schedule): SM split by green contexts
    int cfg_split;            // -1 auto, 0 off, n > 0: SMs of the chain partition
    long long cfg_tape_bytes; // 0 three buffers (default), -1 half the free memory, n > 0 cap
    bool split;               // the current forward half runs split
    int chain_sms, tape_sms;  // SMs of the two green contexts (0: none)
    CUgreenCtx g_chain, g_tape;
    CUcontext x_chain, x_tape;
    cudaStream_t s_chain, s_tape[2];
    // CUDA graph of graph_launches step launches of graph_chunk steps each
    cudaStream_t capture;
    cudaGraphExec_t graph;
    long long graph_chunk;
    // repacking (opt.repack_frozen): a mirror of the state block and the order
    void* state_base;
    size_t state_bytes;
    void* repack_buf;
    WhgState scratch;
    int* order;
    long long since_repack;   // step launches since the last repack
    // work queue (opt.queue_steps > 0): unit counter, per-group chunks done, error flag
    unsigned long long* q_next;
    int* q_done;
    int* q_err;
    char err[256];
};

namespace {

thread_local char g_create_err[256] = "";

int fail(whg_ctx* c, int code, const char* fmt, ...)
{
    char* dst = c ? c->err : g_create_err;
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(dst, 256, fmt, ap);
    va_end(ap);
    return code;
}

int cuda_fail(whg_ctx* c, cudaError_t e, const char* what)
{
    return fail(c, WHG_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define WHG_CUDA(ctx, call)                                          \
    do {                                                             \
        cudaError_t e_ = (call);                                     \
        if (e_ != cudaSuccess) return cuda_fail((ctx), e_, #call);   \
    } while (0)

WhgLaunch launch_cfg(const whg_ctx* c)
{
    WhgLaunch l;
    l.block = c->block;
    const long long threads = (long long)c->bk.warp0[c->bk.nb] * 32;
    l.grid = (int)((threads + c->block - 1) / c->block);
    if (l.grid < 1) l.grid = 1;
    l.stream = c->stream;
    return l;
}

int systems_per_warp(int L) { return 32 / L; }

// Warps needed in the worst case of planet-count mix (packed) or for the
// fixed lane count.
int warps_capacity(int S, int Nmax, int Lfixed)
{
    if (Lfixed) return (S + systems_per_warp(Lfixed) - 1) / systems_per_warp(Lfixed);
    int spw_min = 32;
    for (int n = 1; n <= Nmax; ++n) {
        const int spw = systems_per_warp(whg_lanes_for_planets(n));
        if (spw < spw_min) spw_min = spw;
    }
    return (S + spw_min - 1) / spw_min + 8;
}

// Bucket systems by lanes per system.  nplan may be null (all Nmax planets).
// perm receives, for every internal system, the caller's index (the
// identity when every system gets the same lane group, which repacking
// starts from); returns false when the layout is the identity.
bool plan_layout(int S, int Nmax, int Lfixed, const int* nplan, WhgBuckets* bk, int* perm)
{
    *bk = WhgBuckets{};
    if (Lfixed || !nplan) {
        for (int s = 0; s < S; ++s) perm[s] = s;
        const int L = Lfixed ? Lfixed : whg_lanes_for_planets(Nmax);
        bk->nb = 1;
        bk->L[0] = L;
        bk->warp0[0] = 0;
        bk->warp0[1] = (S + systems_per_warp(L) - 1) / systems_per_warp(L);
        bk->sys0[0] = 0;
        bk->sys0[1] = S;
        return false;
    }
    int count[9] = {0};
    auto lanes_of = [&](int s) {
        const int n = nplan[s];
        return whg_lanes_for_planets(n >= 1 && n <= Nmax ? n : Nmax);   // invalid: frozen anyway
    };
    for (int s = 0; s < S; ++s) count[lanes_of(s)] += 1;
    int next[9] = {0}, nb = 0, warps = 0, sys = 0;
    for (int L = 1; L <= 8; ++L) {
        if (!count[L]) continue;
        bk->L[nb] = L;
        bk->warp0[nb] = warps;
        bk->sys0[nb] = sys;
        next[L] = sys;
        warps += (count[L] + systems_per_warp(L) - 1) / systems_per_warp(L);
        sys += count[L];
        ++nb;
    }
    bk->nb = nb;
    bk->warp0[nb] = warps;
    bk->sys0[nb] = S;
    bool identity = true;
    for (int s = 0; s < S; ++s) {
        const int i = next[lanes_of(s)]++;
        perm[i] = s;
        identity &= (i == s);
    }
    return !identity;
}

bool finite(double x) { return std::isfinite(x); }

// Host-side validation of inertial inputs (returns system index of the first
// bad system, or -1).
int validate(const whg_ctx* c, const double* m, const double* x, const double* u, const int* np,
             const double* dt, char* why, size_t nwhy)
{
    const int B = 1 + c->Nmax;
    for (int s = 0; s < c->S; ++s) {
        const int n = np ? np[s] : c->Nmax;
        const double* ms = m + (size_t)s * B;
        const double* xs = x + (size_t)s * B * 3;
        const double* us = u + (size_t)s * B * 3;
        if (n < 1 || n > c->Nmax) { snprintf(why, nwhy, "n_planets=%d outside 1..%d", n, c->Nmax); return s; }
        if (!(dt[s] > 0.0) || !finite(dt[s])) { snprintf(why, nwhy, "dt=%g must be finite and > 0", dt[s]); return s; }
        if (!(ms[0] > 0.0) || !finite(ms[0])) { snprintf(why, nwhy, "star mass %g must be > 0", ms[0]); return s; }
        for (int k = 0; k <= n; ++k) {
            if (!(ms[k] >= 0.0) || !finite(ms[k])) { snprintf(why, nwhy, "mass of body %d is %g", k, ms[k]); return s; }
            for (int d = 0; d < 3; ++d)
                if (!finite(xs[3 * k + d]) || !finite(us[3 * k + d])) {
                    snprintf(why, nwhy, "non-finite coordinate of body %d", k);
                    return s;
                }
            if (k > 0 && xs[3 * k] == xs[0] && xs[3 * k + 1] == xs[1] && xs[3 * k + 2] == xs[2]) {
                snprintf(why, nwhy, "planet %d sits on the star", k);
                return s;
            }
        }
    }
    return -1;
}

// Point the fields of st into one state block (lane arrays: L entries each,
// per-system arrays: P); returns the block's [P] int region after status
// (the internal -> caller map).
int* carve_state(WhgState& st, void* base, size_t L, size_t P)
{
    double* d = (double*)base;
    st.m = d; d += L;
    st.qx = d; d += L;
    st.qy = d; d += L;
    st.qz = d; d += L;
    st.vx = d; d += L;
    st.vy = d; d += L;
    st.vz = d; d += L;
    st.a0 = d; d += L;
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
    st.status = ip; ip += P;
    return ip;
}

// n_steps for every system on `stream`: the work-queue kernel (its counter
// and per-group flags cleared first) when the launch spans at least
// kQueueMinUnits units per warp-group, else one step kernel.  With fewer
// units there is nothing to rebalance (measured: one unit per group costs
// ~5 % on 65,536 compact systems).
constexpr long long kQueueMinUnits = 4;

// Polls of a work-queue wait before it gives up (each at least ~100 ns of
// sleep: several seconds, against at most ~0.5 s for the longest legitimate
// wait, one unit of 1e4 steps).
constexpr long long kQueueSpinLimit = 1LL << 26;

cudaError_t launch_steps(whg_ctx* c, long long n_steps, const WhgLaunch& l)
{
    const long long qs = c->opt.queue_steps;
    if (!c->q_next || n_steps < kQueueMinUnits * qs)
        return whg_launch_step(c->st, c->bk, n_steps, c->opt.newton_terms, c->opt.gr_mode, l);
    WhgQueue q{c->q_next, c->q_done, c->q_err, qs, (int)((n_steps + qs - 1) / qs), kQueueSpinLimit};
    cudaError_t e = cudaMemsetAsync(c->q_next, 0, sizeof(unsigned long long), l.stream);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(c->q_done, 0, sizeof(int) * (size_t)c->bk.warp0[c->bk.nb], l.stream);
    if (e != cudaSuccess) return e;
    return whg_launch_step_queue(c->st, c->bk, n_steps, c->opt.newton_terms, c->opt.gr_mode, q, l.stream);
}

// After a synchronization: a work-queue wait that gave up is an error.
int check_queue(whg_ctx* c)
{
    if (!c->q_err) return WHG_OK;
    int flag = 0;
    WHG_CUDA(c, cudaMemcpy(&flag, c->q_err, sizeof(int), cudaMemcpyDeviceToHost));
    if (flag) {
        WHG_CUDA(c, cudaMemset(c->q_err, 0, sizeof(int)));   // reported once
        return fail(c, WHG_ECUDA, "work-queue wait gave up (state of this context is inconsistent)");
    }
    return WHG_OK;
}

// Repack on `stream`: live systems first in every bucket, through the mirror
// block, copied back so that every pointer (and captured graph) stays valid.
cudaError_t enqueue_repack(whg_ctx* c, cudaStream_t stream)
{
    cudaError_t e = whg_launch_repack(c->st, c->scratch, c->bk, c->order, stream);
    if (e != cudaSuccess) return e;
    return cudaMemcpyAsync(c->state_base, c->repack_buf, c->state_bytes, cudaMemcpyDeviceToDevice, stream);
}

int launch_check(whg_ctx* c, cudaError_t e, const char* what)
{
    if (e != cudaSuccess) return cuda_fail(c, e, what);
    c->launches += 1;
    return WHG_OK;
}

}  // namespace

void whg_record_error(const char* msg) { snprintf(g_create_err, sizeof g_create_err, "%s", msg); }

extern "C" {

void whg_default_options(whg_options* opt)
{
    if (!opt) return;
    opt->gr_mode = 1;
    opt->c_light = 173.1446326742403 / 0.01720209895;
    opt->newton_terms = 8;
    opt->lanes_per_system = 0;
    opt->block_size = 0;
    opt->steps_per_launch = 0;
    opt->close_encounter_hill = 0.0;
    opt->eject_factor = 0.0;
    opt->graph_launches = 0;
    opt->merge_jumps = 0;
    opt->halley_fp32 = 0;
    opt->repack_frozen = -1;
    opt->interaction_schedule = 0;
    opt->queue_steps = 100;
}

int whg_create(whg_ctx** out, int n_systems, int max_planets, const whg_options* opt_in,
               void* cuda_stream)
{
    if (!out) return fail(nullptr, WHG_EINVAL, "out is NULL");
    *out = nullptr;
    whg_options opt;
    whg_default_options(&opt);
    if (opt_in) opt = *opt_in;
    if (n_systems < 1) return fail(nullptr, WHG_EINVAL, "n_systems=%d must be >= 1", n_systems);
    if (max_planets < 1 || max_planets > WHG_MAX_PLANETS)
        return fail(nullptr, WHG_EINVAL, "max_planets=%d outside 1..%d", max_planets, WHG_MAX_PLANETS);
    if (opt.gr_mode < 0 || opt.gr_mode > 2) return fail(nullptr, WHG_EINVAL, "gr_mode=%d", opt.gr_mode);
    if (opt.gr_mode && !(opt.c_light > 0.0 && std::isfinite(opt.c_light)))
        return fail(nullptr, WHG_EINVAL, "c_light=%g must be > 0", opt.c_light);
    if (opt.newton_terms != 6 && opt.newton_terms != 8)
        return fail(nullptr, WHG_EINVAL, "newton_terms=%d must be 6 or 8", opt.newton_terms);
    const int Lfixed = opt.lanes_per_system;
    if (Lfixed < 0 || Lfixed > 8 || (Lfixed && Lfixed < max_planets))
        return fail(nullptr, WHG_EINVAL, "lanes_per_system=%d must be 0 or in max_planets..8",
                    opt.lanes_per_system);
    if (opt.close_encounter_hill < 0.0 || !std::isfinite(opt.close_encounter_hill) ||
        opt.eject_factor < 0.0 || !std::isfinite(opt.eject_factor))
        return fail(nullptr, WHG_EINVAL, "stop rules must be finite and >= 0");
    int block = opt.block_size ? opt.block_size : 32;
    if (block < 32 || block > WHG_MAX_BLOCK || block % 32)
        return fail(nullptr, WHG_EINVAL, "block_size=%d must be a multiple of 32 in 32..%d", block,
                    WHG_MAX_BLOCK);
    if (opt.steps_per_launch < 0)
        return fail(nullptr, WHG_EINVAL, "steps_per_launch=%lld must be >= 0", opt.steps_per_launch);
    if (opt.graph_launches < 0 || opt.graph_launches > 4096)
        return fail(nullptr, WHG_EINVAL, "graph_launches=%d must be in 0..4096", opt.graph_launches);
    if (opt.repack_frozen < -1 || opt.repack_frozen > 1)
        return fail(nullptr, WHG_EINVAL, "repack_frozen=%d must be -1, 0 or 1", opt.repack_frozen);
    if (opt.repack_frozen < 0)                           // auto: on when a stop rule can stop systems
        opt.repack_frozen = (opt.close_encounter_hill > 0.0 || opt.eject_factor > 0.0) ? 1 : 0;
    if (opt.interaction_schedule != 0 && opt.interaction_schedule != 1)
        return fail(nullptr, WHG_EINVAL, "interaction_schedule=%d must be 0 or 1", opt.interaction_schedule);
    if (opt.queue_steps < 0 || opt.queue_steps > 10000)
        return fail(nullptr, WHG_EINVAL, "queue_steps=%d must be in 0..10000", opt.queue_steps);

    whg_ctx* c = new (std::nothrow) whg_ctx();
    if (!c) return fail(nullptr, WHG_ENOMEM, "host allocation failed");
    c->S = n_systems;
    c->Nmax = max_planets;
    c->Lfixed = Lfixed;
    c->block = block;
    c->warps_cap = warps_capacity(n_systems, max_planets, Lfixed);
    c->opt = opt;
    c->stream = (cudaStream_t)cuda_stream;
    c->cfg_split = -1;
    c->cfg_tape_bytes = 0;
    cudaError_t e = cudaGetDevice(&c->device);
    if (e != cudaSuccess) {
        delete c;
        return fail(nullptr, WHG_ECUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
    }

    const size_t L = (size_t)c->warps_cap * 32, P = (size_t)n_systems;
    const size_t nd = 8 * L + 10 * P;
    void* base = nullptr;
    size_t bytes = nd * sizeof(double) + P * sizeof(long long) + 3 * P * sizeof(int);
    e = cudaMalloc(&base, bytes);
    if (e != cudaSuccess) {
        delete c;
        return fail(nullptr, WHG_ENOMEM, "cudaMalloc(%zu): %s", bytes, cudaGetErrorString(e));
    }
    c->state_base = base;
    c->state_bytes = bytes;
    WhgState& st = c->st;
    c->perm_d = carve_state(st, base, L, P);
    st.perm = nullptr;
    st.nl = (long long)L;
#ifdef WHG_DEBUG_BOUNDS
    e = cudaMalloc(&st.dbg, sizeof(unsigned));
    if (e == cudaSuccess) e = cudaMemset(st.dbg, 0, sizeof(unsigned));
    if (e != cudaSuccess) {
        cudaFree(base);
        delete c;
        return fail(nullptr, WHG_ENOMEM, "cudaMalloc(bounds flag): %s", cudaGetErrorString(e));
    }
#endif
    if (opt.repack_frozen) {                             // mirror block + order array
        e = cudaMalloc(&c->repack_buf, bytes + P * sizeof(int));
        if (e != cudaSuccess) {
            cudaFree(base);
            delete c;
            return fail(nullptr, WHG_ENOMEM, "cudaMalloc(%zu): %s", bytes + P * sizeof(int),
                        cudaGetErrorString(e));
        }
        c->scratch.perm = carve_state(c->scratch, c->repack_buf, L, P);
        c->scratch.S = n_systems;
        c->scratch.nl = (long long)L;
        c->scratch.dbg = st.dbg;
        c->order = (int*)((char*)c->repack_buf + bytes);
    }
    st.S = n_systems;
    st.Nmax = max_planets;
    st.c_light = opt.c_light;
    st.hill = opt.close_encounter_hill;
    st.eject = opt.eject_factor;
    st.merge = (opt.merge_jumps && opt.gr_mode == 0) ? 1 : 0;
    st.halley32 = opt.halley_fp32 ? 1 : 0;
    st.full_rotation = opt.interaction_schedule == 1 ? 1 : 0;

    if (opt.queue_steps > 0) {                           // counter, per-group flags, error flag
        const size_t qbytes = sizeof(unsigned long long) + sizeof(int) * ((size_t)c->warps_cap + 1);
        void* qb = nullptr;
        e = cudaMalloc(&qb, qbytes);
        if (e == cudaSuccess) e = cudaMemset(qb, 0, qbytes);
        if (e != cudaSuccess) {
            if (qb) cudaFree(qb);
            cudaFree(base);
            if (c->repack_buf) cudaFree(c->repack_buf);
            delete c;
            return fail(nullptr, WHG_ENOMEM, "cudaMalloc(%zu): %s", qbytes, cudaGetErrorString(e));
        }
        c->q_next = (unsigned long long*)qb;
        c->q_err = (int*)(c->q_next + 1);
        c->q_done = c->q_err + 1;
    }
    const size_t B = 1 + (size_t)max_planets;
    const size_t sd = (size_t)n_systems * (7 * B + 1);
    const size_t sbytes = sd * sizeof(double) + 2 * (size_t)n_systems * sizeof(int) +
                          (size_t)n_systems * sizeof(long long);
    void* sbase = nullptr;
    e = cudaMalloc(&sbase, sbytes);
    if (e != cudaSuccess) {
        cudaFree(base);
        if (c->repack_buf) cudaFree(c->repack_buf);
        if (c->q_next) cudaFree(c->q_next);
        delete c;
        return fail(nullptr, WHG_ENOMEM, "cudaMalloc(%zu): %s", sbytes, cudaGetErrorString(e));
    }
    c->stage_d = (double*)sbase;
    c->stage_l = (long long*)(c->stage_d + sd);
    c->stage_i = (int*)(c->stage_l + n_systems);
    *out = c;
    return WHG_OK;
}

int whg_set_stream(whg_ctx* c, void* cuda_stream)
{
    if (!c) return WHG_EINVAL;
    c->stream = (cudaStream_t)cuda_stream;
    return WHG_OK;
}

// Lay the ensemble out by planet count (nplan_host: caller's n_planets on the
// host, or null) and run the init kernel on the inputs `in`.
static int init_common(whg_ctx* c, const WhgIn& in, const int* nplan_host)
{
    std::vector<int> perm((size_t)c->S);
    const bool permuted = plan_layout(c->S, c->Nmax, c->Lfixed, nplan_host, &c->bk, perm.data());
    if (c->bk.warp0[c->bk.nb] > c->warps_cap)
        return fail(c, WHG_EINVAL, "internal layout exceeds capacity");
    if (permuted || c->repack_buf) {                     // repacking needs the map even if identity
        WHG_CUDA(c, cudaMemcpyAsync(c->perm_d, perm.data(), perm.size() * sizeof(int),
                                    cudaMemcpyHostToDevice, c->stream));
        c->st.perm = c->perm_d;
    } else {
        c->st.perm = nullptr;
    }
    int rc = launch_check(c, whg_launch_init(c->st, c->bk, in, launch_cfg(c)), "init kernel");
    if (rc) return rc;
    c->initialized = true;
    c->host_nstep = 0;
    c->adj_ready = false;
    c->since_repack = 0;
    if (c->graph) {                                      // kernel arguments changed: capture again
        cudaGraphExecDestroy(c->graph);
        c->graph = nullptr;
    }
    WHG_CUDA(c, cudaStreamSynchronize(c->stream));      // host buffers may be reused on return
    return WHG_OK;
}

int whg_init(whg_ctx* c, const double* masses, const double* pos, const double* vel,
             const int* n_planets, const double* dt)
{
    if (!c) return WHG_EINVAL;
    if (!masses || !pos || !vel || !dt) return fail(c, WHG_EINVAL, "null input array");
    char why[160];
    int bad = validate(c, masses, pos, vel, n_planets, dt, why, sizeof why);
    if (bad >= 0) return fail(c, WHG_EINVAL, "system %d: %s", bad, why);
    const size_t S = c->S, B = 1 + (size_t)c->Nmax;
    double* dm = c->stage_d;
    double* dx = dm + S * B;
    double* du = dx + S * B * 3;
    double* ddt = du + S * B * 3;
    WHG_CUDA(c, cudaMemcpyAsync(dm, masses, S * B * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    WHG_CUDA(c, cudaMemcpyAsync(dx, pos, S * B * 3 * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    WHG_CUDA(c, cudaMemcpyAsync(du, vel, S * B * 3 * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    WHG_CUDA(c, cudaMemcpyAsync(ddt, dt, S * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    int* dn = nullptr;
    if (n_planets) {
        dn = c->stage_i;
        WHG_CUDA(c, cudaMemcpyAsync(dn, n_planets, S * sizeof(int), cudaMemcpyHostToDevice, c->stream));
    }
    WhgIn in{dm, dx, du, dn, ddt};
    return init_common(c, in, n_planets);
}

int whg_init_device(whg_ctx* c, const double* masses, const double* pos, const double* vel,
                    const int* n_planets, const double* dt)
{
    if (!c) return WHG_EINVAL;
    if (!masses || !pos || !vel || !dt) return fail(c, WHG_EINVAL, "null input array");
    WhgIn in{masses, pos, vel, n_planets, dt};
    if (n_planets && !c->Lfixed) {                       // the layout needs the planet counts
        std::vector<int> np((size_t)c->S);
        WHG_CUDA(c, cudaMemcpyAsync(np.data(), n_planets, np.size() * sizeof(int),
                                    cudaMemcpyDeviceToHost, c->stream));
        WHG_CUDA(c, cudaStreamSynchronize(c->stream));
        return init_common(c, in, np.data());
    }
    return init_common(c, in, nullptr);
}

// n steps; repack = false (the adjoint's forward half) keeps every system on
// its lanes: no repack, and no replay of a captured graph that holds one.
// `over` (the adjoint's partition) replaces the launch configuration and
// skips graphs.
static int step_impl(whg_ctx* c, long long n, bool repack, const WhgLaunch* over = nullptr)
{
    long long chunk = c->opt.steps_per_launch;
    if (chunk <= 0) {
        // about 5e7 system-steps per launch (a few tenths of a second)
        chunk = 50000000LL / ((long long)c->bk.warp0[c->bk.nb] * 4 + 1);
        if (chunk < 1) chunk = 1;
    }
    WhgLaunch l = over ? *over : launch_cfg(c);
    if (c->host_nstep >= 0) c->host_nstep += n;
    c->adj_ready = false;
    const long long G = c->opt.graph_launches;
    if (!over && G > 0 && n >= G * chunk && (repack || !c->repack_buf)) {
        if (!c->graph || c->graph_chunk != chunk) {      // capture G launches once
            if (c->graph) {
                cudaGraphExecDestroy(c->graph);
                c->graph = nullptr;
            }
            if (!c->capture) WHG_CUDA(c, cudaStreamCreateWithFlags(&c->capture, cudaStreamNonBlocking));
            WhgLaunch cl = l;
            cl.stream = c->capture;
            WHG_CUDA(c, cudaStreamBeginCapture(c->capture, cudaStreamCaptureModeThreadLocal));
            cudaError_t e = cudaSuccess;
            for (long long i = 0; i < G && e == cudaSuccess; ++i) e = launch_steps(c, chunk, cl);
            if (e == cudaSuccess && c->repack_buf) e = enqueue_repack(c, c->capture);   // once per replay
            cudaGraph_t graph = nullptr;
            const cudaError_t e2 = cudaStreamEndCapture(c->capture, &graph);
            if (e != cudaSuccess) return cuda_fail(c, e, "step kernel (capture)");
            if (e2 != cudaSuccess) return cuda_fail(c, e2, "cudaStreamEndCapture");
            const cudaError_t e3 = cudaGraphInstantiate(&c->graph, graph, 0);
            cudaGraphDestroy(graph);
            if (e3 != cudaSuccess) {
                c->graph = nullptr;
                return cuda_fail(c, e3, "cudaGraphInstantiate");
            }
            c->graph_chunk = chunk;
        }
        while (n >= G * chunk) {                          // replay on the context's stream
            WHG_CUDA(c, cudaGraphLaunch(c->graph, c->stream));
            c->launches += G + (c->repack_buf ? 2 : 0);
            if (c->repack_buf) c->since_repack = 0;
            n -= G * chunk;
        }
    }
    const long long every = G > 0 ? G : 16;              // step launches between repacks
    while (n > 0) {
        const long long k = n < chunk ? n : chunk;
        int rc = launch_check(c, launch_steps(c, k, l), "step kernel");
        if (rc) return rc;
        n -= k;
        if (repack && c->repack_buf && ++c->since_repack >= every) {
            WHG_CUDA(c, enqueue_repack(c, c->stream));
            c->launches += 2;
            c->since_repack = 0;
        }
    }
    return WHG_OK;
}

int whg_step(whg_ctx* c, long long n)
{
    if (!c) return WHG_EINVAL;
    if (!c->initialized) return fail(c, WHG_ESTATE, "whg_step before whg_init");
    if (n < 0) return fail(c, WHG_EINVAL, "n_steps=%lld must be >= 0", n);
    return step_impl(c, n, true);
}

int whg_read_state_device(whg_ctx* c, double* pos, double* vel, int* status, double* t)
{
    if (!c) return WHG_EINVAL;
    if (!c->initialized) return fail(c, WHG_ESTATE, "read before whg_init");
    WhgOut o{};
    o.pos = pos;
    o.vel = vel;
    o.status = status;
    o.t = t;
    return launch_check(c, whg_launch_read(c->st, c->bk, o, c->opt.newton_terms, launch_cfg(c)),
                        "read kernel");
}

int whg_read_state(whg_ctx* c, double* pos, double* vel, int* status, double* t)
{
    if (!c) return WHG_EINVAL;
    if (!pos || !vel) return fail(c, WHG_EINVAL, "null output array");
    const size_t S = c->S, B = 1 + (size_t)c->Nmax;
    double* dx = c->stage_d;
    double* du = dx + S * B * 3;
    double* dtm = du + S * B * 3;
    int* dst = c->stage_i;
    int rc = whg_read_state_device(c, dx, du, dst, dtm);
    if (rc) return rc;
    WHG_CUDA(c, cudaMemcpyAsync(pos, dx, S * B * 3 * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    WHG_CUDA(c, cudaMemcpyAsync(vel, du, S * B * 3 * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    if (status)
        WHG_CUDA(c, cudaMemcpyAsync(status, dst, S * sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    if (t) WHG_CUDA(c, cudaMemcpyAsync(t, dtm, S * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    WHG_CUDA(c, cudaStreamSynchronize(c->stream));
    return check_queue(c);
}

int whg_energy_device(whg_ctx* c, double* E)
{
    if (!c) return WHG_EINVAL;
    if (!c->initialized) return fail(c, WHG_ESTATE, "energy before whg_init");
    if (!E) return fail(c, WHG_EINVAL, "null output array");
    WhgOut o{};
    o.E = E;
    return launch_check(c, whg_launch_energy(c->st, c->bk, o, c->opt.newton_terms, c->opt.gr_mode,
                                             launch_cfg(c)),
                        "energy kernel");
}

int whg_energy(whg_ctx* c, double* E)
{
    if (!c) return WHG_EINVAL;
    if (!E) return fail(c, WHG_EINVAL, "null output array");
    int rc = whg_energy_device(c, c->stage_d);
    if (rc) return rc;
    WHG_CUDA(c, cudaMemcpyAsync(E, c->stage_d, (size_t)c->S * sizeof(double), cudaMemcpyDeviceToHost,
                                c->stream));
    WHG_CUDA(c, cudaStreamSynchronize(c->stream));
    return WHG_OK;
}

int whg_get_raw(whg_ctx* c, double* Q, double* v, long long* nstep, int* status)
{
    if (!c) return WHG_EINVAL;
    if (!c->initialized) return fail(c, WHG_ESTATE, "get_raw before whg_init");
    if (!Q || !v || !nstep || !status) return fail(c, WHG_EINVAL, "null output array");
    const size_t S = c->S, N = c->Nmax;
    WhgOut o{};
    o.rawQ = c->stage_d;
    o.rawv = c->stage_d + S * N * 3;
    o.rawn = c->stage_l;
    o.status = c->stage_i;
    int rc = launch_check(c, whg_launch_raw(c->st, c->bk, o, 0, launch_cfg(c)), "raw kernel");
    if (rc) return rc;
    WHG_CUDA(c, cudaMemcpyAsync(Q, o.rawQ, S * N * 3 * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    WHG_CUDA(c, cudaMemcpyAsync(v, o.rawv, S * N * 3 * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    WHG_CUDA(c, cudaMemcpyAsync(nstep, o.rawn, S * sizeof(long long), cudaMemcpyDeviceToHost, c->stream));
    WHG_CUDA(c, cudaMemcpyAsync(status, o.status, S * sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    WHG_CUDA(c, cudaStreamSynchronize(c->stream));
    return WHG_OK;
}

int whg_set_raw(whg_ctx* c, const double* Q, const double* v, const long long* nstep,
                const int* status)
{
    if (!c) return WHG_EINVAL;
    if (!c->initialized) return fail(c, WHG_ESTATE, "set_raw before whg_init");
    if (!Q || !v || !nstep || !status) return fail(c, WHG_EINVAL, "null input array");
    const size_t S = c->S, N = c->Nmax;
    for (size_t s = 0; s < S; ++s)
        if (nstep[s] < 0) return fail(c, WHG_EINVAL, "nstep[%zu] < 0", s);
    double* dQ = c->stage_d;
    double* dv = dQ + S * N * 3;
    WHG_CUDA(c, cudaMemcpyAsync(dQ, Q, S * N * 3 * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    WHG_CUDA(c, cudaMemcpyAsync(dv, v, S * N * 3 * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    WHG_CUDA(c, cudaMemcpyAsync(c->stage_l, nstep, S * sizeof(long long), cudaMemcpyHostToDevice, c->stream));
    WHG_CUDA(c, cudaMemcpyAsync(c->stage_i, status, S * sizeof(int), cudaMemcpyHostToDevice, c->stream));
    WhgOut o{};
    o.inQ = dQ;
    o.inv = dv;
    o.inn = c->stage_l;
    o.ins = c->stage_i;
    int rc = launch_check(c, whg_launch_raw(c->st, c->bk, o, 1, launch_cfg(c)), "raw kernel");
    if (rc) return rc;
    c->host_nstep = -1;
    c->adj_ready = false;
    WHG_CUDA(c, cudaStreamSynchronize(c->stream));
    return WHG_OK;
}

int whg_synchronize(whg_ctx* c)
{
    if (!c) return WHG_EINVAL;
    WHG_CUDA(c, cudaStreamSynchronize(c->stream));
    return check_queue(c);
}

long long whg_launch_count(const whg_ctx* c) { return c ? c->launches : 0; }

int whg_debug_bounds(whg_ctx* c, unsigned* flag)
{
    if (!c || !flag) return WHG_EINVAL;
#ifdef WHG_DEBUG_BOUNDS
    WHG_CUDA(c, cudaStreamSynchronize(c->stream));
    WHG_CUDA(c, cudaMemcpy(flag, c->st.dbg, sizeof(unsigned), cudaMemcpyDeviceToHost));
    WHG_CUDA(c, cudaMemset(c->st.dbg, 0, sizeof(unsigned)));
    return WHG_OK;
#else
    *flag = 0;
    return fail(c, WHG_EINVAL, "index checks are not compiled in (build with debug=True)");
#endif
}

int whg_test_queue_timeout(whg_ctx* c, long long spin_limit, int* flag)
{
    if (!c || !flag || spin_limit < 1) return WHG_EINVAL;
    if (!c->q_next) return fail(c, WHG_EINVAL, "the work queue is off (queue_steps = 0)");
    if (!c->initialized) return fail(c, WHG_ESTATE, "whg_test_queue_timeout before whg_init");
    const unsigned long long G = (unsigned long long)c->bk.warp0[c->bk.nb];
    const long long qs = c->opt.queue_steps;
    // the counter starts past every group's first unit, whose completion
    // each remaining unit then waits for in vain
    WhgQueue q{c->q_next, c->q_done, c->q_err, qs, 2, spin_limit};
    WHG_CUDA(c, cudaMemcpyAsync(c->q_next, &G, sizeof G, cudaMemcpyHostToDevice, c->stream));
    WHG_CUDA(c, cudaMemsetAsync(c->q_done, 0, sizeof(int) * (size_t)G, c->stream));
    WHG_CUDA(c, whg_launch_step_queue(c->st, c->bk, 2 * qs, c->opt.newton_terms, c->opt.gr_mode, q, c->stream));
    WHG_CUDA(c, cudaStreamSynchronize(c->stream));
    WHG_CUDA(c, cudaMemcpy(flag, c->q_err, sizeof(int), cudaMemcpyDeviceToHost));
    WHG_CUDA(c, cudaMemset(c->q_err, 0, sizeof(int)));
    return WHG_OK;
}

const char* whg_last_error(const whg_ctx* c) { return c ? c->err : g_create_err; }

}  // extern "C"

namespace {

// ---- adjoint scheduling ------------------------------------------------------
//
// The back kernels of consecutive segments form the adjoint's critical path,
// and at the ensemble sizes where the gradient is wanted (about a thousand
// systems) each of their warps runs alone on an SM sub-partition, at the rate
// one warp's dependency chains allow.  The tape kernels' warps, placed by the
// block scheduler on the same sub-partitions, halve that rate.  So, where the
// ensemble's warps fill at most half of the GPU at one warp per sub-partition,
// the SMs are split in two green contexts for the backward half: the back
// kernels run on the first (4 warps per block: one per sub-partition), the
// tape kernels on the second, and the two never share an SM.  The forward
// half's last two segments also run on the first partition while the second
// computes the first two tapes the backward half needs.  Optionally
// (a tape budget) the tapes of the segments already passed are recomputed
// during the forward half instead, into a pool of buffers; the forward half
// then runs on the first partition too.  That measured no faster at a
// thousand systems (the tape partition keeps up with the back kernels either
// way, and the forward half loses a little on fewer SMs), so it is off by
// default.  Results are bitwise the same under every schedule: every
// kernel's arithmetic is per warp.

// Driver entry points for green contexts, fetched through the runtime so that
// the library does not link the driver library.
struct GreenApi {
    PFN_cuDeviceGet_v2000 device_get = nullptr;
    PFN_cuDeviceGetDevResource_v12040 get_resource = nullptr;
    PFN_cuDevSmResourceSplitByCount_v12040 split = nullptr;
    PFN_cuDevResourceGenerateDesc_v12040 make_desc = nullptr;
    PFN_cuGreenCtxCreate_v12040 create = nullptr;
    PFN_cuGreenCtxDestroy_v12040 destroy = nullptr;
    PFN_cuCtxFromGreenCtx_v12040 as_ctx = nullptr;
    PFN_cuGreenCtxStreamCreate_v12050 stream_create = nullptr;
    PFN_cuStreamDestroy_v4000 stream_destroy = nullptr;
    PFN_cuCtxPushCurrent_v4000 push = nullptr;
    PFN_cuCtxPopCurrent_v4000 pop = nullptr;
    bool ok = false;
};

template <class F>
static bool driver_fn(const char* name, unsigned version, F* out)
{
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    void* p = nullptr;
    const cudaError_t e = cudaGetDriverEntryPointByVersion(name, &p, version, cudaEnableDefault, &q);
    if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !p) {
        cudaGetLastError();
        return false;
    }
    *out = reinterpret_cast<F>(p);
    return true;
}

static const GreenApi& green_api()
{
    static const GreenApi api = [] {
        GreenApi a;
        a.ok = driver_fn("cuDeviceGet", 2000, &a.device_get) &&
               driver_fn("cuDeviceGetDevResource", 12040, &a.get_resource) &&
               driver_fn("cuDevSmResourceSplitByCount", 12040, &a.split) &&
               driver_fn("cuDevResourceGenerateDesc", 12040, &a.make_desc) &&
               driver_fn("cuGreenCtxCreate", 12040, &a.create) &&
               driver_fn("cuGreenCtxDestroy", 12040, &a.destroy) &&
               driver_fn("cuCtxFromGreenCtx", 12040, &a.as_ctx) &&
               driver_fn("cuGreenCtxStreamCreate", 12050, &a.stream_create) &&
               driver_fn("cuStreamDestroy", 4000, &a.stream_destroy) &&
               driver_fn("cuCtxPushCurrent", 4000, &a.push) && driver_fn("cuCtxPopCurrent", 4000, &a.pop);
        return a;
    }();
    return api;
}

// Makes a green context current while work is issued into its streams (the
// runtime launches into the current context); a null context does nothing.
struct CtxScope {
    CUcontext ctx;
    bool ok;
    explicit CtxScope(CUcontext x) : ctx(x), ok(true)
    {
        if (ctx) ok = green_api().push(ctx) == CUDA_SUCCESS;
    }
    ~CtxScope()
    {
        CUcontext prev;
        if (ctx && ok) green_api().pop(&prev);
    }
};

#define WHG_SCOPE(ctx_, x)                                                              \
    CtxScope scope_##x(ctx_);                                                           \
    if (!scope_##x.ok) return fail(c, WHG_ECUDA, "cuCtxPushCurrent of a green context failed")

static void release_split(whg_ctx* c)
{
    const GreenApi& g = green_api();
    if (c->s_chain) g.stream_destroy((CUstream)c->s_chain);
    for (int i = 0; i < 2; ++i)
        if (c->s_tape[i]) g.stream_destroy((CUstream)c->s_tape[i]);
    if (c->g_chain) g.destroy(c->g_chain);
    if (c->g_tape) g.destroy(c->g_tape);
    c->s_chain = c->s_tape[0] = c->s_tape[1] = nullptr;
    c->g_chain = c->g_tape = nullptr;
    c->x_chain = c->x_tape = nullptr;
    c->chain_sms = c->tape_sms = 0;
}

// Green contexts of `want` SMs (rounded up to the partition granularity) and
// of the rest, with one stream in the first and two in the second.  Returns
// false, with no partition, where that is not possible.
static bool make_split(whg_ctx* c, int want)
{
    const GreenApi& g = green_api();
    if (!g.ok) return false;
    if (c->g_chain && c->chain_sms >= want && c->chain_sms < want + 8) return true;
    release_split(c);
    CUdevice dev = 0;
    if (g.device_get(&dev, c->device) != CUDA_SUCCESS) return false;
    CUdevResource all{}, part{}, rest{};
    if (g.get_resource(dev, &all, CU_DEV_RESOURCE_TYPE_SM) != CUDA_SUCCESS) return false;
    unsigned n = 1;
    if (g.split(&part, &n, &all, &rest, 0, (unsigned)want) != CUDA_SUCCESS || n != 1 ||
        rest.sm.smCount < 8)
        return false;
    CUdevResourceDesc dc = nullptr, dt = nullptr;
    bool ok = g.make_desc(&dc, &part, 1) == CUDA_SUCCESS && g.make_desc(&dt, &rest, 1) == CUDA_SUCCESS &&
              g.create(&c->g_chain, dc, dev, CU_GREEN_CTX_DEFAULT_STREAM) == CUDA_SUCCESS &&
              g.create(&c->g_tape, dt, dev, CU_GREEN_CTX_DEFAULT_STREAM) == CUDA_SUCCESS &&
              g.as_ctx(&c->x_chain, c->g_chain) == CUDA_SUCCESS && g.as_ctx(&c->x_tape, c->g_tape) == CUDA_SUCCESS;
    CUstream s0 = nullptr, s1 = nullptr, s2 = nullptr;
    ok = ok && g.stream_create(&s0, c->g_chain, CU_STREAM_NON_BLOCKING, 0) == CUDA_SUCCESS;
    c->s_chain = (cudaStream_t)s0;
    ok = ok && g.stream_create(&s1, c->g_tape, CU_STREAM_NON_BLOCKING, 0) == CUDA_SUCCESS;
    c->s_tape[0] = (cudaStream_t)s1;
    ok = ok && g.stream_create(&s2, c->g_tape, CU_STREAM_NON_BLOCKING, 0) == CUDA_SUCCESS;
    c->s_tape[1] = (cudaStream_t)s2;
    if (!ok) {
        release_split(c);
        return false;
    }
    c->chain_sms = (int)part.sm.smCount;
    c->tape_sms = (int)rest.sm.smCount;
    return true;
}

// Side streams and events of the adjoint (created on first use).
static int adjoint_streams(whg_ctx* c)
{
    if (c->side[0]) return WHG_OK;
    for (int i = 0; i < 2; ++i) WHG_CUDA(c, cudaStreamCreateWithFlags(&c->side[i], cudaStreamNonBlocking));
    WHG_CUDA(c, cudaEventCreateWithFlags(&c->ev_entry, cudaEventDisableTiming));
    WHG_CUDA(c, cudaEventCreateWithFlags(&c->ev_ckpt, cudaEventDisableTiming));
    WHG_CUDA(c, cudaEventCreateWithFlags(&c->ev_exit, cudaEventDisableTiming));
    return WHG_OK;
}

// nbuf tape buffers' events and bookkeeping (no segment held).
static int tape_pool(whg_ctx* c, int nbuf)
{
    while ((int)c->ev_tape.size() < nbuf) {
        cudaEvent_t a = nullptr, b = nullptr;
        WHG_CUDA(c, cudaEventCreateWithFlags(&a, cudaEventDisableTiming));
        c->ev_tape.push_back(a);
        WHG_CUDA(c, cudaEventCreateWithFlags(&b, cudaEventDisableTiming));
        c->ev_back.push_back(b);
    }
    c->tape_of.assign((size_t)nbuf, -1);
    c->adj_nbuf = nbuf;
    return WHG_OK;
}

static int segment_length(const whg_ctx* c, int seg)
{
    const long long s0 = (long long)seg * c->adj_K;
    return (int)(s0 + c->adj_K <= c->adj_n ? c->adj_K : c->adj_n - s0);
}

// Launch shapes: the chain (forward steps, checkpoints, loss, back kernels;
// on the first partition when `on_split`) and the tape kernels.
static WhgLaunch chain_cfg(const whg_ctx* c, bool on_split)
{
    WhgLaunch l = launch_cfg(c);
    if (on_split) {
        const long long threads = (long long)c->bk.warp0[c->bk.nb] * 32;
        l.block = 128;
        l.grid = (int)((threads + 127) / 128);
        if (l.grid < 1) l.grid = 1;
        l.stream = c->s_chain;
    }
    return l;
}

static WhgLaunch tape_cfg(const whg_ctx* c, int i)
{
    WhgLaunch l = launch_cfg(c);
    l.stream = c->split ? c->s_tape[i] : c->side[i];
    return l;
}

static int launch_tape(whg_ctx* c, const WhgAdj& a, int j, int i)
{
    const int b = j % c->adj_nbuf;
    const int rc = launch_check(c, whg_launch_adj_tape(c->st, c->bk, a, j, (long long)j * c->adj_K,
                                                       segment_length(c, j), b, c->opt.newton_terms,
                                                       c->opt.gr_mode, tape_cfg(c, i)),
                                "adjoint tape kernel");
    if (rc) return rc;
    c->tape_of[(size_t)b] = j;
    WHG_CUDA(c, cudaEventRecord(c->ev_tape[(size_t)b], tape_cfg(c, i).stream));
    return WHG_OK;
}

// Work issued on the context's stream so far comes before `s`.
static int enter_stream(whg_ctx* c, cudaStream_t s, CUcontext x)
{
    WHG_SCOPE(x, enter);
    WHG_CUDA(c, cudaStreamWaitEvent(s, c->ev_entry, 0));
    return WHG_OK;
}

// The context's stream waits for the work issued on `s`.
static int leave_stream(whg_ctx* c, cudaStream_t s, CUcontext x)
{
    {
        WHG_SCOPE(x, leave);
        WHG_CUDA(c, cudaEventRecord(c->ev_exit, s));
    }
    WHG_CUDA(c, cudaStreamWaitEvent(c->stream, c->ev_exit, 0));
    return WHG_OK;
}

// SMs wanted for the chain partition (0: no split) for this ensemble.
static int chain_sms_wanted(const whg_ctx* c)
{
    if (c->cfg_split == 0) return 0;
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    const int warps = c->bk.warp0[c->bk.nb];
    const int want = c->cfg_split > 0 ? c->cfg_split : (warps + 3) / 4;   // one warp per sub-partition
    if (c->cfg_split < 0 && 2 * want > sms) return 0;                      // the forward fills the GPU
    if (want >= sms) return 0;
    return want;
}

}  // namespace

extern "C" {

int whg_adjoint_schedule(whg_ctx* c, int sm_split, long long tape_bytes)
{
    if (!c) return WHG_EINVAL;
    if (sm_split < -1 || tape_bytes < -1)
        return fail(c, WHG_EINVAL, "sm_split=%d and tape_bytes=%lld must be >= -1", sm_split, tape_bytes);
    c->cfg_split = sm_split;
    c->cfg_tape_bytes = tape_bytes;
    return WHG_OK;
}

int whg_adjoint_layout(const whg_ctx* c, int* chain_sms, int* tape_sms, int* tape_buffers)
{
    if (!c) return WHG_EINVAL;
    if (chain_sms) *chain_sms = c->split ? c->chain_sms : 0;
    if (tape_sms) *tape_sms = c->split ? c->tape_sms : 0;
    if (tape_buffers) *tape_buffers = c->adj_nbuf;
    return WHG_OK;
}

int whg_adjoint_forward(whg_ctx* c, long long n_steps, int checkpoint_every, const double* target,
                        double* loss)
{
    if (!c) return WHG_EINVAL;
    if (!c->initialized || c->host_nstep != 0)
        return fail(c, WHG_ESTATE, "whg_adjoint_forward needs a freshly initialised context (no steps yet)");
    if (n_steps < 0 || checkpoint_every < 1)
        return fail(c, WHG_EINVAL, "need n_steps >= 0 and checkpoint_every >= 1");
    if (!target || !loss) return fail(c, WHG_EINVAL, "null target or loss");
    int rc = adjoint_streams(c);
    if (rc) return rc;
    const size_t NL = (size_t)c->bk.warp0[c->bk.nb] * 32;
    const long long nseg = (n_steps + checkpoint_every - 1) / checkpoint_every;
    const int K = (int)(n_steps < checkpoint_every ? (n_steps > 0 ? n_steps : 1) : checkpoint_every);
    const size_t tgt = (size_t)c->S * c->Nmax * 3;
    const size_t tape_len = (size_t)K * WHG_TAPE_W * NL;
    const size_t fixed = ((size_t)(nseg + 1) * 6 * NL + 8 * NL + tgt) * sizeof(double);
    const size_t tape_bytes = tape_len * sizeof(double);
    // the partition, then the tape pool: with the split and a tape budget, a
    // buffer per segment where they fit (half of the free memory, or the cap)
    const int want = chain_sms_wanted(c);
    c->split = want > 0 && make_split(c, want);
    const bool pre = c->split && c->cfg_tape_bytes != 0;   // tapes beside the forward half
    long long nbuf = WHG_TAPE_BUFFERS;
    if (pre) {
        size_t cap = 0;
        if (c->cfg_tape_bytes > 0) {
            cap = (size_t)c->cfg_tape_bytes;
        } else {
            size_t free_b = 0, total_b = 0;
            WHG_CUDA(c, cudaMemGetInfo(&free_b, &total_b));
            cap = (free_b + (c->adj_buf ? c->adj_bytes : 0)) / 2;
            cap = cap > fixed ? cap - fixed : 0;
        }
        const long long fit = (long long)(cap / tape_bytes);
        nbuf = fit < nseg ? fit : nseg;
        if (nbuf < WHG_TAPE_BUFFERS) nbuf = WHG_TAPE_BUFFERS;
    }
    const size_t bytes = fixed + (size_t)nbuf * tape_bytes;
    if (bytes > c->adj_bytes || (c->adj_bytes > 2 * bytes && c->adj_bytes - bytes > ((size_t)1 << 30))) {
        if (c->adj_buf) {
            WHG_CUDA(c, cudaStreamSynchronize(c->stream));
            cudaFree(c->adj_buf);
        }
        c->adj_buf = nullptr;
        c->adj_bytes = 0;
        cudaError_t e = cudaMalloc(&c->adj_buf, bytes);
        if (e != cudaSuccess) return fail(c, WHG_ENOMEM, "cudaMalloc(%zu) for the adjoint: %s", bytes,
                                          cudaGetErrorString(e));
        c->adj_bytes = bytes;
    }
    rc = tape_pool(c, (int)nbuf);
    if (rc) return rc;
    WhgAdj& a = c->adj;
    a = WhgAdj{};
    a.NL = NL;
    a.ckpt = c->adj_buf;
    a.tape = a.ckpt + (size_t)(nseg + 1) * 6 * NL;
    a.tape_len = tape_len;
    a.lam = a.tape + (size_t)nbuf * tape_len;
    double* tcopy = a.lam + 8 * NL;
    a.target = tcopy;
    c->adj_n = n_steps;
    c->adj_K = K;
    c->adj_nseg = (int)nseg;
    c->adj_ready = false;
    WHG_CUDA(c, cudaMemcpyAsync(tcopy, target, tgt * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
    // Segments whose tapes are recomputed beside the forward half: with a tape
    // budget all that have a buffer, else (split) the last nbuf - 1, which the
    // first back kernels need at once.  From segment `from` on, the forward
    // runs on the first partition, so that no tape kernel shares its SMs.
    const long long npre = !c->split ? 0 : pre ? (nbuf < nseg ? nbuf : nseg)
                                                : (nbuf - 1 < nseg ? nbuf - 1 : nseg);
    const long long first_pre = nseg - npre, from = pre ? 0 : first_pre;
    const CUcontext xt = c->split ? c->x_tape : nullptr;
    WhgLaunch l = chain_cfg(c, false);
    CUcontext xc = nullptr;
    bool switched = false;
    for (long long seg = 0; seg <= nseg; ++seg) {
        if (c->split && seg == from) {                  // onto the partition
            WHG_CUDA(c, cudaEventRecord(c->ev_entry, c->stream));
            for (cudaStream_t s : {c->s_chain, c->s_tape[0], c->s_tape[1]}) {
                rc = enter_stream(c, s, s == c->s_chain ? c->x_chain : xt);
                if (rc) return rc;
            }
            l = chain_cfg(c, true);
            xc = c->x_chain;
            switched = true;
        }
        {
            WHG_SCOPE(xc, save);
            rc = launch_check(c, whg_launch_adj_save(c->st, c->bk, a, (int)seg, l), "checkpoint kernel");
            if (rc) return rc;
            if (seg >= first_pre && seg < nseg) WHG_CUDA(c, cudaEventRecord(c->ev_ckpt, l.stream));
        }
        if (seg == nseg) break;
        if (seg >= first_pre) {
            WHG_SCOPE(xt, tape);
            const int i = (int)(seg % 2);
            WHG_CUDA(c, cudaStreamWaitEvent(c->s_tape[i], c->ev_ckpt, 0));
            rc = launch_tape(c, a, (int)seg, i);
            if (rc) return rc;
        }
        const long long k = (seg + 1) * checkpoint_every <= n_steps ? checkpoint_every
                                                                     : n_steps - seg * checkpoint_every;
        WHG_SCOPE(xc, steps);
        rc = step_impl(c, k, false, switched ? &l : nullptr);
        if (rc) return rc;
    }
    {
        WHG_SCOPE(xc, last);
        a.loss = loss;
        rc = launch_check(c, whg_launch_adj_loss(c->st, c->bk, a, 0, c->opt.newton_terms, l), "loss kernel");
        if (rc) return rc;
    }
    if (switched) {
        for (cudaStream_t s : {c->s_chain, c->s_tape[0], c->s_tape[1]}) {
            rc = leave_stream(c, s, s == c->s_chain ? c->x_chain : xt);
            if (rc) return rc;
        }
    }
    c->adj_ready = true;
    return WHG_OK;
}

int whg_adjoint_backward(whg_ctx* c, const double* loss_weight, double* grad_pos, double* grad_vel,
                         double* grad_mass)
{
    if (!c) return WHG_EINVAL;
    if (!c->adj_ready)
        return fail(c, WHG_ESTATE, "whg_adjoint_backward needs whg_adjoint_forward first (and no steps since)");
    WhgAdj a = c->adj;
    a.weight = loss_weight;
    a.gx = grad_pos;
    a.gu = grad_vel;
    a.gm = grad_mass;
    a.loss = nullptr;
    int rc = adjoint_streams(c);
    if (rc) return rc;
    const WhgLaunch l = chain_cfg(c, c->split);
    const CUcontext xc = c->split ? c->x_chain : nullptr, xt = c->split ? c->x_tape : nullptr;
    const cudaStream_t ts[2] = {tape_cfg(c, 0).stream, tape_cfg(c, 1).stream};
    // every stream starts after everything issued so far (checkpoints, tapes
    // of the forward half, earlier backward halves)
    WHG_CUDA(c, cudaEventRecord(c->ev_entry, c->stream));
    if (c->split) {
        rc = enter_stream(c, l.stream, xc);
        if (rc) return rc;
    }
    for (int i = 0; i < 2; ++i) {
        rc = enter_stream(c, ts[i], xt);
        if (rc) return rc;
    }
    {
        WHG_SCOPE(xc, start);
        rc = launch_check(c, whg_launch_adj_loss(c->st, c->bk, a, 1, c->opt.newton_terms, l), "adjoint start");
        if (rc) return rc;
    }
    // The products of segment s run on the chain stream (the critical path).
    // Segment j's tape lives in buffer j % nbuf; a tape not already there is
    // recomputed on a tape stream nbuf - 1 segments ahead, once the products
    // of segment j + nbuf are done with the buffer.
    const int nseg = c->adj_nseg, nbuf = c->adj_nbuf;
    std::vector<char> fresh((size_t)nbuf, 0);
    auto need_tape = [&](int j, bool after_back) -> int {
        const int b = j % nbuf;
        if (c->tape_of[(size_t)b] == j) return WHG_OK;
        WHG_SCOPE(xt, tape);
        const int i = j % 2;
        if (after_back && j + nbuf <= nseg - 1) WHG_CUDA(c, cudaStreamWaitEvent(ts[i], c->ev_back[(size_t)b], 0));
        const int r = launch_tape(c, a, j, i);
        if (r) return r;
        fresh[(size_t)b] = 1;
        return WHG_OK;
    };
    for (int j = nseg - 1; j >= 0 && j > nseg - nbuf; --j) {
        rc = need_tape(j, false);
        if (rc) return rc;
    }
    for (int seg = nseg - 1; seg >= 0; --seg) {
        const int j = seg - (nbuf - 1);
        if (j >= 0) {
            rc = need_tape(j, true);
            if (rc) return rc;
        }
        const int b = seg % nbuf;
        WHG_SCOPE(xc, back);
        if (fresh[(size_t)b]) WHG_CUDA(c, cudaStreamWaitEvent(l.stream, c->ev_tape[(size_t)b], 0));
        fresh[(size_t)b] = 0;
        rc = launch_check(c, whg_launch_adj_back(c->st, c->bk, a, (long long)seg * c->adj_K,
                                                 segment_length(c, seg), b, c->opt.newton_terms,
                                                 c->opt.gr_mode, l),
                          "adjoint back kernel");
        if (rc) return rc;
        WHG_CUDA(c, cudaEventRecord(c->ev_back[(size_t)b], l.stream));
    }
    {
        WHG_SCOPE(xc, finish);
        rc = launch_check(c, whg_launch_adj_finish(c->st, c->bk, a, l), "adjoint finish kernel");
        if (rc) return rc;
    }
    if (c->split) {
        rc = leave_stream(c, l.stream, xc);
        if (rc) return rc;
    }
    for (int i = 0; i < 2; ++i) {
        rc = leave_stream(c, ts[i], xt);
        if (rc) return rc;
    }
    return WHG_OK;
}

void whg_destroy(whg_ctx* c)
{
    if (!c) return;
    cudaStreamSynchronize(c->stream);
    if (c->g_chain) {
        {
            CtxScope sc(c->x_chain);
            if (sc.ok) cudaStreamSynchronize(c->s_chain);
        }
        {
            CtxScope sc(c->x_tape);
            if (sc.ok)
                for (int i = 0; i < 2; ++i) cudaStreamSynchronize(c->s_tape[i]);
        }
        release_split(c);
    }
    cudaFree(c->st.m);
    cudaFree(c->stage_d);
    if (c->repack_buf) cudaFree(c->repack_buf);
    if (c->q_next) cudaFree(c->q_next);
    if (c->st.dbg) cudaFree(c->st.dbg);
    if (c->adj_buf) cudaFree(c->adj_buf);
    if (c->side[0]) {
        for (int i = 0; i < 2; ++i) cudaStreamSynchronize(c->side[i]);
        for (size_t i = 0; i < c->ev_tape.size(); ++i) {
            cudaEventDestroy(c->ev_tape[i]);
            cudaEventDestroy(c->ev_back[i]);
        }
        cudaEventDestroy(c->ev_entry);
        cudaEventDestroy(c->ev_ckpt);
        cudaEventDestroy(c->ev_exit);
        for (int i = 0; i < 2; ++i) cudaStreamDestroy(c->side[i]);
    }
    if (c->graph) cudaGraphExecDestroy(c->graph);
    if (c->capture) cudaStreamDestroy(c->capture);
    delete c;
}

}  // extern "C"
