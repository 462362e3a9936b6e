// whg_internal.h -- structures shared by the host API and the kernels of libwhg.
#pragma once

#include <cuda_runtime.h>

#include "../../include/whg.h"

// Device-resident ensemble state (structure of arrays).
//
// Systems are grouped into buckets of equal lanes-per-system L (1..8); a warp
// of a bucket holds floor(32 / L) systems, lane p of a system carrying planet
// p.  Lane arrays have one entry per lane of every warp (index warp * 32 +
// lane), including lanes that hold no system and padding lanes of systems
// with fewer than L planets: those carry mass 0, are parked far from the star
// and are never updated.  Per-system arrays are indexed by the internal
// system index (bucket by bucket); perm maps it to the caller's index.
struct WhgState {
    double* m;                       // planet mass
    double *qx, *qy, *qz;            // heliocentric position Q (Sec. 3.1)
    double *vx, *vy, *vz;            // barycentric velocity v = P / m
    double* a0;                      // initial osculating semi-major axis (stop rules)
    double* m0;                      // [S] star mass (mu = G m0, G = 1)
    double* dt;                      // [S]
    double* M;                       // [S] total mass
    double* xcm;                     // [3][S] barycentre position at t = 0
    double* vcm;                     // [3][S] barycentre velocity
    double* rej2;                    // [S] squared ejection distance (+inf = rule off)
    int* nplan;                      // [S] planets per system
    int* status;                     // [S] WHG_STATUS_* bits; non-zero = frozen
    int* perm;                       // [S] caller's index of each internal system (null = identity)
    long long* nstep;                // [S] completed steps (0 = synchronized)
    int S, Nmax;
    double c_light;
    double hill;                     // close-encounter rule: mutual Hill radii (0 = off)
    double eject;                    // ejection rule: factor on the largest initial a (0 = off)
    int merge;                       // one J(dt) before I(dt) (GR off only)
    int halley32;                    // Kepler solver: initial guess and Halley phase in FP32
    int full_rotation;               // interaction: all L-1 rotations, no third-law reactions
    long long nl;                    // lane capacity of the lane arrays
    unsigned* dbg;                   // bounds-check flag word (debug builds only, else null)
};

// Index checks of the debug build (-DWHG_DEBUG_BOUNDS; the stand-in for a
// memory checker): a failed check sets a bit of *st.dbg, never traps.  The
// release build compiles them away.
#define WHG_BOUND_LANE 1u          // lane index outside the lane arrays
#define WHG_BOUND_SYSTEM 2u        // internal system index outside 0..S-1
#define WHG_BOUND_USER 4u          // caller's system index (perm) outside 0..S-1
#define WHG_BOUND_BUCKET 8u        // bucket index outside 0..nb-1
#define WHG_BOUND_REPACK 16u       // repack order outside the bucket
#define WHG_BOUND_QUEUE 32u        // work-queue unit outside the warp-groups
#ifdef WHG_DEBUG_BOUNDS
#define WHG_CHECK(st, cond, bit)                                  \
    do {                                                          \
        if (!(cond)) atomicOr((st).dbg, (bit));                   \
    } while (0)
#else
#define WHG_CHECK(st, cond, bit) ((void)0)
#endif

// Work-queue control of k_step_queue (device pointers; next and done zeroed
// before each launch).
struct WhgQueue {
    unsigned long long* next;        // unit counter
    int* done;                       // [warp-groups] chunks completed
    int* err;                        // set to 1 when a wait gave up
    long long chunk;                 // steps per unit
    int units;                       // units per warp-group
    long long spin_limit;            // polls before a wait gives up
};

// Bucket table (by value in every launch).
struct WhgBuckets {
    int nb;                          // number of buckets, 1..8
    int L[8];                        // lanes per system of bucket b
    int warp0[9];                    // first warp of bucket b; warp0[nb] = warps in use
    int sys0[9];                     // first internal system of bucket b; sys0[nb] = S
};

// Inertial-frame inputs (layouts of whg.h), in the caller's system order.
struct WhgIn {
    const double* masses;
    const double* pos;
    const double* vel;
    const int* nplan;                // may be null: every system has Nmax planets
    const double* dt;
};

// Outputs of the read / energy / raw kernels (any pointer may be null).
struct WhgOut {
    double* pos;
    double* vel;
    int* status;
    double* t;
    double* E;
    double* rawQ;
    double* rawv;
    long long* rawn;
    const double* inQ;               // raw set inputs
    const double* inv;
    const long long* inn;
    const int* ins;
};

// Buffers of the adjoint (reverse-mode) pass; NL = lanes of the layout.
// Doubles per lane and step on the adjoint's tape (layout in whg_adjoint.cu).
#define WHG_TAPE_W 74
// Tape buffers at least (and without the SM split): segments s-1 and s-2 are
// recomputed while the products of segment s run.  Segment j uses buffer
// j mod (number of buffers).
#define WHG_TAPE_BUFFERS 3

struct WhgAdj {
    double* ckpt;                    // [nseg + 1][6][NL] state every K steps
    double* tape;                    // [buffers][K][WHG_TAPE_W][NL] per-step values of a segment
    size_t tape_len;                 // K * WHG_TAPE_W * NL (one buffer)
    double* lam;                     // [8][NL] adjoints: Q (3), v (3), m, m0 (partial)
    const double* target;            // [S][Nmax][3] caller order
    double* loss;                    // [S] caller order
    const double* weight;            // [S] dTotal/dL_s (null = 1)
    double* gx;                      // [S][1+Nmax][3] gradients, caller layout
    double* gu;
    double* gm;                      // [S][1+Nmax]
    size_t NL;
};

struct WhgLaunch {
    int grid, block;
    cudaStream_t stream;
};

// Kernel launchers (whg_kernels_common.cu, whg_kernels_nt6.cu, whg_kernels_nt8.cu).
cudaError_t whg_launch_init(const WhgState&, const WhgBuckets&, const WhgIn&, const WhgLaunch&);
// Repack (live systems first in every bucket) into `scratch` (same layout as
// st; order: S ints of scratch space); the caller copies scratch back.
cudaError_t whg_launch_repack(const WhgState& st, const WhgState& scratch, const WhgBuckets& bk, int* order,
                              cudaStream_t stream);
cudaError_t whg_launch_raw(const WhgState&, const WhgBuckets&, const WhgOut&, int set, const WhgLaunch&);
cudaError_t whg_launch_step(const WhgState&, const WhgBuckets&, long long nsteps, int newton_terms,
                            int gr_mode, const WhgLaunch&);
// Step kernel over the work queue (q.next and q.done zeroed by the caller).
cudaError_t whg_launch_step_queue(const WhgState&, const WhgBuckets&, long long nsteps, int newton_terms,
                                  int gr_mode, const WhgQueue& q, cudaStream_t stream);
cudaError_t whg_launch_read(const WhgState&, const WhgBuckets&, const WhgOut&, int newton_terms,
                            const WhgLaunch&);
cudaError_t whg_launch_energy(const WhgState&, const WhgBuckets&, const WhgOut&, int newton_terms,
                              int gr_mode, const WhgLaunch&);
cudaError_t whg_launch_step_nt6(const WhgState&, const WhgBuckets&, long long, int, const WhgLaunch&);
cudaError_t whg_launch_step_nt8(const WhgState&, const WhgBuckets&, long long, int, const WhgLaunch&);
cudaError_t whg_launch_step_queue_nt6(const WhgState&, const WhgBuckets&, long long, int, const WhgQueue&,
                                      cudaStream_t);
cudaError_t whg_launch_step_queue_nt8(const WhgState&, const WhgBuckets&, long long, int, const WhgQueue&,
                                      cudaStream_t);
cudaError_t whg_launch_read_nt6(const WhgState&, const WhgBuckets&, const WhgOut&, const WhgLaunch&);
cudaError_t whg_launch_read_nt8(const WhgState&, const WhgBuckets&, const WhgOut&, const WhgLaunch&);
cudaError_t whg_launch_energy_nt6(const WhgState&, const WhgBuckets&, const WhgOut&, int, const WhgLaunch&);
cudaError_t whg_launch_energy_nt8(const WhgState&, const WhgBuckets&, const WhgOut&, int, const WhgLaunch&);

cudaError_t whg_launch_adj_save(const WhgState&, const WhgBuckets&, const WhgAdj&, int slot, const WhgLaunch&);
cudaError_t whg_launch_adj_loss(const WhgState&, const WhgBuckets&, const WhgAdj&, int start, int newton_terms,
                                const WhgLaunch&);
cudaError_t whg_launch_adj_tape(const WhgState&, const WhgBuckets&, const WhgAdj&, int seg, long long s0,
                                int nk, int buf, int newton_terms, int gr_mode, const WhgLaunch&);
cudaError_t whg_launch_adj_back(const WhgState&, const WhgBuckets&, const WhgAdj&, long long s0, int nk,
                                int buf, int newton_terms, int gr_mode, const WhgLaunch&);
cudaError_t whg_launch_adj_finish(const WhgState&, const WhgBuckets&, const WhgAdj&, const WhgLaunch&);

// Lanes per system used for a bucket of n-planet systems in the packed layout.
inline int whg_lanes_for_planets(int n) { return n == 7 ? 8 : n; }

#define WHG_MAX_BLOCK 256

// Record the message returned by whg_last_error(NULL) for calls without a context.
void whg_record_error(const char* msg);
