// whg_internal.h -- structures shared by the host API and the kernels of libwhg.
#pragma once

#include <cuda_runtime.h>

#include "../../include/whg.h"

// Device-resident ensemble state (structure of arrays).
//
// Lane arrays hold one value per (system, lane), index s * G + p, with G lanes
// per system and lane p carrying planet p.  Lanes p >= n_planets[s] are
// padding: mass 0, parked far from the star and never updated.  Systems
// s >= S (up to S_pad, a multiple of the systems in one block) are padding too.
struct WhgState {
    double* m;                       // planet mass
    double *qx, *qy, *qz;            // heliocentric position Q (Sec. 3.1)
    double *vx, *vy, *vz;            // barycentric velocity v = P / m
    double* m0;                      // [S_pad] star mass (mu = G m0, G = 1)
    double* dt;                      // [S_pad]
    double* M;                       // [S_pad] total mass
    double* xcm;                     // [3][S_pad] barycentre position at t = 0
    double* vcm;                     // [3][S_pad] barycentre velocity
    int* nplan;                      // [S_pad] planets per system
    int* status;                     // [S_pad] WHG_STATUS_* bits; non-zero = frozen
    long long* nstep;                // [S_pad] completed steps (0 = synchronized)
    int S, S_pad, Nmax;
    double c_light;
};

// Inertial-frame inputs (layouts of whg.h).
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

struct WhgLaunch {
    int grid, block;
    cudaStream_t stream;
};

// One launcher table per lanes-per-system value G (whg_kernels_g{1,2,4,8}.cu).
struct WhgKernels {
    cudaError_t (*init)(const WhgState&, const WhgIn&, const WhgLaunch&);
    cudaError_t (*step)(const WhgState&, long long nsteps, int newton_terms, int gr_mode,
                        const WhgLaunch&);
    cudaError_t (*read)(const WhgState&, const WhgOut&, int newton_terms, const WhgLaunch&);
    cudaError_t (*energy)(const WhgState&, const WhgOut&, int newton_terms, int gr_mode,
                          const WhgLaunch&);
    cudaError_t (*raw)(const WhgState&, const WhgOut&, int set, const WhgLaunch&);
};

extern const WhgKernels whg_kernels_g1;
extern const WhgKernels whg_kernels_g2;
extern const WhgKernels whg_kernels_g4;
extern const WhgKernels whg_kernels_g8;

#define WHG_MAX_BLOCK 256

// Record the message returned by whg_last_error(NULL) for calls without a context.
void whg_record_error(const char* msg);
