// whg_device.cuh -- device code of libwhg: FP64 special functions, the
// Wisdom-Holman sub-steps and the kernels, templated on the number G of warp
// lanes per system (one lane per planet, G in {1, 2, 4, 8}).
//
// GB300 design notes.  The whole step is FP64 arithmetic on a few registers
// per lane; on this part the FP64 pipe retires about 2 lanes per clock per SM
// while FP32, integer, shuffle and MUFU work retire tens of times faster.  So
// the step is bound by the number of FP64 instructions alone, and the code
// spends integer and FP32 work freely to save FP64 instructions:
//   * reciprocals and reciprocal square roots start from the FP32 hardware
//     approximation of a mantissa built with integer operations and take one
//     third-order FP64 refinement (3 and 5 FP64 instructions);
//   * the all-pairs interaction uses Newton's third law (Sec. 3.3), with
//     partner schedules that suit warp shuffles rather than AVX512 lanes;
//   * cross-lane sums are xor butterflies over the system's lanes (Sec. 3.4),
//     so every lane gets the bitwise-identical total.
// State stays in registers for the whole launch; HBM is touched only at load
// and store (coalesced: consecutive lanes read consecutive doubles).
#pragma once

#include <stdint.h>

#include "whg_internal.h"

#define WHG_FULL_MASK 0xffffffffu

namespace whg {

// ------------------------------------------------------------------------
// FP64 reciprocal and reciprocal square root.
//
// Method: Newton-Raphson / Householder iteration for f(y) = 1/y - x (resp.
// 1/y^2 - x) from a low-precision seed (e.g. Muller et al., Handbook of
// Floating-Point Arithmetic, ch. on Newton-Raphson-based division).  The seed
// y0 comes from the PTX instructions rcp.approx / rsqrt.approx on an FP32 copy
// of the mantissa (|y0 x - 1| < 2^-21), the exponent being handled with
// integer arithmetic so that every normal double works.  With e = 1 - x y0
// (resp. e = 1 - x y0^2) the third-order steps are
//     1/x       = y0 (1 + e + e^2 + ...)          ->  y0 + y0 (e + e^2)
//     1/sqrt(x) = y0 (1 + e/2 + 3e^2/8 + ...)     ->  y0 + y0 e (1/2 + 3e/8)
// whose truncation error (~e^3 < 2^-63) is far below double rounding; results
// are within about one ulp of the exact value.

__device__ __forceinline__ float approx_rcp_f32(float x)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

__device__ __forceinline__ float approx_rsqrt_f32(float x)
{
    float r;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// 1/x for finite normal x (either sign).
__device__ __forceinline__ double rcp(double x)
{
    const unsigned hi = (unsigned)__double2hiint(x);
    const unsigned lo = (unsigned)__double2loint(x);
    const int ex = (int)((hi >> 20) & 0x7ffu);                         // biased exponent
    const float mant = __uint_as_float(0x3f800000u | ((hi & 0x000fffffu) << 3) | (lo >> 29));
    const unsigned rb = __float_as_uint(approx_rcp_f32(mant));          // in (0.5, 1]
    const int dex = (int)((rb >> 23) & 0xffu) - 127 + 2046 - ex;        // biased exponent of 1/x
    const unsigned yhi = (hi & 0x80000000u) | ((unsigned)dex << 20) | ((rb >> 3) & 0x000fffffu);
    const double y = __hiloint2double((int)yhi, (int)(rb << 29));
    const double e = fma(-x, y, 1.0);
    return fma(y, fma(e, e, e), y);
}

// 1/sqrt(x) for finite normal x > 0.
__device__ __forceinline__ double rsqrt(double x)
{
    const unsigned hi = (unsigned)__double2hiint(x);
    const unsigned lo = (unsigned)__double2loint(x);
    const int ex = (int)((hi >> 20) & 0x7ffu) - 1023;                  // unbiased exponent
    const int odd = ex & 1;
    const int half = (ex - odd) / 2;                                   // x = 4^half * mant
    const float mant = __uint_as_float(((unsigned)(127 + odd) << 23) | ((hi & 0x000fffffu) << 3) |
                                       (lo >> 29));                    // in [1, 4)
    const unsigned rb = __float_as_uint(approx_rsqrt_f32(mant));       // in (0.5, 1]
    const int dex = (int)((rb >> 23) & 0xffu) - 127 - half + 1023;
    const double y = __hiloint2double((int)(((unsigned)dex << 20) | ((rb >> 3) & 0x000fffffu)),
                                      (int)(rb << 29));
    const double e = fma(-x, y * y, 1.0);
    return fma(y * e, fma(0.375, e, 0.5), y);
}

// x^(-3/2) for finite normal x > 0 (the 1/r^3 of a pair from r^2), straight
// from the rsqrt seed: x^(-3/2) = y0^3 (1 - e)^(-3/2) = y0^3 (1 + 3e/2 + 15e^2/8 + ...)
// with e = 1 - x y0^2; truncation ~ (35/16) e^3 < 2^-61.
__device__ __forceinline__ double rsqrt_cubed(double x)
{
    const unsigned hi = (unsigned)__double2hiint(x);
    const unsigned lo = (unsigned)__double2loint(x);
    const int ex = (int)((hi >> 20) & 0x7ffu) - 1023;
    const int odd = ex & 1;
    const int half = (ex - odd) / 2;
    const float mant = __uint_as_float(((unsigned)(127 + odd) << 23) | ((hi & 0x000fffffu) << 3) |
                                       (lo >> 29));
    const unsigned rb = __float_as_uint(approx_rsqrt_f32(mant));
    const int dex = (int)((rb >> 23) & 0xffu) - 127 - half + 1023;
    const double y = __hiloint2double((int)(((unsigned)dex << 20) | ((rb >> 3) & 0x000fffffu)),
                                      (int)(rb << 29));
    const double y2 = y * y;
    const double e = fma(-x, y2, 1.0);
    const double y3 = y2 * y;
    return fma(y3 * e, fma(1.875, e, 1.5), y3);
}

__device__ __forceinline__ bool is_finite(double x)
{
    return (__double2hiint(x) & 0x7ff00000) != 0x7ff00000;
}

// ------------------------------------------------------------------------
// Stumpff functions c_2(z), c_3(z) by their Taylor series truncated after T
// terms, c_n(z) = sum_{k<T} (-z)^k / (n+2k)! (Sec. 3.2: series with a table of
// coefficients, no quarter-angle reduction).  The coefficients 1/k! are
// compile-time constants: k! is exact in double for k <= 22, and the compiler
// rounds 1/k! once.

template <int N>
struct Factorial {
    static constexpr double value = N * Factorial<N - 1>::value;
};
template <>
struct Factorial<0> {
    static constexpr double value = 1.0;
};

template <int K>
struct StumpffHorner {            // folds in the terms K, K-1, ..., 0
    static __device__ __forceinline__ void run(double z, double& c2, double& c3)
    {
        c2 = fma(-z, c2, 1.0 / Factorial<2 * K + 2>::value);
        c3 = fma(-z, c3, 1.0 / Factorial<2 * K + 3>::value);
        StumpffHorner<K - 1>::run(z, c2, c3);
    }
};
template <>
struct StumpffHorner<-1> {
    static __device__ __forceinline__ void run(double, double&, double&) {}
};

template <int T>
__device__ __forceinline__ void stumpff_c2c3(double z, double& c2, double& c3)
{
    c2 = 1.0 / Factorial<2 * T>::value;          // term k = T-1
    c3 = 1.0 / Factorial<2 * T + 1>::value;
    StumpffHorner<T - 2>::run(z, c2, c3);
}


// ------------------------------------------------------------------------
// Kepler drift of one planet for time h under H_K,i (Sec. 3.2, Eq. 3),
// mu = G m0.  Universal variable X solves Kepler's equation
//     F(X)  = r0 G1 + eta0 G2 + mu G3 - h = r0 X + eta0 G2 + zeta0 G3 - h = 0,
//     F'(X) = r = r0 + eta0 X + zeta0 G2 - beta eta0 G3,
//     F''   = eta0 + zeta0 X - beta eta0 G2 - beta zeta0 G3
// (the second forms use G0 = 1 - beta G2, G1 = X - beta G3 and
// zeta0 = mu - beta r0, so only the c2 and c3 series are needed): initial
// guess h/r0 - eta0 h^2 / (2 r0^3), 2 Halley steps with 4-term series, 2 Newton
// steps with NT-term series.  The G_n at the final X = X1 + d come from the
// values at the last Newton point X1 by one Taylor step (dG_n/dX = G_{n-1});
// |d| is the last Newton correction, so the neglected d^2 terms are far below
// rounding.  Then the Lagrange f - 1, g, fdot, gdot - 1.  No branches.
// Returns beta > 0.
template <int NT>
__device__ __forceinline__ bool kepler_drift(double mu, double h, double& qx, double& qy,
                                             double& qz, double& vx, double& vy, double& vz)
{
    const double r0sq = fma(qx, qx, fma(qy, qy, qz * qz));
    const double r0i = rsqrt(r0sq);
    const double r0 = r0sq * r0i;
    const double eta0 = fma(qx, vx, fma(qy, vy, qz * vz));
    const double v2 = fma(vx, vx, fma(vy, vy, vz * vz));
    const double beta = fma(2.0 * mu, r0i, -v2);
    const double zeta0 = fma(-beta, r0, mu);
    const double beta_eta0 = beta * eta0, beta_zeta0 = beta * zeta0;
    const double hr = h * r0i;
    double X = fma(-0.5 * eta0 * hr * hr, r0i, hr);
    double X2, c2, c3, G2, G3;
#pragma unroll
    for (int it = 0; it < 2; ++it) {                 // Halley
        X2 = X * X;
        stumpff_c2c3<4>(beta * X2, c2, c3);
        G2 = X2 * c2;
        G3 = (X2 * X) * c3;
        const double F = fma(r0, X, fma(eta0, G2, fma(zeta0, G3, -h)));
        const double Fp = fma(zeta0, G2, fma(-beta_eta0, G3, fma(eta0, X, r0)));
        const double Fpp = fma(-beta_zeta0, G3, fma(-beta_eta0, G2, fma(zeta0, X, eta0)));
        const double den = fma(-0.5 * F, Fpp, Fp * Fp);          // (2F'^2 - F F'') / 2
        X = fma(-(F * Fp), rcp(den), X);
    }
    double d = 0.0;
#pragma unroll
    for (int it = 0; it < 2; ++it) {                 // Newton
        X = X + d;
        X2 = X * X;
        stumpff_c2c3<NT>(beta * X2, c2, c3);
        G2 = X2 * c2;
        G3 = (X2 * X) * c3;
        const double F = fma(r0, X, fma(eta0, G2, fma(zeta0, G3, -h)));
        const double Fp = fma(zeta0, G2, fma(-beta_eta0, G3, fma(eta0, X, r0)));
        d = -F * rcp(Fp);
    }
    // G at the final X + d from the last Newton point X.
    const double G1 = fma(-beta, G3, X);
    const double G0 = fma(-beta, G2, 1.0);
    const double Xf = X + d;
    const double G3f = fma(d, G2, G3);
    const double G2f = fma(d, G1, G2);
    const double G1f = fma(d, G0, G1);
    const double r = fma(zeta0, G2f, fma(-beta_eta0, G3f, fma(eta0, Xf, r0)));
    const double ri = rcp(r);
    const double mr0 = mu * r0i;
    const double fm1 = -mr0 * G2f;                   // f - 1
    const double g = fma(-mu, G3f, h);
    const double fd = -(mr0 * ri) * G1f;
    const double gdm1 = -(mu * ri) * G2f;            // gdot - 1
    const double nqx = fma(fm1, qx, fma(g, vx, qx));
    const double nqy = fma(fm1, qy, fma(g, vy, qy));
    const double nqz = fma(fm1, qz, fma(g, vz, qz));
    vx = fma(fd, qx, fma(gdm1, vx, vx));
    vy = fma(fd, qy, fma(gdm1, vy, vy));
    vz = fma(fd, qz, fma(gdm1, vz, vz));
    qx = nqx; qy = nqy; qz = nqz;
    return beta > 0.0;
}

// Sum of x over the G lanes of this system (xor butterfly, Sec. 3.4); every
// lane receives the same bits because each level adds a commuting pair.
template <int G>
__device__ __forceinline__ double group_sum(double x)
{
#pragma unroll
    for (int o = 1; o < G; o <<= 1) x += __shfl_xor_sync(WHG_FULL_MASK, x, o, G);
    return x;
}

// Jump step (Sec. 3.4, Eq. 6): Q_i += (h/m0) sum_j m_j v_j; jc = h / m0.
template <int G>
__device__ __forceinline__ void jump(double m, double jc, double vx, double vy, double vz,
                                     double& qx, double& qy, double& qz)
{
    const double px = group_sum<G>(m * vx);
    const double py = group_sum<G>(m * vy);
    const double pz = group_sum<G>(m * vz);
    qx = fma(jc, px, qx);
    qy = fma(jc, py, qy);
    qz = fma(jc, pz, qz);
}

// Interaction kick (Sec. 3.3, Eq. 5) plus the GR term, for time dt, added
// straight into v.  hm = dt m_i.  Pairs at cyclic lane distance k < G/2 are
// evaluated once, by the lower lane of the pair, and the reaction is passed to
// the partner by a shuffle (Newton's third law); the G/2 pairs at distance G/2
// are evaluated by both of their lanes.  For G = 8 that is 4 reciprocal square
// roots per lane for the 28 pairs, as in the paper, but with rotations that
// cost the same on any lane pair of a warp.
template <int G, int GRM>
__device__ __forceinline__ void kick(int p, double qx, double qy, double qz, double hm,
                                     double mrat, double kgr, double& vx, double& vy, double& vz)
{
#pragma unroll
    for (int k = 1; k < G / 2; ++k) {
        const int to = (p + k) & (G - 1);
        const int from = (p - k) & (G - 1);
        const double dx = __shfl_sync(WHG_FULL_MASK, qx, to, G) - qx;   // Q_j - Q_i
        const double dy = __shfl_sync(WHG_FULL_MASK, qy, to, G) - qy;
        const double dz = __shfl_sync(WHG_FULL_MASK, qz, to, G) - qz;
        const double hmj = __shfl_sync(WHG_FULL_MASK, hm, to, G);
        const double r3 = rsqrt_cubed(fma(dx, dx, fma(dy, dy, dz * dz)));
        const double sj = hmj * r3;
        vx = fma(sj, dx, vx);
        vy = fma(sj, dy, vy);
        vz = fma(sj, dz, vz);
        const double si = hm * r3;                    // reaction on j: -si (Q_j - Q_i)
        const double ex = __shfl_sync(WHG_FULL_MASK, dx, from, G);
        const double ey = __shfl_sync(WHG_FULL_MASK, dy, from, G);
        const double ez = __shfl_sync(WHG_FULL_MASK, dz, from, G);
        const double es = __shfl_sync(WHG_FULL_MASK, si, from, G);
        vx = fma(-es, ex, vx);
        vy = fma(-es, ey, vy);
        vz = fma(-es, ez, vz);
    }
    if (G >= 2) {
        const int to = p ^ (G / 2);
        const double dx = __shfl_sync(WHG_FULL_MASK, qx, to, G) - qx;
        const double dy = __shfl_sync(WHG_FULL_MASK, qy, to, G) - qy;
        const double dz = __shfl_sync(WHG_FULL_MASK, qz, to, G) - qz;
        const double hmj = __shfl_sync(WHG_FULL_MASK, hm, to, G);
        const double sj = hmj * rsqrt_cubed(fma(dx, dx, fma(dy, dy, dz * dz)));
        vx = fma(sj, dx, vx);
        vy = fma(sj, dy, vy);
        vz = fma(sj, dz, vz);
    }
    if (GRM != 0) {
        // a_GR(Q) = -6 (G m0)^2 Q / (c^2 |Q|^4); kgr = -6 m0^2 dt / c^2.
        const double ri2 = rcp(fma(qx, qx, fma(qy, qy, qz * qz)));
        const double c = kgr * (ri2 * ri2);
        if (GRM == 1) {
            vx = fma(c, qx, vx);
            vy = fma(c, qy, vy);
            vz = fma(c, qz, vz);
        } else {
            const double ax = c * qx, ay = c * qy, az = c * qz;
            const double bx = group_sum<G>(mrat * ax);
            const double by = group_sum<G>(mrat * ay);
            const double bz = group_sum<G>(mrat * az);
            vx = vx + (ax - bx);
            vy = vy + (ay - by);
            vz = vz + (az - bz);
        }
    }
}

// Lane mask of the G lanes of this thread's system inside its warp.
template <int G>
__device__ __forceinline__ unsigned group_mask()
{
    const unsigned base = (threadIdx.x & 31u) & ~(unsigned)(G - 1);
    return (G == 32 ? WHG_FULL_MASK : ((1u << G) - 1u)) << base;
}

// Far-away parking spot of padding lanes: distinct, finite, never updated.
__device__ __forceinline__ double parked_x(int p) { return 1.0e6 * (double)(p + 1); }

// ------------------------------------------------------------------------
// Kernels.  The grid covers exactly S_pad * G threads; thread t is lane
// t % G of system t / G.  Shuffles use the full warp mask, so no thread
// returns before the last shuffle.

template <int G>
__global__ void __launch_bounds__(WHG_MAX_BLOCK) k_init(WhgState st, WhgIn in)
{
    const int tid = blockIdx.x * blockDim.x + threadIdx.x;
    const int s = tid / G, p = tid & (G - 1);
    if (s >= st.S_pad) return;
    const size_t lane = (size_t)s * G + p;
    const int B = 1 + st.Nmax;
    int n = 0, ok = 0;
    double mm = 0.0, M = 0.0, xc[3] = {0.0, 0.0, 0.0}, vc[3] = {0.0, 0.0, 0.0}, m0 = 1.0, dt = 1.0;
    if (s < st.S) {
        const double* ms = in.masses + (size_t)s * B;
        const double* xs = in.pos + (size_t)s * B * 3;
        const double* us = in.vel + (size_t)s * B * 3;
        n = in.nplan ? in.nplan[s] : st.Nmax;
        dt = in.dt[s];
        m0 = ms[0];
        ok = n >= 1 && n <= st.Nmax && dt > 0.0 && is_finite(dt) && m0 > 0.0 && is_finite(m0);
        if (ok) {
            for (int k = 0; k <= n; ++k) {
                M += ms[k];
                ok &= ms[k] >= 0.0 && is_finite(ms[k]);
                for (int c = 0; c < 3; ++c) {
                    ok &= is_finite(xs[3 * k + c]) && is_finite(us[3 * k + c]);
                    xc[c] += ms[k] * xs[3 * k + c];
                    vc[c] += ms[k] * us[3 * k + c];
                }
                if (k > 0)
                    ok &= !(xs[3 * k] == xs[0] && xs[3 * k + 1] == xs[1] && xs[3 * k + 2] == xs[2]);
            }
            for (int c = 0; c < 3; ++c) {
                xc[c] /= M;
                vc[c] /= M;
            }
        }
        if (ok && p < n) {
            mm = ms[1 + p];
            st.m[lane] = mm;
            st.qx[lane] = xs[3 * (1 + p) + 0] - xs[0];
            st.qy[lane] = xs[3 * (1 + p) + 1] - xs[1];
            st.qz[lane] = xs[3 * (1 + p) + 2] - xs[2];
            st.vx[lane] = us[3 * (1 + p) + 0] - vc[0];
            st.vy[lane] = us[3 * (1 + p) + 1] - vc[1];
            st.vz[lane] = us[3 * (1 + p) + 2] - vc[2];
        }
    }
    if (!(ok && p < n)) {                            // padding lane or rejected system
        st.m[lane] = 0.0;
        st.qx[lane] = parked_x(p);
        st.qy[lane] = 0.0;
        st.qz[lane] = 0.0;
        st.vx[lane] = 0.0;
        st.vy[lane] = 0.0;
        st.vz[lane] = 0.0;
    }
    if (p == 0) {
        if (!ok) {
            m0 = 1.0;
            dt = 1.0e-3;
            M = 1.0;
        }
        st.m0[s] = m0;
        st.dt[s] = dt;
        st.M[s] = M;
        for (int c = 0; c < 3; ++c) {
            st.xcm[(size_t)c * st.S_pad + s] = xc[c];
            st.vcm[(size_t)c * st.S_pad + s] = vc[c];
        }
        st.nplan[s] = ok ? n : 0;
        st.status[s] = (s < st.S && !ok) ? WHG_STATUS_INVALID : 0;
        st.nstep[s] = 0;
    }
}

// n Wisdom-Holman steps, state in registers (Eq. 2 with fused drifts).
template <int G, int NT, int GRM>
__global__ void __launch_bounds__(WHG_MAX_BLOCK) k_step(WhgState st, long long nsteps)
{
    const int tid = blockIdx.x * blockDim.x + threadIdx.x;
    const int s = tid / G, p = tid & (G - 1);
    const size_t lane = (size_t)s * G + p;
    const double m = st.m[lane];
    double qx = st.qx[lane], qy = st.qy[lane], qz = st.qz[lane];
    double vx = st.vx[lane], vy = st.vy[lane], vz = st.vz[lane];
    const double mu = st.m0[s], dt = st.dt[s];
    const int npl = st.nplan[s];
    int status = st.status[s];
    const long long nstep0 = st.nstep[s];
    const bool real = s < st.S && p < npl;
    bool alive = s < st.S && status == 0;
    const double hm = dt * m;
    const double jc = (0.5 * dt) / mu;
    const double mrat = m / mu;
    const double kgr = GRM ? (-6.0 * mu * mu * dt) / (st.c_light * st.c_light) : 0.0;
    const unsigned gmask = group_mask<G>();
    long long done = 0;
    for (long long k = 0; k < nsteps; ++k) {
        if (!__any_sync(WHG_FULL_MASK, alive)) break;        // whole warp frozen
        const double sqx = qx, sqy = qy, sqz = qz, svx = vx, svy = vy, svz = vz;
        const double hK = (nstep0 + done == 0) ? 0.5 * dt : dt;
        const bool bound = kepler_drift<NT>(mu, hK, qx, qy, qz, vx, vy, vz);
        jump<G>(m, jc, vx, vy, vz, qx, qy, qz);
        kick<G, GRM>(p, qx, qy, qz, hm, mrat, kgr, vx, vy, vz);
        jump<G>(m, jc, vx, vy, vz, qx, qy, qz);
        const bool fin = is_finite(qx) & is_finite(qy) & is_finite(qz) & is_finite(vx) &
                         is_finite(vy) & is_finite(vz);
        const unsigned bad_h = __ballot_sync(WHG_FULL_MASK, real && !bound) & gmask;
        const unsigned bad_n = __ballot_sync(WHG_FULL_MASK, real && !fin) & gmask;
        const bool ok = (bad_h | bad_n) == 0u;
        if (!(alive && real && ok)) {                 // roll back: padding, frozen, failed
            qx = sqx; qy = sqy; qz = sqz;
            vx = svx; vy = svy; vz = svz;
        }
        if (alive && !ok) {
            status |= (bad_n ? WHG_STATUS_NONFINITE : 0) | (bad_h ? WHG_STATUS_HYPERBOLIC : 0);
            alive = false;
        }
        done += alive ? 1 : 0;
    }
    if (real) {
        st.qx[lane] = qx; st.qy[lane] = qy; st.qz[lane] = qz;
        st.vx[lane] = vx; st.vy[lane] = vy; st.vz[lane] = vz;
    }
    if (p == 0 && s < st.S) {
        st.status[s] = status;
        st.nstep[s] = nstep0 + done;
    }
}

// Synchronized copy (pending K(dt/2)) -> inertial frame (Sec. 3.1 inverted):
// x_0 = X_cm + V_cm t - sum m_i Q_i / M, x_i = x_0 + Q_i,
// u_0 = V_cm - sum m_i v_i / m0, u_i = v_i + V_cm.
template <int G, int NT>
__global__ void __launch_bounds__(WHG_MAX_BLOCK) k_read(WhgState st, WhgOut out)
{
    const int tid = blockIdx.x * blockDim.x + threadIdx.x;
    const int s = tid / G, p = tid & (G - 1);
    const size_t lane = (size_t)s * G + p;
    const double m = st.m[lane];
    double qx = st.qx[lane], qy = st.qy[lane], qz = st.qz[lane];
    double vx = st.vx[lane], vy = st.vy[lane], vz = st.vz[lane];
    const double mu = st.m0[s], dt = st.dt[s];
    const long long ns = st.nstep[s];
    if (ns > 0) kepler_drift<NT>(mu, 0.5 * dt, qx, qy, qz, vx, vy, vz);
    const double sqx = group_sum<G>(m * qx), sqy = group_sum<G>(m * qy), sqz = group_sum<G>(m * qz);
    const double spx = group_sum<G>(m * vx), spy = group_sum<G>(m * vy), spz = group_sum<G>(m * vz);
    if (s >= st.S) return;                           // after the last shuffle
    const int npl = st.nplan[s];
    const int B = 1 + st.Nmax;
    const double t = (double)ns * dt;
    const double M = st.M[s];
    double x0[3], u0[3];
    const double sq[3] = {sqx, sqy, sqz}, sp[3] = {spx, spy, spz};
    for (int c = 0; c < 3; ++c) {
        const double X = st.xcm[(size_t)c * st.S_pad + s], V = st.vcm[(size_t)c * st.S_pad + s];
        x0[c] = (X + V * t) - sq[c] / M;
        u0[c] = V - sp[c] / mu;
    }
    if (p < st.Nmax) {
        const size_t o = ((size_t)s * B + 1 + p) * 3;
        const bool live = p < npl;
        if (out.pos) {
            out.pos[o + 0] = live ? x0[0] + qx : 0.0;
            out.pos[o + 1] = live ? x0[1] + qy : 0.0;
            out.pos[o + 2] = live ? x0[2] + qz : 0.0;
        }
        if (out.vel) {
            out.vel[o + 0] = live ? vx + st.vcm[s] : 0.0;
            out.vel[o + 1] = live ? vy + st.vcm[(size_t)st.S_pad + s] : 0.0;
            out.vel[o + 2] = live ? vz + st.vcm[(size_t)2 * st.S_pad + s] : 0.0;
        }
    }
    if (p == 0) {
        const size_t o = (size_t)s * B * 3;
        for (int c = 0; c < 3; ++c) {
            if (out.pos) out.pos[o + c] = x0[c];
            if (out.vel) out.vel[o + c] = u0[c];
        }
        if (out.status) out.status[s] = st.status[s];
        if (out.t) out.t[s] = t;
    }
}

// Energy of the synchronized state: H_0 + H_K + H_I + H_J (Eq. 1) [+ GR].
template <int G, int NT, int GRM>
__global__ void __launch_bounds__(WHG_MAX_BLOCK) k_energy(WhgState st, WhgOut out)
{
    const int tid = blockIdx.x * blockDim.x + threadIdx.x;
    const int s = tid / G, p = tid & (G - 1);
    const size_t lane = (size_t)s * G + p;
    const double m = st.m[lane];
    double qx = st.qx[lane], qy = st.qy[lane], qz = st.qz[lane];
    double vx = st.vx[lane], vy = st.vy[lane], vz = st.vz[lane];
    const double mu = st.m0[s], dt = st.dt[s];
    if (st.nstep[s] > 0) kepler_drift<NT>(mu, 0.5 * dt, qx, qy, qz, vx, vy, vz);
    const double r2 = fma(qx, qx, fma(qy, qy, qz * qz));
    double pair = 0.0;
#pragma unroll
    for (int k = 1; k < G; ++k) {
        const int j = (p + k) & (G - 1);
        const double dx = __shfl_sync(WHG_FULL_MASK, qx, j, G) - qx;
        const double dy = __shfl_sync(WHG_FULL_MASK, qy, j, G) - qy;
        const double dz = __shfl_sync(WHG_FULL_MASK, qz, j, G) - qz;
        const double mj = __shfl_sync(WHG_FULL_MASK, m, j, G);
        pair += m * mj / sqrt(fma(dx, dx, fma(dy, dy, dz * dz)));
    }
    double part = 0.5 * m * fma(vx, vx, fma(vy, vy, vz * vz)) - mu * m / sqrt(r2) - 0.5 * pair;
    if (GRM != 0) part += -3.0 * m * mu * mu / (st.c_light * st.c_light * r2);
    const double tot = group_sum<G>(part);
    const double px = group_sum<G>(m * vx), py = group_sum<G>(m * vy), pz = group_sum<G>(m * vz);
    if (s >= st.S || p != 0) return;
    double h0 = 0.0;
    for (int c = 0; c < 3; ++c) {
        const double V = st.vcm[(size_t)c * st.S_pad + s];
        h0 += 0.5 * st.M[s] * V * V;
    }
    out.E[s] = h0 + tot + (px * px + py * py + pz * pz) / (2.0 * mu);
}

// Raw state copy between the lane arrays and the [S][Nmax][3] layout.
template <int G>
__global__ void __launch_bounds__(WHG_MAX_BLOCK) k_raw(WhgState st, WhgOut io, int set)
{
    const int tid = blockIdx.x * blockDim.x + threadIdx.x;
    const int s = tid / G, p = tid & (G - 1);
    if (s >= st.S) return;
    const size_t lane = (size_t)s * G + p;
    const int npl = st.nplan[s];
    if (p < st.Nmax) {
        const size_t o = ((size_t)s * st.Nmax + p) * 3;
        if (set) {
            if (p < npl) {
                st.qx[lane] = io.inQ[o]; st.qy[lane] = io.inQ[o + 1]; st.qz[lane] = io.inQ[o + 2];
                st.vx[lane] = io.inv[o]; st.vy[lane] = io.inv[o + 1]; st.vz[lane] = io.inv[o + 2];
            }
        } else {
            const bool live = p < npl;
            io.rawQ[o] = live ? st.qx[lane] : 0.0;
            io.rawQ[o + 1] = live ? st.qy[lane] : 0.0;
            io.rawQ[o + 2] = live ? st.qz[lane] : 0.0;
            io.rawv[o] = live ? st.vx[lane] : 0.0;
            io.rawv[o + 1] = live ? st.vy[lane] : 0.0;
            io.rawv[o + 2] = live ? st.vz[lane] : 0.0;
        }
    }
    if (p == 0) {
        if (set) {
            st.nstep[s] = io.inn[s];
            st.status[s] = io.ins[s];
        } else {
            io.rawn[s] = st.nstep[s];
            io.status[s] = st.status[s];
        }
    }
}

// ------------------------------------------------------------------------
// Launchers (host side) for one G.

template <int G>
struct Launchers {
    static cudaError_t init(const WhgState& st, const WhgIn& in, const WhgLaunch& l)
    {
        k_init<G><<<l.grid, l.block, 0, l.stream>>>(st, in);
        return cudaGetLastError();
    }

    template <int NT, int GRM>
    static cudaError_t step_t(const WhgState& st, long long n, const WhgLaunch& l)
    {
        k_step<G, NT, GRM><<<l.grid, l.block, 0, l.stream>>>(st, n);
        return cudaGetLastError();
    }

    static cudaError_t step(const WhgState& st, long long n, int nt, int grm, const WhgLaunch& l)
    {
        if (nt == 8) {
            if (grm == 0) return step_t<8, 0>(st, n, l);
            if (grm == 1) return step_t<8, 1>(st, n, l);
            return step_t<8, 2>(st, n, l);
        }
        if (grm == 0) return step_t<6, 0>(st, n, l);
        if (grm == 1) return step_t<6, 1>(st, n, l);
        return step_t<6, 2>(st, n, l);
    }

    static cudaError_t read(const WhgState& st, const WhgOut& o, int nt, const WhgLaunch& l)
    {
        if (nt == 8)
            k_read<G, 8><<<l.grid, l.block, 0, l.stream>>>(st, o);
        else
            k_read<G, 6><<<l.grid, l.block, 0, l.stream>>>(st, o);
        return cudaGetLastError();
    }

    static cudaError_t energy(const WhgState& st, const WhgOut& o, int nt, int grm,
                              const WhgLaunch& l)
    {
        if (nt == 8) {
            if (grm == 0) k_energy<G, 8, 0><<<l.grid, l.block, 0, l.stream>>>(st, o);
            else k_energy<G, 8, 1><<<l.grid, l.block, 0, l.stream>>>(st, o);
        } else {
            if (grm == 0) k_energy<G, 6, 0><<<l.grid, l.block, 0, l.stream>>>(st, o);
            else k_energy<G, 6, 1><<<l.grid, l.block, 0, l.stream>>>(st, o);
        }
        return cudaGetLastError();
    }

    static cudaError_t raw(const WhgState& st, const WhgOut& o, int set, const WhgLaunch& l)
    {
        k_raw<G><<<l.grid, l.block, 0, l.stream>>>(st, o, set);
        return cudaGetLastError();
    }
};

}  // namespace whg

#define WHG_DEFINE_KERNEL_TABLE(G_)                                                            \
    const WhgKernels whg_kernels_g##G_ = {whg::Launchers<G_>::init, whg::Launchers<G_>::step, \
                                          whg::Launchers<G_>::read, whg::Launchers<G_>::energy, \
                                          whg::Launchers<G_>::raw};
