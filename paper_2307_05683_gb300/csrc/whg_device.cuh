// whg_device.cuh -- device code of libwhg: FP64 special functions, the
// Wisdom-Holman sub-steps and the kernel bodies, templated on the number L of
// warp lanes per system (one lane per planet, L in 1..8, floor(32/L) systems
// per warp).
//
// Why the code looks as it does.  The whole step is FP64 arithmetic on a few registers
// per lane; on this part the FP64 pipe retires about 2 lanes per clock per SM
// while FP32, integer, shuffle and MUFU work retire tens of times faster.  So
// the step is bound by the number of FP64 instructions alone, and the code
// spends integer and FP32 work freely to save FP64 instructions:
//   * reciprocals and reciprocal square roots start from the FP32 hardware
//     approximation of a mantissa built with integer operations and take one
//     third-order refinement whose correction (from the exact 1 - x y or
//     1 - x y^2) is formed in fixed point on the integer pipe, leaving one
//     FP64 FMA per call, and the solver's factors -1/2 are exponent
//     decrements;
//   * the all-pairs interaction uses Newton's third law (Sec. 3.3), with
//     partner schedules that suit warp shuffles rather than AVX512 lanes;
//   * cross-lane sums of 3-vectors are reduce-scatters by xor partners when L
//     is 4 or 8 (Sec. 3.4 reduces with a butterfly), else gathers in fixed
//     lane order; either way every lane gets the bitwise-identical total;
//   * a persistent work queue moves (warp-group, steps) units between SMs so
//     that no SM finishes late.
// State stays in registers during a unit of steps; HBM is touched only at
// load and store (coalesced: consecutive lanes read consecutive doubles).
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
//     1/sqrt(x) = y0 (1 + e/2 + 3e^2/8 + ...)     ->  y0 + y0 (e/2 + 3e^2/8)
// whose truncation error (~e^3 < 2^-61) is far below double rounding; results
// are within about one ulp of the exact value.  e is exact in integer
// arithmetic (the seed has 24 significant bits), and so is the correction to
// the precision it needs, so only the final y0 + y0 t is an FP64 operation.

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

// ------------------------------------------------------------------------
// Integer-pipe pieces of the reciprocal and reciprocal square root.  On this
// GPU an FP64 warp instruction holds the FP64 pipe for 64 cycles and an
// integer one its pipe for about 1, so integer forms replace FP64 operations
// wherever the operands are short: the seeds y below carry 24 significant
// bits (an FP32 approximation widened to FP64).

// D 2^-s rounded to the nearest double (ties to even); D a signed 64-bit
// integer, the result a normal double or zero.
__device__ __forceinline__ double scaled_int_to_double(long long D, int s)
{
    const unsigned long long sign = D < 0 ? 0x8000000000000000ULL : 0ULL;
    const unsigned long long a = D < 0 ? 0ULL - (unsigned long long)D : (unsigned long long)D;
    const int lz = __clzll((long long)a);
    const unsigned long long n = a << (lz & 63);             // leading one at bit 63
    unsigned long long m = n >> 11;                          // 53 bits
    const unsigned long long rem = n & 0x7ffULL;
    m += (rem > 0x400ULL || (rem == 0x400ULL && (m & 1ULL))) ? 1ULL : 0ULL;
    const unsigned long long carry = m >> 53;                // rounding reached 2^53
    m >>= carry;
    const long long E = 63 - lz - s + 1023 + (long long)carry;
    const unsigned long long bits = sign | ((unsigned long long)E << 52) | (m & 0x000fffffffffffffULL);
    return a ? __longlong_as_double((long long)bits) : 0.0;
}

// The double with biased exponent E and fraction bits f, saturated as the
// FP64 product would be: +inf above the exponent range (a zero or tiny
// argument of the reciprocal square roots), 0 below it.
__device__ __forceinline__ double exp_bits_to_double(long long E, unsigned long long f)
{
    const unsigned long long bits = E >= 0x7ff ? 0x7ff0000000000000ULL
                                  : (E <= 0 ? 0ULL : (((unsigned long long)E << 52) | f));
    return __longlong_as_double((long long)bits);
}

// -x/2 exactly, on the integer pipe: an exponent decrement and a sign flip
// for normal x; zero, subnormal and the smallest normals halve their
// significand with round-to-nearest-even (the result's encoding follows from
// the carry); inf and NaN keep their exponent.  Equal to -0.5 * x.
__device__ __forceinline__ double neg_half(double x)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const unsigned long long sign = (b ^ 0x8000000000000000ULL) & 0x8000000000000000ULL;
    const unsigned long long ex = (b >> 52) & 0x7ffULL;
    const unsigned long long f = b & 0x000fffffffffffffULL;
    const unsigned long long M = ex == 1ULL ? (f | 0x0010000000000000ULL) : f;   // subnormal-scale significand
    const unsigned long long half = (M >> 1) + (M & (M >> 1) & 1ULL);            // M/2, ties to even
    const unsigned long long normal = (b - 0x0010000000000000ULL) & 0x7fffffffffffffffULL;
    const unsigned long long mag = ex >= 2ULL ? (ex == 0x7ffULL ? (b & 0x7fffffffffffffffULL) : normal) : half;
    return __longlong_as_double((long long)(sign | mag));
}

// 53-bit significand of a finite normal double as an integer.
__device__ __forceinline__ unsigned long long significand(unsigned hi, unsigned lo)
{
    return ((unsigned long long)((hi & 0x000fffffu) | 0x00100000u) << 32) | lo;
}

// 1/x for finite x with 2^-1022 <= |x| < 2^1021 (either sign; 1/x normal):
// FP32 seed y (24 bits), then
// y (1 + e + e^2) with e = 1 - x y.  The seed is within ~2^-22 of 1/x, so
// x y = 2^s - D with |D| < 2^55 and s = 202 - (y's FP32 exponent) in 75..76:
// D = -(Mx My mod 2^64) in wrap-around integer arithmetic, so e = D 2^-s
// exactly.  The correction t = e + e^2 is formed in the same fixed point (e^2
// from the top 31 bits of D: relative error 2^-30 of a term below 2^-43) and
// rounded once to a double; 1/x = fma(y, t, y), within one ulp (the neglected
// e^3 is below 2^-65).  1 FP64 operation.
__device__ __forceinline__ double rcp(double x)
{
    const unsigned hi = (unsigned)__double2hiint(x);
    const unsigned lo = (unsigned)__double2loint(x);
    const int ex = (int)((hi >> 20) & 0x7ffu);                         // biased exponent
    const float mant = __uint_as_float(0x3f800000u | ((hi & 0x000fffffu) << 3) | (lo >> 29));
    const unsigned rb = __float_as_uint(approx_rcp_f32(mant));          // in (0.5, 1]
    const int erb = (int)((rb >> 23) & 0xffu);
    const int dex = erb - 127 + 2046 - ex;                              // biased exponent of 1/x
    const unsigned yhi = (hi & 0x80000000u) | ((unsigned)dex << 20) | ((rb >> 3) & 0x000fffffu);
    const double y = __hiloint2double((int)yhi, (int)(rb << 29));
    const unsigned long long My = (rb & 0x007fffffu) | 0x00800000u;
    const long long D = (long long)(0ULL - significand(hi, lo) * My);
    const int sc = 202 - erb;                                           // 75..76
    const long long Dh = D >> 24;                                       // |Dh| < 2^31
    const long long T = D + ((Dh * Dh) >> ((sc - 48) & 63));            // (e + e^2) 2^sc
    double t = scaled_int_to_double(T, sc);
    // outside the domain keep the IEEE outcome of the FP64 form: zero and
    // subnormal x give an infinite result, inf and NaN a NaN
    t = ex == 0 ? __longlong_as_double(0x7ff0000000000000LL) : t;
    t = ex == 0x7ff ? __longlong_as_double(0x7ff8000000000000LL) : t;
    return fma(y, t, y);
}

// 1/x^2 for finite x > 0 with 1/x^2 normal: the same seed, y^2 exact (48
// bits) and 1/x^2 = y^2 (1 - e)^-2 = y^2 (1 + 2e + 3e^2 + ...), the
// correction 2e + 3e^2 formed on the integer pipe as in rcp (the neglected
// 4e^3 is below 2^-61).  1 FP64 operation instead of a reciprocal and a
// square.  Zero and subnormal x give +inf, inf and NaN give NaN.
__device__ __forceinline__ double rcp_sq(double x)
{
    const unsigned hi = (unsigned)__double2hiint(x);
    const unsigned lo = (unsigned)__double2loint(x);
    const int ex = (int)((hi >> 20) & 0x7ffu);                         // biased exponent
    const float mant = __uint_as_float(0x3f800000u | ((hi & 0x000fffffu) << 3) | (lo >> 29));
    const unsigned rb = __float_as_uint(approx_rcp_f32(mant));          // in (0.5, 1]
    const int erb = (int)((rb >> 23) & 0xffu);
    const int dex = erb - 127 + 2046 - ex;                              // biased exponent of 1/x
    const unsigned long long My = (rb & 0x007fffffu) | 0x00800000u;
    const unsigned long long S = My * My;                               // [2^46, 2^48), exact
    const unsigned long long top = S >> 47;
    const double y2 = exp_bits_to_double(2 * (long long)dex - 1023 + (long long)top,
                                         (S << (6 - top)) & 0x000fffffffffffffULL);
    const long long D = (long long)(0ULL - significand(hi, lo) * My);   // e 2^sc
    const int sc = 202 - erb;                                           // 75..76
    const long long Dh = D >> 24;
    const long long T = 2 * D + 3 * ((Dh * Dh) >> ((sc - 48) & 63));   // (2e + 3e^2) 2^sc
    double r = fma(y2, scaled_int_to_double(T, sc), y2);
    r = ex == 0 ? __longlong_as_double(0x7ff0000000000000LL) : r;
    r = ex == 0x7ff ? __longlong_as_double(0x7ff8000000000000LL) : r;
    return r;
}

// x^(-1/2) and x^(-3/2) for finite normal x > 0 (x^(-3/2) normal for
// 2^-681 < x < 2^682: the 1/r^3 of a pair from r^2), from the seed y of
// rsqrt.approx on an FP32 copy of the mantissa (24-bit significand My, the
// exponent handled with integers), with the whole correction on the integer
// pipe and a single FP64 operation:
//     x^(-1/2) = y   (1 - e)^(-1/2) = y   (1 + e/2  + 3e^2/8  + ...),
//     x^(-3/2) = y^3 (1 - e)^(-3/2) = y^3 (1 + 3e/2 + 15e^2/8 + ...),
// e = 1 - x y^2.  y^3 is rounded to nearest from the exact My^3 (72 bits).
// x = Mx 2^(ex-52) (53-bit significand Mx) and y^2 = S 2^(2 dex - 2092)
// (S = My^2, 48 bits) give x y^2 = P 2^-s with P = Mx S (101 bits, two
// 64-bit products) and s = 2144 - ex - 2 dex (98..101), so e = (2^s - P) 2^-s
// exactly, |e| < 2^-21 (the FP32 seed's error).  E = e 2^83 fits an int64; the
// correction u = a e + b e^2 is formed from E in fixed point (e^2 from the
// top 32 bits of E: relative error 2^-30 of a term below 2^-42) and rounded
// once to a double, and the result is fma(w, u, w) with w = y or y^3: within
// about one ulp, the neglected terms (~e^3) being below 2^-61.  Zero and
// subnormal x give +inf, inf and NaN give NaN.
template <bool CUBE>
__device__ __forceinline__ double rsqrt_pow(double x)
{
    const unsigned hi = (unsigned)__double2hiint(x);
    const unsigned lo = (unsigned)__double2loint(x);
    const unsigned ef = (hi >> 20) & 0x7ffu;
    const int ex = (int)ef - 1023;                                     // unbiased exponent
    const int odd = ex & 1;
    const int half = (ex - odd) / 2;                                   // x = 4^half * mant
    const float mant = __uint_as_float(((unsigned)(127 + odd) << 23) | ((hi & 0x000fffffu) << 3) |
                                       (lo >> 29));                    // in [1, 4)
    const unsigned rb = __float_as_uint(approx_rsqrt_f32(mant));       // in (0.5, 1]
    const int dex = (int)((rb >> 23) & 0xffu) - 127 - half + 1023;     // biased exponent of y
    const unsigned long long My = (rb & 0x007fffffu) | 0x00800000u;
    const unsigned long long S = My * My;                              // [2^46, 2^48), exact
    double w;
    if (CUBE) {                                                        // My^3 in [2^69, 2^72)
        const unsigned long long clo = S * My, chi = __umul64hi(S, My);
        const int p = 127 - __clzll((long long)chi);                   // leading-one position
        const int sh = p - 52;                                         // 17..19
        unsigned long long m = ((clo >> sh) | (chi << (64 - sh))) & 0x001fffffffffffffULL;
        const unsigned long long rem = clo & ((1ULL << sh) - 1ULL), hb = 1ULL << (sh - 1);
        m += (rem > hb || (rem == hb && (m & 1ULL))) ? 1ULL : 0ULL;
        const unsigned long long carry = m >> 53;
        m >>= carry;
        const long long E3 = p + 3 * dex - 2115 + (long long)carry;
        w = exp_bits_to_double(E3, m & 0x000fffffffffffffULL);
    } else {
        w = __hiloint2double((int)(((unsigned)dex << 20) | ((rb >> 3) & 0x000fffffu)), (int)(rb << 29));
    }
    const unsigned long long Mx = significand(hi, lo);
    const unsigned long long plo = Mx * S, phi = __umul64hi(Mx, S);
    const int s = 2144 - ex - 2 * dex;                                 // 98..101 for normal x
    const unsigned long long dlo = 0ULL - plo;
    const unsigned long long dhi = (1ULL << ((s - 64) & 63)) - phi - (plo != 0ULL ? 1ULL : 0ULL);
    const int sr = (s - 83) & 63;                                      // 15..18
    const long long E = (long long)((dlo >> sr) | (dhi << ((64 - sr) & 63)));   // e 2^83
    const long long Eh = E >> 32;                                      // e 2^51
    const long long E2 = (Eh * Eh) >> 22;                              // e^2 2^80
    const long long U = CUBE ? E + (E >> 1) + 15 * E2 : (E >> 1) + 3 * E2;   // u 2^83
    double r = fma(w, scaled_int_to_double(U, 83), w);
    r = ef == 0u ? __longlong_as_double(0x7ff0000000000000LL) : r;
    r = ef == 0x7ffu ? __longlong_as_double(0x7ff8000000000000LL) : r;
    return r;
}

__device__ __forceinline__ double rsqrt(double x) { return rsqrt_pow<false>(x); }
__device__ __forceinline__ double rsqrt_cubed(double x) { return rsqrt_pow<true>(x); }

// FP64 -> FP32 from the bit fields (sign, exponent rebiased from 1023 to
// 127, mantissa truncated to 23 bits) on the integer pipe: the hardware
// conversion runs on the FP64 pipe, the scarce unit here.  Rounds toward
// zero; |x| below the FP32 normal range gives a signed zero, above it (and
// inf, NaN) a signed infinity.
__device__ __forceinline__ float to_f32(double x)
{
    const unsigned hi = (unsigned)__double2hiint(x);
    const unsigned lo = (unsigned)__double2loint(x);
    const unsigned sign = hi & 0x80000000u;
    const int ex = (int)((hi >> 20) & 0x7ffu) - 1023 + 127;            // FP32 biased exponent
    unsigned b = sign | ((unsigned)ex << 23) | ((hi & 0x000fffffu) << 3) | (lo >> 29);
    b = ex <= 0 ? sign : b;
    b = ex >= 255 ? (sign | 0x7f800000u) : b;
    return __uint_as_float(b);
}

// FP32 -> FP64 from the bit fields (exact for normal numbers; subnormals give
// a signed zero; inf and NaN stay inf and NaN), on the integer pipe.
__device__ __forceinline__ double to_f64(float f)
{
    const unsigned b = __float_as_uint(f);
    const unsigned sign = b & 0x80000000u;
    const unsigned ex = (b >> 23) & 0xffu;
    const unsigned man = b & 0x007fffffu;
    unsigned hi = sign | ((ex + 896u) << 20) | (man >> 3);
    unsigned lo = man << 29;
    hi = ex == 0u ? sign : hi;
    lo = ex == 0u ? 0u : lo;
    hi = ex == 255u ? (sign | 0x7ff00000u | (man ? 0x00080000u : 0u)) : hi;
    lo = ex == 255u ? 0u : lo;
    return __hiloint2double((int)hi, (int)lo);
}

__device__ __forceinline__ bool is_finite(double x)
{
    return (__double2hiint(x) & 0x7ff00000) != 0x7ff00000;
}

// ------------------------------------------------------------------------
// Stumpff functions c_2(z), c_3(z) by their T-term Taylor series, carried
// through the z^T term: c_n(z) = sum_{k<=T} (-z)^k / (n+2k)! (Sec. 3.2: series
// with a table of coefficients, no quarter-angle reduction; T terms after the
// leading 1/n!).  The coefficients 1/k! are compile-time constants: k! is
// exact in double for k <= 22, and the compiler rounds 1/k! once.

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
    c2 = 1.0 / Factorial<2 * T + 2>::value;      // term k = T
    c3 = 1.0 / Factorial<2 * T + 3>::value;
    StumpffHorner<T - 1>::run(z, c2, c3);
}

// The same series in FP32 (coefficients 1/k! rounded to float), for the
// Halley phase's starting point only.
template <int K>
struct StumpffHornerF {
    static __device__ __forceinline__ void run(float z, float& c2, float& c3)
    {
        c2 = fmaf(-z, c2, (float)(1.0 / Factorial<2 * K + 2>::value));
        c3 = fmaf(-z, c3, (float)(1.0 / Factorial<2 * K + 3>::value));
        StumpffHornerF<K - 1>::run(z, c2, c3);
    }
};
template <>
struct StumpffHornerF<-1> {
    static __device__ __forceinline__ void run(float, float&, float&) {}
};

template <int T>
__device__ __forceinline__ void stumpff_c2c3_f32(float z, float& c2, float& c3)
{
    c2 = (float)(1.0 / Factorial<2 * T + 2>::value);
    c3 = (float)(1.0 / Factorial<2 * T + 3>::value);
    StumpffHornerF<T - 1>::run(z, c2, c3);
}


// ------------------------------------------------------------------------
// Kepler drift of one planet for time h under H_K,i (Sec. 3.2, Eq. 3),
// mu = G m0.  Universal variable X solves Kepler's equation
//     F(X)  = r0 G1 + eta0 G2 + mu G3 - h = r0 X + eta0 G2 + zeta0 G3 - h = 0,
//     F'(X) = r = r0 + eta0 G1 + zeta0 G2,
//     F''   = eta0 G0 + zeta0 G1
// (the second forms use G0 = 1 - beta G2, G1 = X - beta G3 and
// zeta0 = mu - beta r0, so only the c2 and c3 series are needed): initial
// guess h/r0 (the first-order value of X(h); the paper gives none), 2 Halley
// steps with 4-term series, 2 Newton steps with NT-term series.  The G_n at
// the final X = X1 + d come from the values at the last Newton point X1 by
// one Taylor step (dG_n/dX = G_{n-1}); |d| is the last Newton correction, so
// the neglected d^2 terms are far below rounding.  Then the Lagrange f - 1,
// g, fdot, gdot - 1.
// h32 (uniform across the warp) runs the initial guess and the Halley phase
// in FP32: they only supply the Newton phase's starting point, and from a
// start within ~1e-7 two FP64 Newton steps reach FP64 rounding
// (quadratic convergence: 1e-7 -> 1e-14 -> rounding), so the result keeps
// FP64 accuracy wherever the FP64 Halley phase converges, while ~60 FP64
// operations per drift move to the FP32 pipe.  No other branches.
// Returns beta > 0; Xout receives the final universal variable.  With
// VALS, *dv also receives the drift's intermediate values (for the adjoint's
// tape); the arithmetic is the same either way.
struct DriftVals {
    double r0i, r0, eta0, beta;          // of the initial state
    double G1, G2, G3;                   // Stiefel functions at the final X
    double ri, A, fm1, g, fd, gdm1;      // 1/r, mu/r0, Lagrange coefficients
};

template <int NT, bool VALS = false>
__device__ __forceinline__ bool kepler_drift(double mu, double h, double& qx, double& qy,
                                             double& qz, double& vx, double& vy, double& vz,
                                             double& Xout, bool h32 = false, DriftVals* dv = nullptr)
{
    const double r0sq = fma(qx, qx, fma(qy, qy, qz * qz));
    const double r0i = rsqrt(r0sq);
    const double r0 = r0sq * r0i;
    const double eta0 = fma(qx, vx, fma(qy, vy, qz * vz));
    const double v2 = fma(vx, vx, fma(vy, vy, vz * vz));
    const double beta = fma(2.0 * mu, r0i, -v2);
    const double zeta0 = fma(-beta, r0, mu);
    double X, X2, c2, c3, G1, G2, G3;
    if (h32) {
        const float r0f = to_f32(r0), r0if = to_f32(r0i), eta0f = to_f32(eta0);
        const float zeta0f = to_f32(zeta0), betaf = to_f32(beta), hf = to_f32(h);
        const float beta_eta0f = betaf * eta0f, beta_zeta0f = betaf * zeta0f;
        float Xs = hf * r0if;
#pragma unroll
        for (int it = 0; it < 2; ++it) {             // Halley (FP32)
            const float Y2 = Xs * Xs;
            float s2, s3;
            stumpff_c2c3_f32<4>(betaf * Y2, s2, s3);
            const float H2 = Y2 * s2, H3 = (Y2 * Xs) * s3;
            const float F = fmaf(r0f, Xs, fmaf(eta0f, H2, fmaf(zeta0f, H3, -hf)));
            const float Fp = fmaf(zeta0f, H2, fmaf(-beta_eta0f, H3, fmaf(eta0f, Xs, r0f)));
            const float Fpp = fmaf(-beta_zeta0f, H3, fmaf(-beta_eta0f, H2, fmaf(zeta0f, Xs, eta0f)));
            const float den = fmaf(-0.5f * F, Fpp, Fp * Fp);
            Xs = Xs - __fdividef(F * Fp, den);
        }
        X = to_f64(Xs);
    } else {
        X = h * r0i;
#pragma unroll
        for (int it = 0; it < 2; ++it) {             // Halley
            X2 = X * X;
            stumpff_c2c3<4>(beta * X2, c2, c3);
            G2 = X2 * c2;
            G3 = (X2 * X) * c3;
            G1 = fma(-beta, G3, X);
            const double G0 = fma(-beta, G2, 1.0);
            const double F = fma(r0, X, fma(eta0, G2, fma(zeta0, G3, -h)));
            const double Fp = fma(zeta0, G2, fma(eta0, G1, r0));
            const double Fpp = fma(zeta0, G1, eta0 * G0);
            const double den = fma(neg_half(F), Fpp, Fp * Fp);   // (2F'^2 - F F'') / 2
            X = fma(-(F * Fp), rcp(den), X);
        }
    }
    double d = 0.0;
#pragma unroll
    for (int it = 0; it < 2; ++it) {                 // Newton
        X2 = X * X;
        stumpff_c2c3<NT>(beta * X2, c2, c3);
        G2 = X2 * c2;
        G3 = (X2 * X) * c3;
        G1 = fma(-beta, G3, X);
        const double F = fma(r0, X, fma(eta0, G2, fma(zeta0, G3, -h)));
        const double Fp = fma(zeta0, G2, fma(eta0, G1, r0));
        if (it == 0) X = fma(-F, rcp(Fp), X);        // the first correction applied at once
        else d = -F * rcp(Fp);                       // the last one kept for the G_n update
    }
    // G at the final X + d from the last Newton point X.
    const double G0 = fma(-beta, G2, 1.0);
    const double Xf = X + d;
    const double G3f = fma(d, G2, G3);
    const double G2f = fma(d, G1, G2);
    const double G1f = fma(d, G0, G1);
    const double r = fma(zeta0, G2f, fma(eta0, G1f, r0));
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
    Xout = Xf;
    if constexpr (VALS) {
        dv->r0i = r0i; dv->r0 = r0; dv->eta0 = eta0; dv->beta = beta;
        dv->G1 = G1f; dv->G2 = G2f; dv->G3 = G3f;
        dv->ri = ri; dv->A = mr0; dv->fm1 = fm1; dv->g = g; dv->fd = fd; dv->gdm1 = gdm1;
    }
    return beta > 0.0;
}

template <int NT>
__device__ __forceinline__ bool kepler_drift(double mu, double h, double& qx, double& qy,
                                             double& qz, double& vx, double& vy, double& vz,
                                             bool h32 = false)
{
    double X;
    return kepler_drift<NT>(mu, h, qx, qy, qz, vx, vy, vz, X, h32);
}

// ------------------------------------------------------------------------
// Lane groups: L lanes per system, floor(32/L) systems per warp; lanes beyond
// the last whole group hold no system.
template <int L>
struct Group {
    static constexpr int SPW = 32 / L;     // systems per warp
    int lane, slot, p, base;
    bool in_group;
    __device__ __forceinline__ Group()
    {
        lane = (int)(threadIdx.x & 31u);
        slot = lane / L;
        in_group = slot < SPW;
        p = in_group ? lane - slot * L : 0;
        base = slot * L;
    }
    // lane holding planet (p + k) mod L of this system (own lane outside groups)
    __device__ __forceinline__ int at(int k) const
    {
        int q = p + k;
        q = q >= L ? q - L : (q < 0 ? q + L : q);
        return in_group ? base + q : lane;
    }
    __device__ __forceinline__ unsigned mask() const
    {
        return in_group ? (((L == 32) ? WHG_FULL_MASK : ((1u << L) - 1u)) << base) : (1u << lane);
    }
};

// Sum of x over the system's lanes, the same bits in every lane: xor
// butterfly (Sec. 3.4) for power-of-two L, else a fixed-order gather.
template <int L>
__device__ __forceinline__ double group_sum(const Group<L>& g, double x)
{
    if ((L & (L - 1)) == 0) {
#pragma unroll
        for (int o = 1; o < L; o <<= 1) x += __shfl_xor_sync(WHG_FULL_MASK, x, o);
        return x;
    } else {
        double s = __shfl_sync(WHG_FULL_MASK, x, g.in_group ? g.base : g.lane);
#pragma unroll
        for (int j = 1; j < L; ++j) s += __shfl_sync(WHG_FULL_MASK, x, g.in_group ? g.base + j : g.lane);
        return s;
    }
}

// Sums of the 3-vector (x, y, z) over the system's lanes, the same bits in
// every lane.  L = 4, 8: reduce-scatter of (x, y, z, 0) by xor partners
// (keep half, send half: 2 + 1 (+ 1) additions per lane instead of 3 log2 L),
// after which one lane pair holds each finished component (both lanes
// compute a + b, which is commutative in IEEE arithmetic), then three
// shuffles from those lanes give every lane the same values.  Other L:
// three group_sum.
template <int L>
__device__ __forceinline__ void group_sum3(const Group<L>& g, double x, double y, double z,
                                           double& sx, double& sy, double& sz)
{
    if (L == 4 || L == 8) {
        constexpr int H = L / 2, Q = L / 4;
        const bool hi = (g.p & H) != 0;          // keeps (z, 0), else (x, y)
        double k0 = hi ? z : x, k1 = hi ? 0.0 : y;
        const double s0 = hi ? x : z, s1 = hi ? y : 0.0;
        k0 += __shfl_xor_sync(WHG_FULL_MASK, s0, H);
        k1 += __shfl_xor_sync(WHG_FULL_MASK, s1, H);
        const bool mid = (g.p & Q) != 0;         // keeps the second of the pair
        double k = mid ? k1 : k0;
        k += __shfl_xor_sync(WHG_FULL_MASK, mid ? k0 : k1, Q);
        if (L == 8) k += __shfl_xor_sync(WHG_FULL_MASK, k, 1);
        // lane base + 2*hi + mid (L = 4), base + 4*hi + 2*mid (+1) (L = 8)
        // now holds component 2*hi + mid
        sx = __shfl_sync(WHG_FULL_MASK, k, g.base);
        sy = __shfl_sync(WHG_FULL_MASK, k, g.base + Q);
        sz = __shfl_sync(WHG_FULL_MASK, k, g.base + H);
    } else {
        sx = group_sum<L>(g, x);
        sy = group_sum<L>(g, y);
        sz = group_sum<L>(g, z);
    }
}

// Sums of m (x, y, z) over the system's lanes, the same bits in every lane.
// L = 4, 8: as group_sum3, with the products by the masses taken inside the
// first reduce-scatter round, where each kept component needs the partner's
// product and the lane's own one: m_p x_p + m_q x_q as one product and one
// FMA (2 products and 2 FMAs per lane for the two kept components, against 3
// products and 2 additions when every lane first forms its whole m x).
// Each partial sum is formed by one lane only, and the last round adds a
// pair's two values in both lanes (commutative), so every lane still ends
// with the same bits.
template <int L>
__device__ __forceinline__ void group_msum3(const Group<L>& g, double m, double x, double y, double z,
                                            double& sx, double& sy, double& sz)
{
    if (L == 4 || L == 8) {
        constexpr int H = L / 2, Q = L / 4;
        const bool hi = (g.p & H) != 0;          // keeps (z, 0), else (x, y)
        const double o0 = hi ? z : x, o1 = hi ? 0.0 : y;     // own values of the kept components
        const double s0 = hi ? x : z, s1 = hi ? y : 0.0;     // own values the partner keeps
        const double q0 = __shfl_xor_sync(WHG_FULL_MASK, s0, H);
        const double q1 = __shfl_xor_sync(WHG_FULL_MASK, s1, H);
        const double mq = __shfl_xor_sync(WHG_FULL_MASK, m, H);
        const double k0 = fma(m, o0, mq * q0);
        const double k1 = fma(m, o1, mq * q1);
        const bool mid = (g.p & Q) != 0;         // keeps the second of the pair
        double k = mid ? k1 : k0;
        k += __shfl_xor_sync(WHG_FULL_MASK, mid ? k0 : k1, Q);
        if (L == 8) k += __shfl_xor_sync(WHG_FULL_MASK, k, 1);
        sx = __shfl_sync(WHG_FULL_MASK, k, g.base);
        sy = __shfl_sync(WHG_FULL_MASK, k, g.base + Q);
        sz = __shfl_sync(WHG_FULL_MASK, k, g.base + H);
    } else {
        group_sum3<L>(g, m * x, m * y, m * z, sx, sy, sz);
    }
}

// Jump step (Sec. 3.4, Eq. 6): Q_i += (h/m0) sum_j m_j v_j; jc = h / m0.
template <int L>
__device__ __forceinline__ void jump(const Group<L>& g, double m, double jc, double vx, double vy,
                                     double vz, double& qx, double& qy, double& qz)
{
    double px, py, pz;
    group_msum3<L>(g, m, vx, vy, vz, px, py, pz);
    qx = fma(jc, px, qx);
    qy = fma(jc, py, qy);
    qz = fma(jc, pz, qz);
}

// Interaction kick (Sec. 3.3, Eq. 5) plus the GR term, for time dt, added
// straight into v; hm = dt m_i.  Pairs at cyclic lane distance k, 1 <= k <
// L/2, are evaluated once, by the lane at the lower end of the rotation, and
// the reaction is passed to the partner by a shuffle (Newton's third law);
// for even L the L/2 pairs at distance L/2 are evaluated by both of their
// lanes.  For L = 8 that is 4 reciprocal square roots per lane for the 28
// pairs, as in the paper, with rotations that cost the same on any lanes of a
// warp.  thr2[k-1] is the squared close-encounter distance of this lane's
// pair at distance k (0 when the rule is off); returns true if a pair it
// evaluates is closer (compared on the bit patterns of positive doubles, so
// no FP64 instruction is spent).
// `full` (uniform across the warp) selects the other schedule: all L-1
// rotations, every lane summing its own pairs with no reactions (each pair
// evaluated by both of its lanes: 7 reciprocal square roots per lane for
// L = 8); the close-encounter test then uses the distances k <= L/2, which
// cover every pair from one side.
// With GEOM (the adjoint's tape kernel), the factors of the kick's
// vector-Jacobian product that do not depend on the adjoints are written to
// kt: pair round r (partner j at distance k = r + 1 <= L/2, this lane i) at
// kt.p[(8r + n) kt.NL], n = 0..7: Q_j - Q_i (3), hm_j r^-3, hm_i r^-3,
// 3 hm_j r^-5, 3 hm_i r^-5, dt r^-3; the GR factors at kt.p[(32 + n) kt.NL]:
// c = kgr/|Q|^4, 4 c/|Q|^2, 2 c/m0.  The velocities come out the same.
struct KickTape {
    double* p;
    size_t NL;
    double dt, two_muinv;
};
constexpr int kKickTapeRound = 8;

template <bool GEOM>
__device__ __forceinline__ void kick_geom(const KickTape* kt, int round, double dx, double dy, double dz,
                                          double r2, double r3, double hmj, double hmi)
{
    if constexpr (GEOM) {
        double* t = kt->p + (size_t)(kKickTapeRound * round) * kt->NL;
        const double r5x3 = 3.0 * (r3 * rcp(r2));
        t[0] = dx;
        t[kt->NL] = dy;
        t[2 * kt->NL] = dz;
        t[3 * kt->NL] = hmj * r3;
        t[4 * kt->NL] = hmi * r3;
        t[5 * kt->NL] = hmj * r5x3;
        t[6 * kt->NL] = hmi * r5x3;
        t[7 * kt->NL] = kt->dt * r3;
    }
}

template <int L, int GRM, bool GEOM = false>
__device__ __forceinline__ bool kick(const Group<L>& g, double qx, double qy, double qz, double hm,
                                     double mrat, double kgr, const double* thr2, double& vx,
                                     double& vy, double& vz, bool full = false, const KickTape* kt = nullptr)
{
    bool close = false;
    if (full) {
#pragma unroll
        for (int k = 1; k < L; ++k) {
            const int to = g.at(k);
            const double dx = __shfl_sync(WHG_FULL_MASK, qx, to) - qx;
            const double dy = __shfl_sync(WHG_FULL_MASK, qy, to) - qy;
            const double dz = __shfl_sync(WHG_FULL_MASK, qz, to) - qz;
            const double hmj = __shfl_sync(WHG_FULL_MASK, hm, to);
            const double r2 = fma(dx, dx, fma(dy, dy, dz * dz));
            if (2 * k <= L) close |= __double_as_longlong(r2) < __double_as_longlong(thr2[k - 1]);
            const double r3 = rsqrt_cubed(r2);
            if (2 * k <= L) kick_geom<GEOM>(kt, k - 1, dx, dy, dz, r2, r3, hmj, hm);
            const double sj = hmj * r3;
            vx = fma(sj, dx, vx);
            vy = fma(sj, dy, vy);
            vz = fma(sj, dz, vz);
        }
    } else {
#pragma unroll
        for (int k = 1; 2 * k < L; ++k) {
            const int to = g.at(k), from = g.at(-k);
            const double dx = __shfl_sync(WHG_FULL_MASK, qx, to) - qx;   // Q_j - Q_i
            const double dy = __shfl_sync(WHG_FULL_MASK, qy, to) - qy;
            const double dz = __shfl_sync(WHG_FULL_MASK, qz, to) - qz;
            const double hmj = __shfl_sync(WHG_FULL_MASK, hm, to);
            const double r2 = fma(dx, dx, fma(dy, dy, dz * dz));
            close |= __double_as_longlong(r2) < __double_as_longlong(thr2[k - 1]);
            const double r3 = rsqrt_cubed(r2);
            kick_geom<GEOM>(kt, k - 1, dx, dy, dz, r2, r3, hmj, hm);
            const double sj = hmj * r3;
            vx = fma(sj, dx, vx);
            vy = fma(sj, dy, vy);
            vz = fma(sj, dz, vz);
            const double si = hm * r3;                    // reaction on j: -si (Q_j - Q_i)
            const double ex = __shfl_sync(WHG_FULL_MASK, dx, from);
            const double ey = __shfl_sync(WHG_FULL_MASK, dy, from);
            const double ez = __shfl_sync(WHG_FULL_MASK, dz, from);
            const double es = __shfl_sync(WHG_FULL_MASK, si, from);
            vx = fma(-es, ex, vx);
            vy = fma(-es, ey, vy);
            vz = fma(-es, ez, vz);
        }
        if (L >= 2 && (L & 1) == 0) {
            const int to = g.at(L / 2);
            const double dx = __shfl_sync(WHG_FULL_MASK, qx, to) - qx;
            const double dy = __shfl_sync(WHG_FULL_MASK, qy, to) - qy;
            const double dz = __shfl_sync(WHG_FULL_MASK, qz, to) - qz;
            const double hmj = __shfl_sync(WHG_FULL_MASK, hm, to);
            const double r2 = fma(dx, dx, fma(dy, dy, dz * dz));
            close |= __double_as_longlong(r2) < __double_as_longlong(thr2[L / 2 - 1]);
            const double r3 = rsqrt_cubed(r2);
            kick_geom<GEOM>(kt, L / 2 - 1, dx, dy, dz, r2, r3, hmj, hm);
            const double sj = hmj * r3;
            vx = fma(sj, dx, vx);
            vy = fma(sj, dy, vy);
            vz = fma(sj, dz, vz);
        }
    }
    if (GRM != 0) {
        // a_GR(Q) = -6 (G m0)^2 Q / (c^2 |Q|^4); kgr = -6 m0^2 dt / c^2.
        const double r2 = fma(qx, qx, fma(qy, qy, qz * qz));
        const double c = kgr * rcp_sq(r2);
        if constexpr (GEOM) {
            double* t = kt->p + (size_t)(4 * kKickTapeRound) * kt->NL;
            t[0] = c;
            t[kt->NL] = 4.0 * c * rcp(r2);
            t[2 * kt->NL] = c * kt->two_muinv;
        }
        if (GRM == 1) {
            vx = fma(c, qx, vx);
            vy = fma(c, qy, vy);
            vz = fma(c, qz, vz);
        } else {
            const double ax = c * qx, ay = c * qy, az = c * qz;
            double bx, by, bz;
            group_sum3<L>(g, mrat * ax, mrat * ay, mrat * az, bx, by, bz);
            vx = vx + (ax - bx);
            vy = vy + (ay - by);
            vz = vz + (az - bz);
        }
    }
    return close;
}

// Far-away parking spot of lanes without a planet: distinct, finite, fixed.
__device__ __forceinline__ double parked_x(int p) { return 1.0e6 * (double)(p + 1); }

// Where a warp's lanes live: bucket b, warp wb inside it, this lane's system.
template <int L>
struct Place {
    Group<L> g;
    int sys;             // internal system index (valid only if has_sys)
    bool has_sys;
    size_t lane;         // index into the lane arrays
    __device__ __forceinline__ Place(const WhgState& st, const WhgBuckets& bk, int b, int w)
    {
        const int sl = (w - bk.warp0[b]) * Group<L>::SPW + g.slot;
        has_sys = g.in_group && sl < bk.sys0[b + 1] - bk.sys0[b];
        sys = has_sys ? bk.sys0[b] + sl : 0;
        lane = (size_t)w * 32 + g.lane;
        WHG_CHECK(st, b >= 0 && b < bk.nb, WHG_BOUND_BUCKET);
        WHG_CHECK(st, (long long)lane < st.nl, WHG_BOUND_LANE);
        WHG_CHECK(st, !has_sys || (sys >= 0 && sys < st.S), WHG_BOUND_SYSTEM);
        (void)st;
    }
};

__device__ __forceinline__ int user_index(const WhgState& st, int sys)
{
    const int u = st.perm ? st.perm[sys] : sys;
    WHG_CHECK(st, sys >= 0 && sys < st.S && u >= 0 && u < st.S, WHG_BOUND_USER);
    return u;
}

// ------------------------------------------------------------------------
// Kernel bodies.  A warp belongs to one bucket; shuffles use the full warp
// mask, so no lane leaves a body before its last shuffle.

// Inertial -> DH (Sec. 3.1): Q_i = x_i - x_0, v_i = u_i - V_cm; M, X_cm, V_cm
// kept; initial osculating a_i (mu = G(m0 + m_i)) for the stop rules.
template <int L>
__device__ __forceinline__ void init_body(const WhgState& st, const WhgBuckets& bk, const WhgIn& in,
                                          int b, int w)
{
    const Place<L> pl(st, bk, b, w);
    const int p = pl.g.p;
    const size_t lane = pl.lane;
    int n = 0, ok = 0;
    double M = 0.0, xc[3] = {0.0, 0.0, 0.0}, vc[3] = {0.0, 0.0, 0.0}, m0 = 1.0, dt = 1.0e-3;
    double amax = 0.0, a_mine = 0.0;
    if (pl.has_sys) {
        const int u = user_index(st, pl.sys);
        const int B = 1 + st.Nmax;
        const double* ms = in.masses + (size_t)u * B;
        const double* xs = in.pos + (size_t)u * B * 3;
        const double* us = in.vel + (size_t)u * B * 3;
        n = in.nplan ? in.nplan[u] : st.Nmax;
        dt = in.dt[u];
        m0 = ms[0];
        ok = n >= 1 && n <= st.Nmax && n <= L && dt > 0.0 && is_finite(dt) && m0 > 0.0 &&
             is_finite(m0);
        if (ok) {
            for (int k = 0; k <= n; ++k) {
                M += ms[k];
                ok &= ms[k] >= 0.0 && is_finite(ms[k]);
                for (int c = 0; c < 3; ++c) {
                    ok &= is_finite(xs[3 * k + c]) && is_finite(us[3 * k + c]);
                    xc[c] += ms[k] * xs[3 * k + c];
                    vc[c] += ms[k] * us[3 * k + c];
                }
                if (k > 0) {
                    ok &= !(xs[3 * k] == xs[0] && xs[3 * k + 1] == xs[1] && xs[3 * k + 2] == xs[2]);
                    double r2 = 0.0, w2 = 0.0;
                    for (int c = 0; c < 3; ++c) {
                        const double dx = __dsub_rn(xs[3 * k + c], xs[c]);
                        const double du = __dsub_rn(us[3 * k + c], us[c]);
                        r2 = __dadd_rn(r2, __dmul_rn(dx, dx));
                        w2 = __dadd_rn(w2, __dmul_rn(du, du));
                    }
                    const double a = 1.0 / __dsub_rn(2.0 / sqrt(r2), w2 / __dadd_rn(m0, ms[k]));
                    amax = fmax(amax, a);
                    if (k == p + 1) a_mine = a;
                }
            }
            for (int c = 0; c < 3; ++c) {
                xc[c] /= M;
                vc[c] /= M;
            }
        }
        if (ok && p < n) {
            st.m[lane] = ms[1 + p];
            st.qx[lane] = xs[3 * (1 + p) + 0] - xs[0];
            st.qy[lane] = xs[3 * (1 + p) + 1] - xs[1];
            st.qz[lane] = xs[3 * (1 + p) + 2] - xs[2];
            st.vx[lane] = us[3 * (1 + p) + 0] - vc[0];
            st.vy[lane] = us[3 * (1 + p) + 1] - vc[1];
            st.vz[lane] = us[3 * (1 + p) + 2] - vc[2];
            st.a0[lane] = a_mine;
        }
    }
    if (!(ok && p < n)) {                            // no planet on this lane
        st.m[lane] = 0.0;
        st.qx[lane] = parked_x(p);
        st.qy[lane] = 0.0;
        st.qz[lane] = 0.0;
        st.vx[lane] = 0.0;
        st.vy[lane] = 0.0;
        st.vz[lane] = 0.0;
        st.a0[lane] = 0.0;
    }
    if (pl.has_sys && p == 0) {
        const int s = pl.sys;
        if (!ok) {
            m0 = 1.0;
            dt = 1.0e-3;
            M = 1.0;
        }
        st.m0[s] = m0;
        st.dt[s] = dt;
        st.M[s] = M;
        for (int c = 0; c < 3; ++c) {
            st.xcm[(size_t)c * st.S + s] = xc[c];
            st.vcm[(size_t)c * st.S + s] = vc[c];
        }
        const double rej = st.eject * amax;
        st.rej2[s] = (st.eject > 0.0 && ok && amax > 0.0) ? rej * rej : __longlong_as_double(0x7ff0000000000000LL);
        st.nplan[s] = ok ? n : 0;
        st.status[s] = ok ? 0 : WHG_STATUS_INVALID;
        st.nstep[s] = 0;
    }
}

// n Wisdom-Holman steps, state in registers (Eq. 2 with fused drifts).
// Load of state that other warps of the same launch may have written (the
// work queue moves a warp-group between SMs): through L2, bypassing a
// possibly stale L1 line.
template <bool COH, typename T>
__device__ __forceinline__ T ld_state(const T* p)
{
    if (COH) return __ldcg(p);
    return *p;
}

template <int L, int NT, int GRM, bool COH = false>
__device__ __forceinline__ void step_body(const WhgState& st, const WhgBuckets& bk, int b, int w,
                                          long long nsteps)
{
    const Place<L> pl(st, bk, b, w);
    const Group<L>& g = pl.g;
    const size_t lane = pl.lane;
    const int s = pl.sys;
    const double m = st.m[lane];
    double qx = ld_state<COH>(st.qx + lane), qy = ld_state<COH>(st.qy + lane), qz = ld_state<COH>(st.qz + lane);
    double vx = ld_state<COH>(st.vx + lane), vy = ld_state<COH>(st.vy + lane), vz = ld_state<COH>(st.vz + lane);
    const double mu = pl.has_sys ? st.m0[s] : 1.0;
    const double dt = pl.has_sys ? st.dt[s] : 1.0e-3;
    const int npl = pl.has_sys ? st.nplan[s] : 0;
    int status = pl.has_sys ? ld_state<COH>(st.status + s) : 0;
    const long long nstep0 = pl.has_sys ? ld_state<COH>(st.nstep + s) : 0;
    const double rej2 = pl.has_sys ? st.rej2[s] : 0.0;
    const bool real = pl.has_sys && g.p < npl;
    bool alive = pl.has_sys && status == 0;
    const double hm = dt * m;
    const double jc = (0.5 * dt) / mu;
    const double mrat = m / mu;
    const double kgr = GRM ? (-6.0 * mu * mu * dt) / (st.c_light * st.c_light) : 0.0;
    const bool h32 = st.halley32 != 0;
    const bool full = st.full_rotation != 0;
    // close-encounter distances of this lane's pairs (once per launch)
    double thr2[4] = {0.0, 0.0, 0.0, 0.0};
    {
        const double a = st.a0[lane];
#pragma unroll
        for (int k = 1; 2 * k <= L; ++k) {
            const int to = g.at(k);
            const double mj = __shfl_sync(WHG_FULL_MASK, m, to);
            const double aj = __shfl_sync(WHG_FULL_MASK, a, to);
            if (st.hill > 0.0 && k - 1 < 4) {
                const double rh = st.hill * cbrt((m + mj) / (3.0 * mu)) * 0.5 * (a + aj);
                thr2[k - 1] = rh * rh;
            }
        }
    }
    const unsigned gmask = g.mask();
    long long done = 0;
    for (long long k = 0; k < nsteps; ++k) {
        if (!__any_sync(WHG_FULL_MASK, alive)) break;        // whole warp frozen
        const double sqx = qx, sqy = qy, sqz = qz, svx = vx, svy = vy, svz = vz;
        const double hK = (nstep0 + done == 0) ? 0.5 * dt : dt;
        const double r0sq = fma(qx, qx, fma(qy, qy, qz * qz));
        const bool far = __double_as_longlong(r0sq) > __double_as_longlong(rej2);
        const bool bound = kepler_drift<NT>(mu, hK, qx, qy, qz, vx, vy, vz, h32);
        bool close;
        if (GRM == 0 && st.merge) {                   // J(dt) I(dt): J and I commute without GR
            jump<L>(g, m, 2.0 * jc, vx, vy, vz, qx, qy, qz);
            close = kick<L, GRM>(g, qx, qy, qz, hm, mrat, kgr, thr2, vx, vy, vz, full);
        } else {
            jump<L>(g, m, jc, vx, vy, vz, qx, qy, qz);
            close = kick<L, GRM>(g, qx, qy, qz, hm, mrat, kgr, thr2, vx, vy, vz, full);
            jump<L>(g, m, jc, vx, vy, vz, qx, qy, qz);
        }
        const bool fin = is_finite(qx) & is_finite(qy) & is_finite(qz) & is_finite(vx) &
                         is_finite(vy) & is_finite(vz);
        const unsigned bad_h = __ballot_sync(WHG_FULL_MASK, real && !bound) & gmask;
        const unsigned bad_n = __ballot_sync(WHG_FULL_MASK, real && !fin) & gmask;
        const unsigned bad_c = __ballot_sync(WHG_FULL_MASK, real && close) & gmask;
        const unsigned bad_e = __ballot_sync(WHG_FULL_MASK, real && far) & gmask;
        const bool ok = (bad_h | bad_n | bad_c | bad_e) == 0u;
        if (!(alive && real && ok)) {                 // roll back: no planet, frozen, failed
            qx = sqx; qy = sqy; qz = sqz;
            vx = svx; vy = svy; vz = svz;
        }
        if (alive && !ok) {
            status |= (bad_n ? WHG_STATUS_NONFINITE : 0) | (bad_h ? WHG_STATUS_HYPERBOLIC : 0) |
                      (bad_c ? WHG_STATUS_CLOSE_ENCOUNTER : 0) | (bad_e ? WHG_STATUS_EJECTED : 0);
            alive = false;
        }
        done += alive ? 1 : 0;
    }
    if (real) {
        st.qx[lane] = qx; st.qy[lane] = qy; st.qz[lane] = qz;
        st.vx[lane] = vx; st.vy[lane] = vy; st.vz[lane] = vz;
    }
    if (pl.has_sys && g.p == 0) {
        st.status[s] = status;
        st.nstep[s] = nstep0 + done;
    }
}

// Synchronized copy (pending K(dt/2)) -> inertial frame (Sec. 3.1 inverted):
// x_0 = X_cm + V_cm t - sum m_i Q_i / M, x_i = x_0 + Q_i,
// u_0 = V_cm - sum m_i v_i / m0, u_i = v_i + V_cm.  Caller's order and layout.
template <int L, int NT>
__device__ __forceinline__ void read_body(const WhgState& st, const WhgBuckets& bk, const WhgOut& out,
                                          int b, int w)
{
    const Place<L> pl(st, bk, b, w);
    const Group<L>& g = pl.g;
    const size_t lane = pl.lane;
    const int s = pl.sys;
    const double m = st.m[lane];
    double qx = st.qx[lane], qy = st.qy[lane], qz = st.qz[lane];
    double vx = st.vx[lane], vy = st.vy[lane], vz = st.vz[lane];
    const double mu = pl.has_sys ? st.m0[s] : 1.0;
    const double dt = pl.has_sys ? st.dt[s] : 1.0e-3;
    const long long ns = pl.has_sys ? st.nstep[s] : 0;
    if (ns > 0) kepler_drift<NT>(mu, 0.5 * dt, qx, qy, qz, vx, vy, vz, st.halley32 != 0);
    const double sqx = group_sum<L>(g, m * qx), sqy = group_sum<L>(g, m * qy), sqz = group_sum<L>(g, m * qz);
    const double spx = group_sum<L>(g, m * vx), spy = group_sum<L>(g, m * vy), spz = group_sum<L>(g, m * vz);
    if (!pl.has_sys) return;                         // after the last shuffle
    const int npl = st.nplan[s];
    const int u = user_index(st, s);
    const int B = 1 + st.Nmax;
    const double t = (double)ns * dt;
    const double M = st.M[s];
    const double sq[3] = {sqx, sqy, sqz}, sp[3] = {spx, spy, spz}, q[3] = {qx, qy, qz}, v[3] = {vx, vy, vz};
    double x0[3], u0[3], V[3];
    for (int c = 0; c < 3; ++c) {
        const double X = st.xcm[(size_t)c * st.S + s];
        V[c] = st.vcm[(size_t)c * st.S + s];
        x0[c] = (X + V[c] * t) - sq[c] / M;
        u0[c] = V[c] - sp[c] / mu;
    }
    for (int slot = g.p; slot < st.Nmax; slot += L) {    // planet slots of this lane
        const size_t o = ((size_t)u * B + 1 + slot) * 3;
        const bool live = slot == g.p && slot < npl;
        for (int c = 0; c < 3; ++c) {
            if (out.pos) out.pos[o + c] = live ? x0[c] + q[c] : 0.0;
            if (out.vel) out.vel[o + c] = live ? v[c] + V[c] : 0.0;
        }
    }
    if (g.p == 0) {
        const size_t o = (size_t)u * B * 3;
        for (int c = 0; c < 3; ++c) {
            if (out.pos) out.pos[o + c] = x0[c];
            if (out.vel) out.vel[o + c] = u0[c];
        }
        if (out.status) out.status[u] = st.status[s];
        if (out.t) out.t[u] = t;
    }
}

// Energy of the synchronized state: H_0 + H_K + H_I + H_J (Eq. 1) [+ GR].
template <int L, int NT, int GRM>
__device__ __forceinline__ void energy_body(const WhgState& st, const WhgBuckets& bk,
                                            const WhgOut& out, int b, int w)
{
    const Place<L> pl(st, bk, b, w);
    const Group<L>& g = pl.g;
    const size_t lane = pl.lane;
    const int s = pl.sys;
    const double m = st.m[lane];
    double qx = st.qx[lane], qy = st.qy[lane], qz = st.qz[lane];
    double vx = st.vx[lane], vy = st.vy[lane], vz = st.vz[lane];
    const double mu = pl.has_sys ? st.m0[s] : 1.0;
    const double dt = pl.has_sys ? st.dt[s] : 1.0e-3;
    if (pl.has_sys && st.nstep[s] > 0)
        kepler_drift<NT>(mu, 0.5 * dt, qx, qy, qz, vx, vy, vz, st.halley32 != 0);
    const double r2 = fma(qx, qx, fma(qy, qy, qz * qz));
    double pair = 0.0;
#pragma unroll
    for (int k = 1; k < L; ++k) {
        const int j = g.at(k);
        const double dx = __shfl_sync(WHG_FULL_MASK, qx, j) - qx;
        const double dy = __shfl_sync(WHG_FULL_MASK, qy, j) - qy;
        const double dz = __shfl_sync(WHG_FULL_MASK, qz, j) - qz;
        const double mj = __shfl_sync(WHG_FULL_MASK, m, j);
        pair += m * mj / sqrt(fma(dx, dx, fma(dy, dy, dz * dz)));
    }
    double part = 0.5 * m * fma(vx, vx, fma(vy, vy, vz * vz)) - mu * m / sqrt(r2) - 0.5 * pair;
    if (GRM != 0) part += -3.0 * m * mu * mu / (st.c_light * st.c_light * r2);
    const double tot = group_sum<L>(g, part);
    const double px = group_sum<L>(g, m * vx), py = group_sum<L>(g, m * vy), pz = group_sum<L>(g, m * vz);
    if (!pl.has_sys || g.p != 0) return;
    double h0 = 0.0;
    for (int c = 0; c < 3; ++c) {
        const double V = st.vcm[(size_t)c * st.S + s];
        h0 += 0.5 * st.M[s] * V * V;
    }
    out.E[user_index(st, s)] = h0 + tot + (px * px + py * py + pz * pz) / (2.0 * mu);
}

// Raw state copy between the lane arrays and the caller's [S][Nmax][3] layout.
template <int L>
__device__ __forceinline__ void raw_body(const WhgState& st, const WhgBuckets& bk, const WhgOut& io,
                                         int set, int b, int w)
{
    const Place<L> pl(st, bk, b, w);
    if (!pl.has_sys) return;                         // no shuffles in this body
    const size_t lane = pl.lane;
    const int s = pl.sys, p = pl.g.p;
    const int u = user_index(st, s);
    const int npl = st.nplan[s];
    for (int slot = p; slot < st.Nmax; slot += L) {
        const size_t o = ((size_t)u * st.Nmax + slot) * 3;
        const bool live = slot == p && slot < npl;
        if (set) {
            if (live) {
                st.qx[lane] = io.inQ[o]; st.qy[lane] = io.inQ[o + 1]; st.qz[lane] = io.inQ[o + 2];
                st.vx[lane] = io.inv[o]; st.vy[lane] = io.inv[o + 1]; st.vz[lane] = io.inv[o + 2];
            }
        } else {
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
            st.nstep[s] = io.inn[u];
            st.status[s] = io.ins[u];
        } else {
            io.rawn[u] = st.nstep[s];
            io.status[u] = st.status[s];
        }
    }
}

// ------------------------------------------------------------------------
// Bucket dispatch: the warp's bucket (warp-uniform), then its L instance.

__device__ __forceinline__ int warp_index() { return (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5); }

__device__ __forceinline__ int bucket_of(const WhgBuckets& bk, int w)
{
    int b = 0;
    while (b + 1 < bk.nb && w >= bk.warp0[b + 1]) ++b;
    return b;
}

#define WHG_DISPATCH_L(Lvar, CALL)          \
    switch (Lvar) {                         \
    case 1: { constexpr int L_ = 1; CALL; } break; \
    case 2: { constexpr int L_ = 2; CALL; } break; \
    case 3: { constexpr int L_ = 3; CALL; } break; \
    case 4: { constexpr int L_ = 4; CALL; } break; \
    case 5: { constexpr int L_ = 5; CALL; } break; \
    case 6: { constexpr int L_ = 6; CALL; } break; \
    case 7: { constexpr int L_ = 7; CALL; } break; \
    default: { constexpr int L_ = 8; CALL; } break; \
    }

template <int NT, int GRM>
__global__ void __launch_bounds__(WHG_MAX_BLOCK) k_step(WhgState st, WhgBuckets bk, long long n)
{
    const int w = warp_index();
    if (w >= bk.warp0[bk.nb]) return;                // whole warps beyond the last bucket
    const int b = bucket_of(bk, w);
    WHG_DISPATCH_L(bk.L[b], (step_body<L_, NT, GRM>(st, bk, b, w, n)))
}

__device__ __forceinline__ int ld_acquire_gpu(const int* p)
{
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release_gpu(int* p, int v)
{
    asm volatile("st.release.gpu.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}


// Work queue over warp-groups (no counterpart in the paper).  Unit
// u = k G + g advances warp-group g (one warp's worth of systems) by steps
// [k chunk, min(n, (k+1) chunk)).  Resident warps take units in increasing u
// from an atomic counter; unit (g, k) first waits until done[g] == k.  The
// smallest incomplete u always has its predecessor complete and is held by
// a running warp (a warp takes a unit only when it runs), so the queue
// always progresses.  Work thus moves between SMs and the launch ends within
// about one unit of the balanced time, whatever the warp count per SM.  A
// wait that exceeds q.spin_limit polls sets *err and ends the warp.
// One unit of the work queue, kept out of line so that its step loop is
// compiled as in k_step (the unit loop around it would otherwise keep the
// bucket table in local memory).
template <int L, int NT, int GRM>
__device__ __noinline__ void queue_unit(const WhgState& st, const WhgBuckets& bk, int b, int g, long long m)
{
    step_body<L, NT, GRM, true>(st, bk, b, g, m);
}

template <int NT, int GRM>
__global__ void __launch_bounds__(WHG_MAX_BLOCK) k_step_queue(WhgState st, WhgBuckets bk, long long n,
                                                             WhgQueue q)
{
    const int G = bk.warp0[bk.nb];
    const unsigned long long total = (unsigned long long)G * (unsigned long long)q.units;
    const int lane = (int)(threadIdx.x & 31u);
    for (;;) {
        unsigned long long u = 0;
        if (lane == 0) u = atomicAdd(q.next, 1ULL);
        u = __shfl_sync(WHG_FULL_MASK, u, 0);
        if (u >= total) return;
        const int k = (int)(u / (unsigned long long)G), g = (int)(u % (unsigned long long)G);
        WHG_CHECK(st, g >= 0 && g < G && k < q.units, WHG_BOUND_QUEUE);
        int ok = 1;
        if (lane == 0 && k > 0) {
            long long polls = 0;
            while (ld_acquire_gpu(q.done + g) < k) {
                if (++polls > q.spin_limit) {
                    atomicExch(q.err, 1);
                    ok = 0;
                    break;
                }
                __nanosleep(100);
            }
        }
        ok = __shfl_sync(WHG_FULL_MASK, ok, 0);
        if (!ok) return;
        if (k > 0) (void)ld_acquire_gpu(q.done + g);  // every lane acquires before reading the state
        const long long s0 = (long long)k * q.chunk;
        const long long m = n - s0 < q.chunk ? n - s0 : q.chunk;
        const int b = bucket_of(bk, g);
        WHG_DISPATCH_L(bk.L[b], (queue_unit<L_, NT, GRM>(st, bk, b, g, m)))
        __threadfence();                             // each lane's state stores, then the release
        __syncwarp();
        if (lane == 0) st_release_gpu(q.done + g, k + 1);
    }
}

template <int NT>
__global__ void __launch_bounds__(WHG_MAX_BLOCK) k_read(WhgState st, WhgBuckets bk, WhgOut out)
{
    const int w = warp_index();
    if (w >= bk.warp0[bk.nb]) return;
    const int b = bucket_of(bk, w);
    WHG_DISPATCH_L(bk.L[b], (read_body<L_, NT>(st, bk, out, b, w)))
}

template <int NT, int GRM>
__global__ void __launch_bounds__(WHG_MAX_BLOCK) k_energy(WhgState st, WhgBuckets bk, WhgOut out)
{
    const int w = warp_index();
    if (w >= bk.warp0[bk.nb]) return;
    const int b = bucket_of(bk, w);
    WHG_DISPATCH_L(bk.L[b], (energy_body<L_, NT, GRM>(st, bk, out, b, w)))
}

}  // namespace whg
