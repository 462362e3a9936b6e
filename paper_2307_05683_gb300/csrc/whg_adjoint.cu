// whg_adjoint.cu -- reverse-mode (adjoint) kernels of libwhg.
//
// Gradient of L_s = sum_i |Q_i(T) - target_i|^2 (heliocentric positions of the
// synchronized state after n steps, per system s) with respect to the initial
// inertial positions, velocities and masses.  The forward run keeps the state
// every K steps (checkpoints); the backward walks the segments in reverse:
// each segment's K steps are recomputed from its checkpoint while a per-step
// tape is written, then the vector-Jacobian products of J, I (+GR), J and K
// are applied step by step in reverse.  The tape holds, besides the state the
// products need, every part of them that does not depend on the adjoints
// (pair separations and powers of 1/r, the GR factors, the Kepler drift's
// coefficients), so that the back kernels, which run one after another and
// form the critical path, do only the work linear in the adjoints.  The tape
// kernels run beside them: on two side streams, segments s-1 and s-2 while the
// products of segment s run, or, with the host's SM split, on SMs of their own
// during the forward half (see whg_api.cu).
//
// VJPs, with lambda the adjoint of each quantity:
//   J:  Q_i += c sum_j m_j v_j (c = (dt/2)/m0): lambda_v_j += c m_j Lambda,
//       lambda_m_j += c v_j.Lambda, lambda_m0 -= (c/m0) P.Lambda, Lambda =
//       sum_i lambda_Q_i;
//   I:  a pair term r^-3 (hm_j lambda_v_i - hm_i lambda_v_j).d with d = Q_j - Q_i
//       gives lambda_d = r^-3 w - 3 (w.d) r^-5 d, w = hm_j lambda_v_i -
//       hm_i lambda_v_j (hm = dt m), and mass terms dt r^-3 lambda_v.d;
//   GR: v += k Q/|Q|^4, k = -6 m0^2 dt/c^2: lambda_Q += k (lambda_v/r^4 -
//       4 (Q.lambda_v) Q/r^6), lambda_m0 += 2 (k/m0) (Q.lambda_v)/r^4;
//   K:  the Kepler flow through the implicit function theorem at the final X
//       (F(X) = r0 G1 + eta0 G2 + mu G3 - h = 0, F'(X) = r), with
//       dG_n/dX = G_{n-1}, dG_0/dX = -beta G_1 and
//       dG_n/dbeta = (n G_{n+2} - X G_{n+1}) / 2.
// The fixed-iteration solver converges to machine precision inside its domain,
// so the derivative of the converged flow is the derivative of the map.
#include "whg_device.cuh"

namespace whg {

// c_N(z) by its T-term series (Horner), N = 2..5.
template <int N, int K>
struct CnHorner {
    static __device__ __forceinline__ double run(double z, double acc)
    {
        return CnHorner<N, K - 1>::run(z, fma(-z, acc, 1.0 / Factorial<N + 2 * K>::value));
    }
};
template <int N>
struct CnHorner<N, -1> {
    static __device__ __forceinline__ double run(double, double acc) { return acc; }
};
template <int N, int T>
__device__ __forceinline__ double stumpff_c(double z)
{
    return CnHorner<N, T - 2>::run(z, 1.0 / Factorial<N + 2 * (T - 1)>::value);
}

// Adjoint of one Kepler drift (Q0, v0) -> (Q1, v1) for time h, mu = G m0,
// final universal variable X, split into the part that depends only on the
// state (KeplerCoef, computed by the tape kernel off the critical path) and
// the part linear in the adjoints (kepler_vjp_apply, run by the back kernel).
//
// c4, c5 come from their NT-term series and c2 = 1/2 - z c4, c3 = 1/6 - z c5
// from the recurrence: the same series through z^NT that the forward drift
// sums.  Every Lagrange coefficient is mu times a function of the G_n, so the
// adjoints of mu, r, r0 and G_n are written with f - 1, fdot and gdot - 1
// themselves:
//   mub  = ((f-1) fb + fdot fdb + (gdot-1) gdb) / mu - G3 gb,
//   rb   = -((fdot fdb + (gdot-1) gdb) / r,   r0b = -((f-1) fb + fdot fdb) / r0,
//   G1b  = -(mu / (r r0)) fdb,  G2b = -(mu / r0) fb - (mu / r) gdb,  G3b = -mu gb,
// with fb = lq.Q0, gb = lq.v0, fdb = lv.Q0, gdb = lv.v0.
struct KeplerCoef {
    double f, fd, g, gd, fm1, gdm1;      // Lagrange coefficients (and f - 1, gdot - 1)
    double G0, G1, G2, G3;               // Stiefel functions at the final X
    double ri, r0i, r0, eta0;            // 1/r, 1/r0, r0, Q0.v0
    double A, B, C, Ar0i;                // mu/r0, mu/r, mu/(r r0), mu/r0^2
    double bG1;                          // beta G1
    double dG0, dG1, dG2, dG3;           // dG_n/dbeta
    double dF;                           // dF/dbeta = r0 dG1 + eta0 dG2 + mu dG3
};
constexpr int kKeplerCoefs = 24;

template <int NT>
__device__ __forceinline__ KeplerCoef kepler_vjp_coef(double mu, double h, double qx, double qy, double qz,
                                                      double vx, double vy, double vz, double X)
{
    KeplerCoef k;
    const double r0sq = fma(qx, qx, fma(qy, qy, qz * qz));
    k.r0i = rsqrt(r0sq);
    k.r0 = r0sq * k.r0i;
    k.eta0 = fma(qx, vx, fma(qy, vy, qz * vz));
    const double v2 = fma(vx, vx, fma(vy, vy, vz * vz));
    const double beta = fma(2.0 * mu, k.r0i, -v2);
    const double X2 = X * X, X4 = X2 * X2;
    const double z = beta * X2;
    const double c4 = stumpff_c<4, NT>(z), c5 = stumpff_c<5, NT>(z);
    const double c2 = fma(-z, c4, 0.5), c3 = fma(-z, c5, 1.0 / 6.0);
    k.G2 = X2 * c2;
    k.G3 = (X2 * X) * c3;
    const double G4 = X4 * c4, G5 = (X4 * X) * c5;
    k.G0 = fma(-beta, k.G2, 1.0);
    k.G1 = fma(-beta, k.G3, X);
    const double r = fma(k.r0, k.G0, fma(k.eta0, k.G1, mu * k.G2));
    k.ri = rcp(r);
    k.A = mu * k.r0i;
    k.B = mu * k.ri;
    k.C = k.A * k.ri;
    k.Ar0i = k.A * k.r0i;
    k.fm1 = -k.A * k.G2;
    k.g = fma(-mu, k.G3, h);
    k.fd = -k.C * k.G1;
    k.gdm1 = -k.B * k.G2;
    k.f = 1.0 + k.fm1;
    k.gd = 1.0 + k.gdm1;
    k.bG1 = beta * k.G1;
    // dG_n/dbeta = (n G_{n+2} - X G_{n+1}) / 2
    const double hX = 0.5 * X;
    k.dG0 = -hX * k.G1;
    k.dG1 = fma(-hX, k.G2, 0.5 * k.G3);
    k.dG2 = fma(-hX, k.G3, G4);
    k.dG3 = fma(-hX, G4, 1.5 * G5);
    k.dF = fma(k.r0, k.dG1, fma(k.eta0, k.dG2, mu * k.dG3));
    return k;
}

// The same coefficients from the values the forward drift computed anyway
// (prologue, G1..G3 at the final X, 1/r and the Lagrange coefficients): only
// the c4, c5 series for dG_n/dbeta are added.
template <int NT>
__device__ __forceinline__ KeplerCoef kepler_vjp_coef(double mu, double X, const DriftVals& dv)
{
    KeplerCoef k;
    k.r0i = dv.r0i;
    k.r0 = dv.r0;
    k.eta0 = dv.eta0;
    const double beta = dv.beta;
    k.G1 = dv.G1;
    k.G2 = dv.G2;
    k.G3 = dv.G3;
    k.G0 = fma(-beta, k.G2, 1.0);
    k.ri = dv.ri;
    k.A = dv.A;
    k.B = mu * k.ri;
    k.C = k.A * k.ri;
    k.Ar0i = k.A * k.r0i;
    k.fm1 = dv.fm1;
    k.g = dv.g;
    k.fd = dv.fd;
    k.gdm1 = dv.gdm1;
    k.f = 1.0 + k.fm1;
    k.gd = 1.0 + k.gdm1;
    k.bG1 = beta * k.G1;
    const double X2 = X * X, X4 = X2 * X2;
    const double z = beta * X2;
    const double G4 = X4 * stumpff_c<4, NT>(z), G5 = (X4 * X) * stumpff_c<5, NT>(z);
    const double hX = 0.5 * X;
    k.dG0 = -hX * k.G1;
    k.dG1 = fma(-hX, k.G2, 0.5 * k.G3);
    k.dG2 = fma(-hX, k.G3, G4);
    k.dG3 = fma(-hX, G4, 1.5 * G5);
    k.dF = fma(k.r0, k.dG1, fma(k.eta0, k.dG2, mu * k.dG3));
    return k;
}

// In: lq, lv = adjoints of Q1, v1.  Out: lq, lv = adjoints of Q0, v0; lmu
// accumulates the adjoint of mu.
__device__ __forceinline__ void kepler_vjp_apply(const KeplerCoef& k, double mu, double muinv, double qx,
                                                 double qy, double qz, double vx, double vy, double vz,
                                                 double& lqx, double& lqy, double& lqz, double& lvx,
                                                 double& lvy, double& lvz, double& lmu)
{
    // (a) outputs Q1 = f Q0 + g v0, v1 = fd Q0 + gd v0
    const double fb = fma(lqx, qx, fma(lqy, qy, lqz * qz));
    const double gb = fma(lqx, vx, fma(lqy, vy, lqz * vz));
    const double fdb = fma(lvx, qx, fma(lvy, qy, lvz * qz));
    const double gdb = fma(lvx, vx, fma(lvy, vy, lvz * vz));
    double nqx = fma(k.f, lqx, k.fd * lvx), nqy = fma(k.f, lqy, k.fd * lvy), nqz = fma(k.f, lqz, k.fd * lvz);
    double nvx = fma(k.g, lqx, k.gd * lvx), nvy = fma(k.g, lqy, k.gd * lvy), nvz = fma(k.g, lqz, k.gd * lvz);
    // (b) through f, g, fd, gd
    const double tf = k.fm1 * fb, tfd = k.fd * fdb, tgd = k.gdm1 * gdb;
    double mub = fma(tf + tfd + tgd, muinv, -k.G3 * gb);
    const double rb = -(tfd + tgd) * k.ri;
    double r0b = -(tf + tfd) * k.r0i;
    double G1b = -k.C * fdb;
    double G2b = fma(-k.A, fb, -k.B * gdb);
    const double G3b = -mu * gb;
    // (c) r = r0 G0 + eta0 G1 + mu G2
    r0b = fma(rb, k.G0, r0b);
    double eta0b = rb * k.G1;
    mub = fma(rb, k.G2, mub);
    const double G0b = rb * k.r0;
    G1b = fma(rb, k.eta0, G1b);
    G2b = fma(rb, mu, G2b);
    // (d) G_n(beta, X): dG_n/dX = G_{n-1}, dG_0/dX = -beta G1
    const double Xb = fma(-G0b, k.bG1, fma(G1b, k.G0, fma(G2b, k.G1, G3b * k.G2)));
    double betab = fma(G0b, k.dG0, fma(G1b, k.dG1, fma(G2b, k.dG2, G3b * k.dG3)));
    // (e) X implicit in F = r0 G1 + eta0 G2 + mu G3 - h = 0, dF/dX = r
    const double w = Xb * k.ri;
    r0b = fma(-w, k.G1, r0b);
    eta0b = fma(-w, k.G2, eta0b);
    mub = fma(-w, k.G3, mub);
    betab = fma(-w, k.dF, betab);
    // (f) beta = 2 mu / r0 - v.v, eta0 = Q.v, r0 = |Q|
    const double b2 = 2.0 * betab;
    mub = fma(b2, k.r0i, mub);
    r0b = fma(-b2, k.Ar0i, r0b);
    const double rq = r0b * k.r0i;
    nvx = fma(-b2, vx, fma(eta0b, qx, nvx));
    nvy = fma(-b2, vy, fma(eta0b, qy, nvy));
    nvz = fma(-b2, vz, fma(eta0b, qz, nvz));
    nqx = fma(eta0b, vx, fma(rq, qx, nqx));
    nqy = fma(eta0b, vy, fma(rq, qy, nqy));
    nqz = fma(eta0b, vz, fma(rq, qz, nqz));
    lqx = nqx; lqy = nqy; lqz = nqz;
    lvx = nvx; lvy = nvy; lvz = nvz;
    lmu += mub;
}

template <int NT>
__device__ __forceinline__ void kepler_vjp(double mu, double muinv, double h, double qx, double qy,
                                           double qz, double vx, double vy, double vz, double X,
                                           double& lqx, double& lqy, double& lqz, double& lvx,
                                           double& lvy, double& lvz, double& lmu)
{
    const KeplerCoef k = kepler_vjp_coef<NT>(mu, h, qx, qy, qz, vx, vy, vz, X);
    kepler_vjp_apply(k, mu, muinv, qx, qy, qz, vx, vy, vz, lqx, lqy, lqz, lvx, lvy, lvz, lmu);
}

// Adjoint of a jump Q_i += c sum_j m_j v_j with the velocities (vx, vy, vz)
// it used; lambda_Q passes through unchanged.  cmu = c / m0.
template <int L>
__device__ __forceinline__ void jump_vjp(const Group<L>& g, double m, double c, double cmu, double vx,
                                         double vy, double vz, double lqx, double lqy, double lqz,
                                         double& lvx, double& lvy, double& lvz, double& lm, double& lmu)
{
    double Lx, Ly, Lz;
    group_sum3<L>(g, lqx, lqy, lqz, Lx, Ly, Lz);
    const double cm = c * m;
    lvx = fma(cm, Lx, lvx);
    lvy = fma(cm, Ly, lvy);
    lvz = fma(cm, Lz, lvz);
    const double vd = fma(vx, Lx, fma(vy, Ly, vz * Lz));
    lm = fma(c, vd, lm);
    lmu = fma(-cmu * m, vd, lmu);
}

// Hint that the line holding *p will be read soon: fetched into L2, no
// register written and no fault on any address.
__device__ __forceinline__ void prefetch_l2(const double* p)
{
    asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

// Tape layout: per lane and step, WHG_TAPE_W doubles at stride NL.  Besides
// the state the back kernel needs (velocities for the jumps, positions for
// the GR term, the drift input), the tape holds everything of the kick and
// drift VJPs that does not depend on the adjoints, computed by the tape
// kernel: per pair round the separation d = Q_j - Q_i, r^-3, 3 r^-5 and
// dt r^-3, the GR factors, and the Kepler coefficients.
constexpr int kTV3 = 0;        // v after the kick (input of the second jump)
constexpr int kTQ2 = 3;        // Q during the kick
constexpr int kTRound = 6;     // 4 rounds x 8 pair factors (see KickTape), written by kick()
constexpr int kTGR = 38;       // c = kgr/|Q|^4, 4 c/|Q|^2, 2 c/m0, written by kick()
constexpr int kTV1 = 41;       // v after the drift (input of the first jump)
constexpr int kTQ0 = 44;       // drift input Q0
constexpr int kTV0 = 47;       // drift input v0
constexpr int kTKC = 50;       // KeplerCoef
static_assert(kTKC + kKeplerCoefs == WHG_TAPE_W, "tape layout");
static_assert(kTGR == kTRound + 4 * kKickTapeRound, "kick() writes its GR factors after 4 rounds");

// Adjoint of the interaction kick (+GR) from the tape, with lambda_v the
// adjoint of the velocities after it (which pass through unchanged).  Per
// pair (d = Q_j - Q_i, a = lambda_v_i.d, b = lambda_v_j.d):
//   lambda_d = hm_j r^-3 lambda_v_i - hm_i r^-3 lambda_v_j - s d,
//   s = 3 r^-5 (hm_j a - hm_i b), lambda_Q_j += lambda_d, lambda_Q_i -= lambda_d,
//   lambda_m_i -= dt r^-3 b, lambda_m_j += dt r^-3 a.
template <int L, int GRM>
__device__ __forceinline__ void kick_vjp(const Group<L>& g, const double* tp, size_t NL, double qx, double qy,
                                         double qz, double m, double hm, double muinv, double lvx,
                                         double lvy, double lvz, double& lqx, double& lqy, double& lqz,
                                         double& lm, double& lmu)
{
    (void)hm;
#pragma unroll
    for (int k = 1; 2 * k < L; ++k) {
        const int to = g.at(k), from = g.at(-k);
        const double* t = tp + (size_t)(kTRound + kKickTapeRound * (k - 1)) * NL;
        const double dx = t[0], dy = t[NL], dz = t[2 * NL];
        const double p3j = t[3 * NL], p3i = t[4 * NL], p5j = t[5 * NL], p5i = t[6 * NL], dtr3 = t[7 * NL];
        const double ljx = __shfl_sync(WHG_FULL_MASK, lvx, to);
        const double ljy = __shfl_sync(WHG_FULL_MASK, lvy, to);
        const double ljz = __shfl_sync(WHG_FULL_MASK, lvz, to);
        const double a = fma(lvx, dx, fma(lvy, dy, lvz * dz));
        const double b = fma(ljx, dx, fma(ljy, dy, ljz * dz));
        const double sd = fma(p5j, a, -p5i * b);
        const double ldx = fma(p3j, lvx, fma(-p3i, ljx, -sd * dx));
        const double ldy = fma(p3j, lvy, fma(-p3i, ljy, -sd * dy));
        const double ldz = fma(p3j, lvz, fma(-p3i, ljz, -sd * dz));
        lqx -= ldx;
        lqy -= ldy;
        lqz -= ldz;
        lm = fma(-dtr3, b, lm);
        const double lmj = dtr3 * a;                  // for the partner
        lqx += __shfl_sync(WHG_FULL_MASK, ldx, from);
        lqy += __shfl_sync(WHG_FULL_MASK, ldy, from);
        lqz += __shfl_sync(WHG_FULL_MASK, ldz, from);
        lm += __shfl_sync(WHG_FULL_MASK, lmj, from);
    }
    if (L >= 2 && (L & 1) == 0) {                     // both lanes of each pair evaluate it
        const int to = g.at(L / 2);
        const double* t = tp + (size_t)(kTRound + kKickTapeRound * (L / 2 - 1)) * NL;
        const double dx = t[0], dy = t[NL], dz = t[2 * NL];
        const double p3j = t[3 * NL], p5j = t[5 * NL], dtr3 = t[7 * NL];
        const double a = fma(lvx, dx, fma(lvy, dy, lvz * dz));
        const double sd = p5j * a;
        const double ldx = fma(p3j, lvx, -sd * dx);
        const double ldy = fma(p3j, lvy, -sd * dy);
        const double ldz = fma(p3j, lvz, -sd * dz);
        lqx -= ldx;
        lqy -= ldy;
        lqz -= ldz;
        const double lmj = dtr3 * a;
        lqx += __shfl_sync(WHG_FULL_MASK, ldx, to);
        lqy += __shfl_sync(WHG_FULL_MASK, ldy, to);
        lqz += __shfl_sync(WHG_FULL_MASK, ldz, to);
        lm += __shfl_sync(WHG_FULL_MASK, lmj, to);
    }
    if (GRM != 0) {
        const double c = tp[kTGR * NL], c4r = tp[(kTGR + 1) * NL], c2mu = tp[(kTGR + 2) * NL];
        double ax = lvx, ay = lvy, az = lvz;             // adjoint of this planet's a_GR
        if (GRM == 2) {
            double Lx, Ly, Lz;
            group_sum3<L>(g, lvx, lvy, lvz, Lx, Ly, Lz);
            const double aL = c * fma(qx, Lx, fma(qy, Ly, qz * Lz));   // a_i . Lambda_v
            lm = fma(-aL, muinv, lm);
            lmu = fma(m * aL, muinv * muinv, lmu);
            const double mr = m * muinv;
            ax = fma(-mr, Lx, ax);
            ay = fma(-mr, Ly, ay);
            az = fma(-mr, Lz, az);
        }
        const double s = fma(qx, ax, fma(qy, ay, qz * az));
        const double c4 = c4r * s;
        lqx += fma(c, ax, -c4 * qx);
        lqy += fma(c, ay, -c4 * qy);
        lqz += fma(c, az, -c4 * qz);
        lmu = fma(c2mu, s, lmu);
    }
}

// ------------------------------------------------------------------------
// Kernel bodies.

// Copy the live lane state (Q, v) into checkpoint slot `slot`.
template <int L>
__device__ __forceinline__ void save_body(const WhgState& st, const WhgAdj& adj, int slot, int w)
{
    const size_t lane = (size_t)w * 32 + (threadIdx.x & 31u);
    double* c = adj.ckpt + (size_t)slot * 6 * adj.NL;
    c[0 * adj.NL + lane] = st.qx[lane];
    c[1 * adj.NL + lane] = st.qy[lane];
    c[2 * adj.NL + lane] = st.qz[lane];
    c[3 * adj.NL + lane] = st.vx[lane];
    c[4 * adj.NL + lane] = st.vy[lane];
    c[5 * adj.NL + lane] = st.vz[lane];
}

// Loss of every system from the live (final) state, and with `start` set the
// adjoint of the final state: lambda_Q = 2 w (Q_sync - T) pulled back through
// the pending synchronizing K(dt/2).
template <int L, int NT>
__device__ __forceinline__ void loss_body(const WhgState& st, const WhgBuckets& bk, const WhgAdj& adj,
                                          int b, int w, int start)
{
    const Place<L> pl(st, bk, b, w);
    const Group<L>& g = pl.g;
    const size_t lane = pl.lane;
    const int s = pl.sys;
    const double qx = st.qx[lane], qy = st.qy[lane], qz = st.qz[lane];
    const double vx = st.vx[lane], vy = st.vy[lane], vz = st.vz[lane];
    const double mu = pl.has_sys ? st.m0[s] : 1.0;
    const double dt = pl.has_sys ? st.dt[s] : 1.0e-3;
    const long long ns = pl.has_sys ? st.nstep[s] : 0;
    const bool real = pl.has_sys && g.p < st.nplan[s];
    double sx = qx, sy = qy, sz = qz, svx = vx, svy = vy, svz = vz, X = 0.0;
    if (ns > 0) kepler_drift<NT>(mu, 0.5 * dt, sx, sy, sz, svx, svy, svz, X, st.halley32 != 0);
    const int u = pl.has_sys ? user_index(st, s) : 0;
    double ex = 0.0, ey = 0.0, ez = 0.0;
    if (real) {
        const double* T = adj.target + ((size_t)u * st.Nmax + g.p) * 3;
        ex = sx - T[0];
        ey = sy - T[1];
        ez = sz - T[2];
    }
    const double tot = group_sum<L>(g, ex * ex + ey * ey + ez * ez);
    if (!start) {
        if (pl.has_sys && g.p == 0) adj.loss[u] = tot;
        return;
    }
    const double wgt = (pl.has_sys && adj.weight) ? adj.weight[u] : 1.0;
    double lqx = 2.0 * wgt * ex, lqy = 2.0 * wgt * ey, lqz = 2.0 * wgt * ez;
    double lvx = 0.0, lvy = 0.0, lvz = 0.0, lmu = 0.0;
    if (ns > 0)
        kepler_vjp<NT>(mu, 1.0 / mu, 0.5 * dt, qx, qy, qz, vx, vy, vz, X, lqx, lqy, lqz, lvx, lvy, lvz, lmu);
    if (!real) {
        lqx = lqy = lqz = lvx = lvy = lvz = lmu = 0.0;
    }
    double* lam = adj.lam;
    lam[0 * adj.NL + lane] = lqx;
    lam[1 * adj.NL + lane] = lqy;
    lam[2 * adj.NL + lane] = lqz;
    lam[3 * adj.NL + lane] = lvx;
    lam[4 * adj.NL + lane] = lvy;
    lam[5 * adj.NL + lane] = lvz;
    lam[6 * adj.NL + lane] = 0.0;                    // lambda_m
    lam[7 * adj.NL + lane] = lmu;                    // lambda_m0 (partial, summed over lanes)
}

// Tape of one segment: its steps recomputed from the checkpoint (bitwise the
// forward's arithmetic), writing per step the tape fields listed above.
template <int L, int NT, int GRM>
__device__ __forceinline__ void tape_body(const WhgState& st, const WhgBuckets& bk, const WhgAdj& adj,
                                          int b, int w, int seg, long long s0, int nk, int buf)
{
    const Place<L> pl(st, bk, b, w);
    const Group<L>& g = pl.g;
    const size_t lane = pl.lane;
    const int s = pl.sys;
    const size_t NL = adj.NL;
    const double m = st.m[lane];
    const double mu = pl.has_sys ? st.m0[s] : 1.0;
    const double dt = pl.has_sys ? st.dt[s] : 1.0e-3;
    const bool real = pl.has_sys && g.p < st.nplan[s];
    const double hm = dt * m, c = (0.5 * dt) / mu, mrat = m / mu;
    const double kgr = GRM ? (-6.0 * mu * mu * dt) / (st.c_light * st.c_light) : 0.0;
    const double* ck = adj.ckpt + (size_t)seg * 6 * NL;
    double qx = ck[0 * NL + lane], qy = ck[1 * NL + lane], qz = ck[2 * NL + lane];
    double vx = ck[3 * NL + lane], vy = ck[4 * NL + lane], vz = ck[5 * NL + lane];
    const double pqx = qx, pqy = qy, pqz = qz, pvx = vx, pvy = vy, pvz = vz;
    const double nothr[4] = {0.0, 0.0, 0.0, 0.0};
    double* tape = adj.tape + (size_t)buf * adj.tape_len;
    for (int k = 0; k < nk; ++k) {
        double* tp = tape + (size_t)k * WHG_TAPE_W * NL + lane;
        tp[kTQ0 * NL] = qx; tp[(kTQ0 + 1) * NL] = qy; tp[(kTQ0 + 2) * NL] = qz;
        tp[kTV0 * NL] = vx; tp[(kTV0 + 1) * NL] = vy; tp[(kTV0 + 2) * NL] = vz;
        const double h = (s0 + k == 0) ? 0.5 * dt : dt;
        double X;
        DriftVals dv;
        kepler_drift<NT, true>(mu, h, qx, qy, qz, vx, vy, vz, X, st.halley32 != 0, &dv);
        {
            const KeplerCoef kc = kepler_vjp_coef<NT>(mu, X, dv);
            const double* kv = reinterpret_cast<const double*>(&kc);
#pragma unroll
            for (int i = 0; i < kKeplerCoefs; ++i) tp[(kTKC + i) * NL] = kv[i];
        }
        tp[kTV1 * NL] = vx; tp[(kTV1 + 1) * NL] = vy; tp[(kTV1 + 2) * NL] = vz;
        const bool merged = GRM == 0 && st.merge;
        jump<L>(g, m, merged ? 2.0 * c : c, vx, vy, vz, qx, qy, qz);
        tp[kTQ2 * NL] = qx; tp[(kTQ2 + 1) * NL] = qy; tp[(kTQ2 + 2) * NL] = qz;
        const KickTape kt{tp + (size_t)kTRound * NL, NL, dt, 2.0 / mu};
        kick<L, GRM, true>(g, qx, qy, qz, hm, mrat, kgr, nothr, vx, vy, vz, st.full_rotation != 0, &kt);
        tp[kTV3 * NL] = vx; tp[(kTV3 + 1) * NL] = vy; tp[(kTV3 + 2) * NL] = vz;
        if (!merged) jump<L>(g, m, c, vx, vy, vz, qx, qy, qz);
        if (!real) {                                  // lanes without a planet stay parked
            qx = pqx; qy = pqy; qz = pqz;
            vx = pvx; vy = pvy; vz = pvz;
        }
    }
}

// Pull the adjoint back through the steps of one segment, last step first,
// from tape buffer `buf`.  Only the work linear in the adjoints runs here:
// the back kernels of consecutive segments form the critical path, while the
// tape kernels run beside them.
template <int L, int NT, int GRM>
__device__ __forceinline__ void back_body(const WhgState& st, const WhgBuckets& bk, const WhgAdj& adj,
                                          int b, int w, long long s0, int nk, int buf)
{
    const Place<L> pl(st, bk, b, w);
    const Group<L>& g = pl.g;
    const size_t lane = pl.lane;
    const int s = pl.sys;
    const size_t NL = adj.NL;
    const double m = st.m[lane];
    const double mu = pl.has_sys ? st.m0[s] : 1.0;
    const double dt = pl.has_sys ? st.dt[s] : 1.0e-3;
    const bool real = pl.has_sys && g.p < st.nplan[s];
    const double hm = dt * m, c = (0.5 * dt) / mu, muinv = 1.0 / mu, cmu = c * muinv;
    const double* tape = adj.tape + (size_t)buf * adj.tape_len;
    double* lam = adj.lam;
    double lqx = lam[0 * NL + lane], lqy = lam[1 * NL + lane], lqz = lam[2 * NL + lane];
    double lvx = lam[3 * NL + lane], lvy = lam[4 * NL + lane], lvz = lam[5 * NL + lane];
    double lm = lam[6 * NL + lane], lmu = lam[7 * NL + lane];
    for (int k = nk - 1; k >= 0; --k) {
        const double* tp = tape + (size_t)k * WHG_TAPE_W * NL + lane;
        if (k >= 2) {                                 // this step's fields two steps ahead, into L2
            const double* pf = tp - (size_t)2 * WHG_TAPE_W * NL;
#pragma unroll
            for (int f = 0; f < WHG_TAPE_W; ++f) prefetch_l2(pf + (size_t)f * NL);
        }
        const bool merged = GRM == 0 && st.merge;
        if (!merged)
            jump_vjp<L>(g, m, c, cmu, tp[kTV3 * NL], tp[(kTV3 + 1) * NL], tp[(kTV3 + 2) * NL], lqx, lqy, lqz,
                        lvx, lvy, lvz, lm, lmu);
        kick_vjp<L, GRM>(g, tp, NL, tp[kTQ2 * NL], tp[(kTQ2 + 1) * NL], tp[(kTQ2 + 2) * NL], m, hm, muinv,
                         lvx, lvy, lvz, lqx, lqy, lqz, lm, lmu);
        const double cj = merged ? 2.0 * c : c;
        jump_vjp<L>(g, m, cj, cj * muinv, tp[kTV1 * NL], tp[(kTV1 + 1) * NL], tp[(kTV1 + 2) * NL], lqx, lqy,
                    lqz, lvx, lvy, lvz, lm, lmu);
        KeplerCoef kc;
        double* kv = reinterpret_cast<double*>(&kc);
#pragma unroll
        for (int i = 0; i < kKeplerCoefs; ++i) kv[i] = tp[(kTKC + i) * NL];
        kepler_vjp_apply(kc, mu, muinv, tp[kTQ0 * NL], tp[(kTQ0 + 1) * NL], tp[(kTQ0 + 2) * NL], tp[kTV0 * NL],
                         tp[(kTV0 + 1) * NL], tp[(kTV0 + 2) * NL], lqx, lqy, lqz, lvx, lvy, lvz, lmu);
        if (!real) {
            lqx = lqy = lqz = lvx = lvy = lvz = lm = lmu = 0.0;
        }
    }
    lam[0 * NL + lane] = lqx; lam[1 * NL + lane] = lqy; lam[2 * NL + lane] = lqz;
    lam[3 * NL + lane] = lvx; lam[4 * NL + lane] = lvy; lam[5 * NL + lane] = lvz;
    lam[6 * NL + lane] = lm; lam[7 * NL + lane] = lmu;
}

// Pull the adjoint at step 0 back through the inertial -> DH transform and
// write the gradients in the caller's layout (NaN for frozen systems).
template <int L>
__device__ __forceinline__ void finish_body(const WhgState& st, const WhgBuckets& bk, const WhgAdj& adj,
                                            int b, int w)
{
    const Place<L> pl(st, bk, b, w);
    const Group<L>& g = pl.g;
    const size_t lane = pl.lane;
    const size_t NL = adj.NL;
    const int s = pl.sys;
    const bool real = pl.has_sys && g.p < st.nplan[s];
    const double m = st.m[lane];
    const double* ck = adj.ckpt;                     // checkpoint 0: the initial DH state
    const double vx = ck[3 * NL + lane], vy = ck[4 * NL + lane], vz = ck[5 * NL + lane];
    const double* lam = adj.lam;
    double lqx = lam[0 * NL + lane], lqy = lam[1 * NL + lane], lqz = lam[2 * NL + lane];
    double lvx = lam[3 * NL + lane], lvy = lam[4 * NL + lane], lvz = lam[5 * NL + lane];
    double lm = lam[6 * NL + lane], lmu = lam[7 * NL + lane];
    if (!real) lqx = lqy = lqz = lvx = lvy = lvz = lm = lmu = 0.0;
    const double Sqx = group_sum<L>(g, lqx), Sqy = group_sum<L>(g, lqy), Sqz = group_sum<L>(g, lqz);
    const double Lx = group_sum<L>(g, lvx), Ly = group_sum<L>(g, lvy), Lz = group_sum<L>(g, lvz);
    const double Px = group_sum<L>(g, real ? m * vx : 0.0), Py = group_sum<L>(g, real ? m * vy : 0.0),
                 Pz = group_sum<L>(g, real ? m * vz : 0.0);
    const double Lmu = group_sum<L>(g, lmu);
    if (!pl.has_sys) return;
    const int u = user_index(st, s);
    const int B = 1 + st.Nmax;
    const double mu = st.m0[s], M = st.M[s];
    const bool bad = st.status[s] != 0;
    const double nan = __longlong_as_double(0x7ff8000000000000LL);
    for (int slot = g.p; slot < st.Nmax; slot += L) {
        const size_t o = (size_t)u * B + 1 + slot;
        const bool live = slot == g.p && real;
        double gx[3] = {0.0, 0.0, 0.0}, gu[3] = {0.0, 0.0, 0.0}, gm = 0.0;
        if (live) {
            gx[0] = lqx; gx[1] = lqy; gx[2] = lqz;
            gu[0] = lvx - (m / M) * Lx;
            gu[1] = lvy - (m / M) * Ly;
            gu[2] = lvz - (m / M) * Lz;
            gm = lm - (vx * Lx + vy * Ly + vz * Lz) / M;
        }
        for (int d = 0; d < 3; ++d) {
            if (adj.gx) adj.gx[o * 3 + d] = bad && live ? nan : gx[d];
            if (adj.gu) adj.gu[o * 3 + d] = bad && live ? nan : gu[d];
        }
        if (adj.gm) adj.gm[o] = bad && live ? nan : gm;
    }
    if (g.p == 0) {
        const size_t o = (size_t)u * B;
        const double g0[3] = {-Sqx, -Sqy, -Sqz};
        const double L3[3] = {Lx, Ly, Lz};
        for (int d = 0; d < 3; ++d) {
            if (adj.gx) adj.gx[o * 3 + d] = bad ? nan : g0[d];
            if (adj.gu) adj.gu[o * 3 + d] = bad ? nan : -(mu / M) * L3[d];
        }
        // u_0 - V_cm = -P / m0
        const double gm0 = Lmu + (Px * Lx + Py * Ly + Pz * Lz) / (mu * M);
        if (adj.gm) adj.gm[o] = bad ? nan : gm0;
    }
}

template <int NT, int GRM>
__global__ void __launch_bounds__(WHG_MAX_BLOCK) k_adj_tape(WhgState st, WhgBuckets bk, WhgAdj adj, int seg,
                                                            long long s0, int nk, int buf)
{
    const int w = warp_index();
    if (w >= bk.warp0[bk.nb]) return;
    const int b = bucket_of(bk, w);
    WHG_DISPATCH_L(bk.L[b], (tape_body<L_, NT, GRM>(st, bk, adj, b, w, seg, s0, nk, buf)))
}

template <int NT, int GRM>
__global__ void __launch_bounds__(WHG_MAX_BLOCK) k_adj_back(WhgState st, WhgBuckets bk, WhgAdj adj,
                                                            long long s0, int nk, int buf)
{
    const int w = warp_index();
    if (w >= bk.warp0[bk.nb]) return;
    const int b = bucket_of(bk, w);
    WHG_DISPATCH_L(bk.L[b], (back_body<L_, NT, GRM>(st, bk, adj, b, w, s0, nk, buf)))
}

template <int NT>
__global__ void __launch_bounds__(WHG_MAX_BLOCK) k_adj_loss(WhgState st, WhgBuckets bk, WhgAdj adj, int start)
{
    const int w = warp_index();
    if (w >= bk.warp0[bk.nb]) return;
    const int b = bucket_of(bk, w);
    WHG_DISPATCH_L(bk.L[b], (loss_body<L_, NT>(st, bk, adj, b, w, start)))
}

__global__ void __launch_bounds__(WHG_MAX_BLOCK) k_adj_save(WhgState st, WhgBuckets bk, WhgAdj adj, int slot)
{
    const int w = warp_index();
    if (w >= bk.warp0[bk.nb]) return;
    save_body<1>(st, adj, slot, w);
}

__global__ void __launch_bounds__(WHG_MAX_BLOCK) k_adj_finish(WhgState st, WhgBuckets bk, WhgAdj adj)
{
    const int w = warp_index();
    if (w >= bk.warp0[bk.nb]) return;
    const int b = bucket_of(bk, w);
    WHG_DISPATCH_L(bk.L[b], (finish_body<L_>(st, bk, adj, b, w)))
}

}  // namespace whg

cudaError_t whg_launch_adj_save(const WhgState& st, const WhgBuckets& bk, const WhgAdj& adj, int slot,
                                const WhgLaunch& l)
{
    whg::k_adj_save<<<l.grid, l.block, 0, l.stream>>>(st, bk, adj, slot);
    return cudaGetLastError();
}

cudaError_t whg_launch_adj_loss(const WhgState& st, const WhgBuckets& bk, const WhgAdj& adj, int start,
                                int newton_terms, const WhgLaunch& l)
{
    if (newton_terms == 6)
        whg::k_adj_loss<6><<<l.grid, l.block, 0, l.stream>>>(st, bk, adj, start);
    else
        whg::k_adj_loss<8><<<l.grid, l.block, 0, l.stream>>>(st, bk, adj, start);
    return cudaGetLastError();
}

cudaError_t whg_launch_adj_tape(const WhgState& st, const WhgBuckets& bk, const WhgAdj& adj, int seg,
                                long long s0, int nk, int buf, int newton_terms, int gr_mode, const WhgLaunch& l)
{
#define WHG_ADJ_TAPE(NT_, GR_) whg::k_adj_tape<NT_, GR_><<<l.grid, l.block, 0, l.stream>>>(st, bk, adj, seg, s0, nk, buf)
    if (newton_terms == 6) {
        if (gr_mode == 0) WHG_ADJ_TAPE(6, 0);
        else if (gr_mode == 1) WHG_ADJ_TAPE(6, 1);
        else WHG_ADJ_TAPE(6, 2);
    } else {
        if (gr_mode == 0) WHG_ADJ_TAPE(8, 0);
        else if (gr_mode == 1) WHG_ADJ_TAPE(8, 1);
        else WHG_ADJ_TAPE(8, 2);
    }
#undef WHG_ADJ_TAPE
    return cudaGetLastError();
}

cudaError_t whg_launch_adj_back(const WhgState& st, const WhgBuckets& bk, const WhgAdj& adj, long long s0,
                                int nk, int buf, int newton_terms, int gr_mode, const WhgLaunch& l)
{
#define WHG_ADJ_BACK(NT_, GR_) whg::k_adj_back<NT_, GR_><<<l.grid, l.block, 0, l.stream>>>(st, bk, adj, s0, nk, buf)
    if (newton_terms == 6) {
        if (gr_mode == 0) WHG_ADJ_BACK(6, 0);
        else if (gr_mode == 1) WHG_ADJ_BACK(6, 1);
        else WHG_ADJ_BACK(6, 2);
    } else {
        if (gr_mode == 0) WHG_ADJ_BACK(8, 0);
        else if (gr_mode == 1) WHG_ADJ_BACK(8, 1);
        else WHG_ADJ_BACK(8, 2);
    }
#undef WHG_ADJ_BACK
    return cudaGetLastError();
}

cudaError_t whg_launch_adj_finish(const WhgState& st, const WhgBuckets& bk, const WhgAdj& adj,
                                  const WhgLaunch& l)
{
    whg::k_adj_finish<<<l.grid, l.block, 0, l.stream>>>(st, bk, adj);
    return cudaGetLastError();
}
