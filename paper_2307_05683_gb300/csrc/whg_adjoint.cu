// whg_adjoint.cu -- reverse-mode (adjoint) kernels of libwhg.
//
// Gradient of L_s = sum_i |Q_i(T) - target_i|^2 (heliocentric positions of the
// synchronized state after n steps, per system s) with respect to the initial
// inertial positions, velocities and masses.  The forward run keeps the state
// every K steps (checkpoints); the backward walks the segments in reverse:
// each segment's K steps are recomputed from its checkpoint while a per-step
// tape is written (drift input Q0, v0, final universal variable X, v after the
// drift, Q during the kick, v after the kick), then the vector-Jacobian
// products of J, I (+GR), J and K are applied step by step in reverse.  The
// tape of segment s-1 is recomputed (second stream, second tape buffer) while
// the products of segment s run.
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
// final universal variable X.  In: lq, lv = adjoints of Q1, v1.  Out: lq, lv
// = adjoints of Q0, v0; lmu accumulates the adjoint of mu.
//
// c4, c5 come from their NT-term series and c2 = 1/2 - z c4, c3 = 1/6 - z c5
// from the recurrence: the same series through z^NT that the forward drift
// sums.  Every
// Lagrange coefficient is mu times a function of the G_n, so the adjoints of
// mu, r, r0 and G_n are written with f - 1, fdot and gdot - 1 themselves:
//   mub  = ((f-1) fb + fdot fdb + (gdot-1) gdb) / mu - G3 gb,
//   rb   = -((fdot fdb + (gdot-1) gdb) / r,   r0b = -((f-1) fb + fdot fdb) / r0,
//   G1b  = -(mu / (r r0)) fdb,  G2b = -(mu / r0) fb - (mu / r) gdb,  G3b = -mu gb,
// with fb = lq.Q0, gb = lq.v0, fdb = lv.Q0, gdb = lv.v0.
template <int NT>
__device__ __forceinline__ void kepler_vjp(double mu, double muinv, double h, double qx, double qy,
                                           double qz, double vx, double vy, double vz, double X,
                                           double& lqx, double& lqy, double& lqz, double& lvx,
                                           double& lvy, double& lvz, double& lmu)
{
    const double r0sq = fma(qx, qx, fma(qy, qy, qz * qz));
    const double r0i = rsqrt(r0sq);
    const double r0 = r0sq * r0i;
    const double eta0 = fma(qx, vx, fma(qy, vy, qz * vz));
    const double v2 = fma(vx, vx, fma(vy, vy, vz * vz));
    const double beta = fma(2.0 * mu, r0i, -v2);
    const double X2 = X * X, X4 = X2 * X2;
    const double z = beta * X2;
    const double c4 = stumpff_c<4, NT>(z), c5 = stumpff_c<5, NT>(z);
    const double c2 = fma(-z, c4, 0.5), c3 = fma(-z, c5, 1.0 / 6.0);
    const double G2 = X2 * c2, G3 = (X2 * X) * c3, G4 = X4 * c4, G5 = (X4 * X) * c5;
    const double G0 = fma(-beta, G2, 1.0), G1 = fma(-beta, G3, X);
    const double r = fma(r0, G0, fma(eta0, G1, mu * G2));
    const double ri = rcp(r);
    const double A = mu * r0i, B = mu * ri, C = A * ri;
    const double fm1 = -A * G2, g = fma(-mu, G3, h), fd = -C * G1, gdm1 = -B * G2;
    // (a) outputs Q1 = f Q0 + g v0, v1 = fd Q0 + gd v0
    const double fb = fma(lqx, qx, fma(lqy, qy, lqz * qz));
    const double gb = fma(lqx, vx, fma(lqy, vy, lqz * vz));
    const double fdb = fma(lvx, qx, fma(lvy, qy, lvz * qz));
    const double gdb = fma(lvx, vx, fma(lvy, vy, lvz * vz));
    const double f = 1.0 + fm1, gd = 1.0 + gdm1;
    double nqx = fma(f, lqx, fd * lvx), nqy = fma(f, lqy, fd * lvy), nqz = fma(f, lqz, fd * lvz);
    double nvx = fma(g, lqx, gd * lvx), nvy = fma(g, lqy, gd * lvy), nvz = fma(g, lqz, gd * lvz);
    // (b) through f, g, fd, gd
    const double tf = fm1 * fb, tfd = fd * fdb, tgd = gdm1 * gdb;
    double mub = fma(tf + tfd + tgd, muinv, -G3 * gb);
    const double rb = -(tfd + tgd) * ri;
    double r0b = -(tf + tfd) * r0i;
    double G1b = -C * fdb;
    double G2b = fma(-A, fb, -B * gdb);
    const double G3b = -mu * gb;
    // (c) r = r0 G0 + eta0 G1 + mu G2
    r0b = fma(rb, G0, r0b);
    double eta0b = rb * G1;
    mub = fma(rb, G2, mub);
    const double G0b = rb * r0;
    G1b = fma(rb, eta0, G1b);
    G2b = fma(rb, mu, G2b);
    // (d) G_n(beta, X): dG_n/dX = G_{n-1}, dG_0/dX = -beta G1, dG_n/dbeta = (n G_{n+2} - X G_{n+1})/2
    const double hX = 0.5 * X;
    const double dG0 = -hX * G1, dG1 = fma(-hX, G2, 0.5 * G3);
    const double dG2 = fma(-hX, G3, G4), dG3 = fma(-hX, G4, 1.5 * G5);
    const double Xb = fma(-G0b * beta, G1, fma(G1b, G0, fma(G2b, G1, G3b * G2)));
    double betab = fma(G0b, dG0, fma(G1b, dG1, fma(G2b, dG2, G3b * dG3)));
    // (e) X implicit in F = r0 G1 + eta0 G2 + mu G3 - h = 0, dF/dX = r
    const double w = Xb * ri;
    r0b = fma(-w, G1, r0b);
    eta0b = fma(-w, G2, eta0b);
    mub = fma(-w, G3, mub);
    betab = fma(-w, fma(r0, dG1, fma(eta0, dG2, mu * dG3)), betab);
    // (f) beta = 2 mu / r0 - v.v, eta0 = Q.v, r0 = |Q|
    const double b2 = 2.0 * betab;
    mub = fma(b2, r0i, mub);
    r0b = fma(-b2 * A, r0i, r0b);
    const double rq = r0b * r0i;
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

// Adjoint of a jump Q_i += c sum_j m_j v_j with the velocities (vx, vy, vz)
// it used; lambda_Q passes through unchanged.
template <int L>
__device__ __forceinline__ void jump_vjp(const Group<L>& g, double m, double c, double mu, double vx,
                                         double vy, double vz, double lqx, double lqy, double lqz,
                                         double& lvx, double& lvy, double& lvz, double& lm, double& lmu)
{
    double Lx, Ly, Lz;
    group_sum3<L>(g, lqx, lqy, lqz, Lx, Ly, Lz);
    lvx += c * m * Lx;
    lvy += c * m * Ly;
    lvz += c * m * Lz;
    const double vd = vx * Lx + vy * Ly + vz * Lz;
    lm += c * vd;
    lmu -= (c / mu) * m * vd;
}

// Adjoint of the interaction kick (+GR) at positions Q, with lambda_v the
// adjoint of the velocities after it (which pass through unchanged).
template <int L, int GRM>
__device__ __forceinline__ void kick_vjp(const Group<L>& g, double qx, double qy, double qz, double m,
                                         double hm, double dt, double mu, double kgr, double lvx,
                                         double lvy, double lvz, double& lqx, double& lqy,
                                         double& lqz, double& lm, double& lmu)
{
#pragma unroll
    for (int k = 1; 2 * k < L; ++k) {
        const int to = g.at(k), from = g.at(-k);
        const double dx = __shfl_sync(WHG_FULL_MASK, qx, to) - qx;
        const double dy = __shfl_sync(WHG_FULL_MASK, qy, to) - qy;
        const double dz = __shfl_sync(WHG_FULL_MASK, qz, to) - qz;
        const double hmj = __shfl_sync(WHG_FULL_MASK, hm, to);
        const double ljx = __shfl_sync(WHG_FULL_MASK, lvx, to);
        const double ljy = __shfl_sync(WHG_FULL_MASK, lvy, to);
        const double ljz = __shfl_sync(WHG_FULL_MASK, lvz, to);
        const double r2 = fma(dx, dx, fma(dy, dy, dz * dz));
        const double r1i = rsqrt(r2);
        const double r2i = r1i * r1i, r3i = r2i * r1i, r5i = r3i * r2i;
        const double wx = hmj * lvx - hm * ljx, wy = hmj * lvy - hm * ljy, wz = hmj * lvz - hm * ljz;
        const double s3 = 3.0 * (wx * dx + wy * dy + wz * dz) * r5i;
        const double ldx = r3i * wx - s3 * dx, ldy = r3i * wy - s3 * dy, ldz = r3i * wz - s3 * dz;
        lqx -= ldx;
        lqy -= ldy;
        lqz -= ldz;
        lm -= dt * r3i * (ljx * dx + ljy * dy + ljz * dz);
        const double lmj = dt * r3i * (lvx * dx + lvy * dy + lvz * dz);   // for the partner
        lqx += __shfl_sync(WHG_FULL_MASK, ldx, from);
        lqy += __shfl_sync(WHG_FULL_MASK, ldy, from);
        lqz += __shfl_sync(WHG_FULL_MASK, ldz, from);
        lm += __shfl_sync(WHG_FULL_MASK, lmj, from);
    }
    if (L >= 2 && (L & 1) == 0) {
        const int to = g.at(L / 2);
        const double dx = __shfl_sync(WHG_FULL_MASK, qx, to) - qx;
        const double dy = __shfl_sync(WHG_FULL_MASK, qy, to) - qy;
        const double dz = __shfl_sync(WHG_FULL_MASK, qz, to) - qz;
        const double hmj = __shfl_sync(WHG_FULL_MASK, hm, to);
        const double r2 = fma(dx, dx, fma(dy, dy, dz * dz));
        const double r1i = rsqrt(r2);
        const double r2i = r1i * r1i, r3i = r2i * r1i, r5i = r3i * r2i;
        const double wx = hmj * lvx, wy = hmj * lvy, wz = hmj * lvz;
        const double s3 = 3.0 * (wx * dx + wy * dy + wz * dz) * r5i;
        const double ldx = r3i * wx - s3 * dx, ldy = r3i * wy - s3 * dy, ldz = r3i * wz - s3 * dz;
        lqx -= ldx;
        lqy -= ldy;
        lqz -= ldz;
        const double lmj = dt * r3i * (lvx * dx + lvy * dy + lvz * dz);
        lqx += __shfl_sync(WHG_FULL_MASK, ldx, to);
        lqy += __shfl_sync(WHG_FULL_MASK, ldy, to);
        lqz += __shfl_sync(WHG_FULL_MASK, ldz, to);
        lm += __shfl_sync(WHG_FULL_MASK, lmj, to);
    }
    if (GRM != 0) {
        const double r2 = fma(qx, qx, fma(qy, qy, qz * qz));
        const double ri2 = rcp(r2);
        const double c = kgr * (ri2 * ri2);
        double ax = lvx, ay = lvy, az = lvz;             // adjoint of this planet's a_GR
        if (GRM == 2) {
            double Lx, Ly, Lz;
            group_sum3<L>(g, lvx, lvy, lvz, Lx, Ly, Lz);
            const double aL = c * (qx * Lx + qy * Ly + qz * Lz);   // a_i . Lambda_v
            lm -= aL / mu;
            lmu += m * aL / (mu * mu);
            const double mr = m / mu;
            ax -= mr * Lx;
            ay -= mr * Ly;
            az -= mr * Lz;
        }
        const double s = qx * ax + qy * ay + qz * az;
        const double c4 = 4.0 * c * s * ri2;
        lqx += c * ax - c4 * qx;
        lqy += c * ay - c4 * qy;
        lqz += c * az - c4 * qz;
        lmu += 2.0 * (c / mu) * s;
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

// Tape of one segment: its steps recomputed from the checkpoint, writing per
// step the drift input (Q0, v0), the final X, v after the drift, Q during the
// kick and v after the kick into tape buffer `buf`.
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
        double* tp = tape + (size_t)k * 16 * NL + lane;
        tp[0 * NL] = qx; tp[1 * NL] = qy; tp[2 * NL] = qz;
        tp[3 * NL] = vx; tp[4 * NL] = vy; tp[5 * NL] = vz;
        const double h = (s0 + k == 0) ? 0.5 * dt : dt;
        double X;
        kepler_drift<NT>(mu, h, qx, qy, qz, vx, vy, vz, X, st.halley32 != 0);
        tp[6 * NL] = X;
        tp[7 * NL] = vx; tp[8 * NL] = vy; tp[9 * NL] = vz;
        const bool merged = GRM == 0 && st.merge;
        jump<L>(g, m, merged ? 2.0 * c : c, vx, vy, vz, qx, qy, qz);
        tp[10 * NL] = qx; tp[11 * NL] = qy; tp[12 * NL] = qz;
        kick<L, GRM>(g, qx, qy, qz, hm, mrat, kgr, nothr, vx, vy, vz, st.full_rotation != 0);
        tp[13 * NL] = vx; tp[14 * NL] = vy; tp[15 * NL] = vz;
        if (!merged) jump<L>(g, m, c, vx, vy, vz, qx, qy, qz);
        if (!real) {                                  // lanes without a planet stay parked
            qx = pqx; qy = pqy; qz = pqz;
            vx = pvx; vy = pvy; vz = pvz;
        }
    }
}

// Pull the adjoint back through the steps of one segment, last step first,
// from tape buffer `buf`.
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
    const double hm = dt * m, c = (0.5 * dt) / mu, muinv = 1.0 / mu;
    const double kgr = GRM ? (-6.0 * mu * mu * dt) / (st.c_light * st.c_light) : 0.0;
    const double* tape = adj.tape + (size_t)buf * adj.tape_len;
    double* lam = adj.lam;
    double lqx = lam[0 * NL + lane], lqy = lam[1 * NL + lane], lqz = lam[2 * NL + lane];
    double lvx = lam[3 * NL + lane], lvy = lam[4 * NL + lane], lvz = lam[5 * NL + lane];
    double lm = lam[6 * NL + lane], lmu = lam[7 * NL + lane];
    for (int k = nk - 1; k >= 0; --k) {
        const double* tp = tape + (size_t)k * 16 * NL + lane;
        const double q0x = tp[0 * NL], q0y = tp[1 * NL], q0z = tp[2 * NL];
        const double v0x = tp[3 * NL], v0y = tp[4 * NL], v0z = tp[5 * NL];
        const double X = tp[6 * NL];
        const double v1x = tp[7 * NL], v1y = tp[8 * NL], v1z = tp[9 * NL];
        const double q2x = tp[10 * NL], q2y = tp[11 * NL], q2z = tp[12 * NL];
        const double v3x = tp[13 * NL], v3y = tp[14 * NL], v3z = tp[15 * NL];
        const double h = (s0 + k == 0) ? 0.5 * dt : dt;
        const bool merged = GRM == 0 && st.merge;
        if (!merged) jump_vjp<L>(g, m, c, mu, v3x, v3y, v3z, lqx, lqy, lqz, lvx, lvy, lvz, lm, lmu);
        kick_vjp<L, GRM>(g, q2x, q2y, q2z, m, hm, dt, mu, kgr, lvx, lvy, lvz, lqx, lqy, lqz, lm, lmu);
        jump_vjp<L>(g, m, merged ? 2.0 * c : c, mu, v1x, v1y, v1z, lqx, lqy, lqz, lvx, lvy, lvz, lm, lmu);
        kepler_vjp<NT>(mu, muinv, h, q0x, q0y, q0z, v0x, v0y, v0z, X, lqx, lqy, lqz, lvx, lvy, lvz, lmu);
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
