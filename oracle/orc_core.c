/*
 * orc_core.c -- CPU ORACLE for the WHFast512 timestep.  TEST INFRASTRUCTURE ONLY.
 *
 * Only the tests, the package's smoke() check and the benchmark's CPU-baseline
 * leg may load this code.  The product (the CUDA library) never calls it and
 * shares no code, header, table or constant with it.
 *
 * A plain, scalar, FP64 restatement of the map the paper defines
 * (Javaheri, Rein & Tamayo 2023, "WHFast512"): one Wisdom-Holman step in
 * democratic heliocentric coordinates (Sec. 3.1, Eq. 1 and Eq. 2), built from
 *   - the Kepler drift H_K (Sec. 3.2, Eq. 3): fixed 2 Halley + 2 Newton
 *     iterations on the universal-variable Kepler equation, Stumpff series
 *     with 4 terms (Halley) and 8 (or 6, Appendix A) terms (Newton),
 *   - the jump step H_J (Sec. 3.4, Eq. 6),
 *   - the interaction kick H_I (Sec. 3.3, Eq. 5),
 *   - the optional 1/r^2 "GR" potential centred on the star (Sec. 3.3, last
 *     paragraphs).
 * Loops are the obvious ones (planets in index order, pairs i < j, sequential
 * sums); nothing is blocked, fused or reordered.  Build with -O2 -ffp-contract=off so that no
 * multiply-add is contracted.
 *
 * Readings where the paper is silent:
 *   - Kepler mu = G m_0 (H_K of Eq. 3 uses G m_0 m_i, not G(m_0+m_i)).
 *   - initial guess X_0 = h / r_0 (the first-order value of X(h) = int dt/r;
 *     the paper gives no guess).  Of the guesses tried (0, first and second
 *     order), only this one makes 2 Halley steps need 2 Newton steps, as
 *     Appendix A states; with the second-order guess one Newton step is on
 *     the edge of the requirement.
 *   - "T terms" = the series of c_2 and c_3 carried through the z^T term:
 *     c_n(z) ~ sum_{k=0..T} (-z)^k / (n+2k)!, i.e. T terms after the leading
 *     1/n! (equivalently T terms each of the c_4, c_5 series, with
 *     c_2 = 1/2 - z c_4 and c_3 = 1/6 - z c_5); c_0, c_1 follow from
 *     c_0 = 1 - z c_2, c_1 = 1 - z c_3.  With this count the main text's
 *     default (4 and 8 terms) meets Appendix A's requirement (relative a
 *     error below 1e-13 at a = 0.387 AU, 5-day step, 10 yr, e <= 0.7) and
 *     8 is the shortest Newton-phase series that does; counting the leading
 *     term as one of the T (T terms in all), it misses at e = 0.7 by a
 *     factor of 2.  Appendix A's 6 terms miss the requirement under every
 *     count tried (5.8e-11 at e = 0.7 with this one).
 *   - f, g, fdot, gdot use G_n re-evaluated at the final X (T_N terms).
 *   - GR: Phi(r) = -3 (G m_0)^2 / (c^2 r^2) per unit planet mass.  gr_mode 1
 *     kicks v_i by h a_GR(Q_i) (canonical in these coordinates); gr_mode 2 also
 *     subtracts sum_j (m_j/m_0) a_GR(Q_j) from every planet (the literal
 *     reading of the back-reaction sentence).
 *   - the two J(dt/2) half-steps are applied separately, unless merge_jumps
 *     is set and the GR term is off: then one J(dt) precedes I(dt), the
 *     combination Sec. 3.1 allows because J and I commute without GR.
 *   - the interaction visits each unordered pair once (Newton's third law,
 *     Sec. 3.3), in plain i < j order.
 *   - a system whose step produces a non-finite value, or that starts a
 *     Kepler drift with beta <= 0 (unbound; outside the solver's domain,
 *     Sec. 3.2), is rolled back to the start of that step and frozen.
 *   - optional ensemble stopping rules (not part of the paper's map), with the
 *     same rollback: a pair closer than K mutual Hill radii
 *     ((m_i+m_j)/(3 m_0))^(1/3) (a_i+a_j)/2 during the interaction step, or a
 *     planet farther than F times the system's largest initial a at the start
 *     of a drift; a_i are the osculating heliocentric semi-major axes
 *     (mu = G(m_0+m_i)) of the initial state.
 *
 * This file is C99 and also compiles as C++ with ORC_REAL set to a counting
 * number type (oracle/flopcount.cpp; it only counts operations) or, together
 * with ORC_MASS, to a dual number (oracle/tangent.cpp: forward-mode
 * derivatives of the same map).
 */
#ifndef ORC_CORE_C
#define ORC_CORE_C

#include <math.h>
#include <string.h>

#ifndef ORC_REAL
#define ORC_REAL double
static double orc_sqrt(double x) { return sqrt(x); }
static int orc_isfinite(double x) { return isfinite(x) != 0; }
static double orc_value(double x) { return x; }
#endif
#ifndef ORC_MASS
#define ORC_MASS double          /* masses: double, or the tangent type in tangent.cpp */
static double orc_mass_value(double x) { return x; }
#endif
typedef ORC_REAL orc_real;
typedef ORC_MASS orc_mass;

#define ORC_NMAX 8            /* planets per system */
#define ORC_TMAX 12           /* longest Stumpff series supported */

#define ORC_STATUS_NONFINITE 1
#define ORC_STATUS_HYPERBOLIC 2
#define ORC_STATUS_CLOSE_ENCOUNTER 8
#define ORC_STATUS_EJECTED 16

typedef struct {
    int gr_mode;         /* 0 off, 1 canonical, 2 with explicit back-reaction */
    double c_light;      /* speed of light, code units */
    int halley_iters;    /* 2 (Sec. 3.2) */
    int halley_terms;    /* 4 (Sec. 3.2) */
    int newton_iters;    /* 2 (Sec. 3.2) */
    int newton_terms;    /* 8 (Sec. 3.2) or 6 (Appendix A) */
    double encounter_hill; /* stop rule: pair closer than this many mutual Hill radii (0 = off) */
    double eject_factor;   /* stop rule: |Q_i| beyond this many initial outermost a (0 = off) */
    int merge_jumps;       /* without GR: one J(dt) then I(dt) instead of J(dt/2) I(dt) J(dt/2) */
} orc_options;

/* One system in democratic heliocentric coordinates (Sec. 3.1).
 * Q[i] is planet i's position relative to the star, v[i] = P_i / m_i its
 * velocity relative to the barycentre; Xcm, Vcm, M describe H_0. */
typedef struct {
    int n;                      /* number of planets, 1..ORC_NMAX */
    orc_mass m0;                /* star mass */
    orc_mass m[ORC_NMAX];
    orc_real Q[ORC_NMAX][3];
    orc_real v[ORC_NMAX][3];
    double dt;
    orc_mass M;                 /* total mass */
    orc_real Xcm[3], Vcm[3];    /* barycentre position (at t = 0) and velocity */
    long long nstep;            /* completed steps; 0 = synchronized state */
    int status;
    double a0[ORC_NMAX];        /* osculating heliocentric semi-major axes at init (stop rules) */
} orc_system;

/* 1/k! for the Stumpff series: k! is exact in double for k <= 22, so one
 * division rounds it correctly (the default 8-term series needs k <= 19). */
static double orc_inv_factorial(int k)
{
    double f = 1.0;
    int i;
    for (i = 2; i <= k; ++i) f *= (double)i;
    return 1.0 / f;
}

/* Stumpff functions c_2(z), c_3(z) by their Taylor series truncated after
 * the z^terms term, c_n(z) = sum_{k=0..terms} (-z)^k / (n+2k)!, evaluated by
 * Horner's rule (Sec. 3.2: series plus a precomputed table, no quarter-angle
 * reduction). */
static void orc_stumpff_c2c3(orc_real z, int terms, orc_real* c2, orc_real* c3)
{
    orc_real s2 = orc_inv_factorial(2 * terms + 2);  /* k = terms: 1/(2+2k)! */
    orc_real s3 = orc_inv_factorial(2 * terms + 3);  /*            1/(3+2k)! */
    int k;
    for (k = terms - 1; k >= 0; --k) {
        s2 = orc_inv_factorial(2 * k + 2) - z * s2;
        s3 = orc_inv_factorial(2 * k + 3) - z * s3;
    }
    *c2 = s2;
    *c3 = s3;
}

/* Stiefel functions G_n(beta, X) = X^n c_n(beta X^2), n = 0..3, with
 * c_0 = 1 - z c_2 and c_1 = 1 - z c_3. */
static void orc_stiefel(orc_real beta, orc_real X, int terms, orc_real G[4])
{
    orc_real X2 = X * X;
    orc_real z = beta * X2;
    orc_real c2, c3;
    orc_stumpff_c2c3(z, terms, &c2, &c3);
    G[0] = 1.0 - z * c2;
    G[1] = X * (1.0 - z * c3);
    G[2] = X2 * c2;
    G[3] = X2 * X * c3;
}

/* Kepler drift for one planet under H_K,i = P_i^2/2m_i - G m_0 m_i / Q_i
 * (Sec. 3.2, Eq. 3) for time h with mu = G m_0 (G = 1).  Universal variable X,
 * Kepler function F(X) = r_0 G_1 + eta_0 G_2 + mu G_3 - h, F' = r, F'' = dr/dX.
 * Fixed iteration count, no convergence test, no branches.  Writes beta. */
/* Hook for the flop counter (flopcount.cpp): marks the solver's starting
 * phase, the initial guess and the Halley steps.  No-op elsewhere. */
#ifndef ORC_START_PHASE
#define ORC_START_PHASE(on) ((void)0)
#endif

static void orc_kepler_drift(orc_mass mu, double h, orc_real Q[3], orc_real v[3],
                             const orc_options* opt, orc_real* beta_out)
{
    orc_real r0 = orc_sqrt(Q[0] * Q[0] + Q[1] * Q[1] + Q[2] * Q[2]);
    orc_real eta0 = Q[0] * v[0] + Q[1] * v[1] + Q[2] * v[2];
    orc_real v2 = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
    orc_real beta = 2.0 * mu / r0 - v2;
    orc_real zeta0 = mu - beta * r0;
    orc_real X, G[4];
    int it;
    *beta_out = beta;
    ORC_START_PHASE(1);
    X = h / r0;

    for (it = 0; it < opt->halley_iters; ++it) {           /* Halley's method */
        orc_stiefel(beta, X, opt->halley_terms, G);
        {
            orc_real F = r0 * G[1] + eta0 * G[2] + mu * G[3] - h;
            orc_real Fp = r0 * G[0] + eta0 * G[1] + mu * G[2];
            orc_real Fpp = eta0 * G[0] + zeta0 * G[1];
            X = X - 2.0 * F * Fp / (2.0 * Fp * Fp - F * Fpp);
        }
    }
    ORC_START_PHASE(0);
    for (it = 0; it < opt->newton_iters; ++it) {           /* Newton's method */
        orc_stiefel(beta, X, opt->newton_terms, G);
        {
            orc_real F = r0 * G[1] + eta0 * G[2] + mu * G[3] - h;
            orc_real Fp = r0 * G[0] + eta0 * G[1] + mu * G[2];
            X = X - F / Fp;
        }
    }
    orc_stiefel(beta, X, opt->newton_terms, G);             /* final X */
    {
        orc_real r = r0 * G[0] + eta0 * G[1] + mu * G[2];
        orc_real f = 1.0 - mu * G[2] / r0;
        orc_real g = h - mu * G[3];
        orc_real fd = -mu * G[1] / (r * r0);
        orc_real gd = 1.0 - mu * G[2] / r;
        orc_real Qn[3], vn[3];
        int c;
        for (c = 0; c < 3; ++c) {
            Qn[c] = f * Q[c] + g * v[c];
            vn[c] = fd * Q[c] + gd * v[c];
        }
        for (c = 0; c < 3; ++c) {
            Q[c] = Qn[c];
            v[c] = vn[c];
        }
    }
}

/* Jump step H_J for time h (Sec. 3.4, Eq. 6): every planet's position moves by
 * (h / m_0) sum_j P_j with P_j = m_j v_j summed over planets only; velocities
 * are unchanged and the star does not move. */
static void orc_jump(orc_system* s, double h)
{
    orc_real Psum[3] = {0.0, 0.0, 0.0};
    int i, c;
    for (i = 0; i < s->n; ++i)
        for (c = 0; c < 3; ++c) Psum[c] = Psum[c] + s->m[i] * s->v[i][c];
    for (i = 0; i < s->n; ++i)
        for (c = 0; c < 3; ++c) s->Q[i][c] = s->Q[i][c] + h / s->m0 * Psum[c];
}

/* Interaction kick H_I for time h (Sec. 3.3, Eq. 5):
 * a_i = -sum_{j != i} G m_j Q_ij / |Q_ij|^3 with Q_ij = Q_i - Q_j; v_i += h a_i.
 * Each unordered pair i < j is visited once and gives both accelerations
 * (Newton's third law, as Sec. 3.3 does to halve the square roots).
 * Returns 1 if a pair is closer than the close-encounter stop rule allows
 * (not part of the paper's map: an ensemble stopping rule, see orc_step). */
static int orc_interaction(orc_system* s, double h, const orc_options* opt)
{
    orc_real a[ORC_NMAX][3];
    int i, j, c, close = 0;
    for (i = 0; i < s->n; ++i)
        for (c = 0; c < 3; ++c) a[i][c] = 0.0;
    for (i = 0; i < s->n; ++i) {
        for (j = i + 1; j < s->n; ++j) {
            orc_real d[3], r2, r3, ki, kj;
            for (c = 0; c < 3; ++c) d[c] = s->Q[i][c] - s->Q[j][c];
            r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
            if (opt->encounter_hill > 0.0) {
                /* mutual Hill radius from the initial semi-major axes */
                double rh = opt->encounter_hill *
                            cbrt(orc_mass_value(s->m[i] + s->m[j]) / (3.0 * orc_mass_value(s->m0))) *
                            0.5 * (s->a0[i] + s->a0[j]);
                if (r2 < rh * rh) close = 1;
            }
            r3 = r2 * orc_sqrt(r2);
            ki = s->m[j] / r3;
            kj = s->m[i] / r3;
            for (c = 0; c < 3; ++c) {
                a[i][c] = a[i][c] - ki * d[c];
                a[j][c] = a[j][c] + kj * d[c];
            }
        }
    }
    for (i = 0; i < s->n; ++i)
        for (c = 0; c < 3; ++c) s->v[i][c] = s->v[i][c] + h * a[i][c];
    return close;
}

/* Acceleration from the 1/r^2 potential centred on the star (Sec. 3.3, GR
 * paragraph; Nobili & Roxburgh 1986): Phi = -3 (G m_0)^2 / (c^2 r^2) per unit
 * planet mass, a_GR(Q) = -grad Phi = -6 (G m_0)^2 Q / (c^2 |Q|^4). */
static void orc_gr_acc(orc_mass m0, double c_light, const orc_real Q[3], orc_real a[3])
{
    orc_real r2 = Q[0] * Q[0] + Q[1] * Q[1] + Q[2] * Q[2];
    orc_real k = -6.0 * m0 * m0 / (c_light * c_light) / (r2 * r2);
    int c;
    for (c = 0; c < 3; ++c) a[c] = k * Q[c];
}

/* GR kick for time h.  gr_mode 1: v_i += h a_GR(Q_i).  gr_mode 2: the
 * accelerations are scaled by m_j/m_0, summed, and the sum is subtracted from
 * every planet's own term (the paper's back-reaction sentence). */
static void orc_gr_kick(orc_system* s, double h, const orc_options* opt)
{
    orc_real a[ORC_NMAX][3];
    int i, c;
    for (i = 0; i < s->n; ++i) orc_gr_acc(s->m0, opt->c_light, s->Q[i], a[i]);
    if (opt->gr_mode == 2) {
        orc_real back[3] = {0.0, 0.0, 0.0};
        for (i = 0; i < s->n; ++i)
            for (c = 0; c < 3; ++c) back[c] = back[c] + s->m[i] / s->m0 * a[i][c];
        for (i = 0; i < s->n; ++i)
            for (c = 0; c < 3; ++c) a[i][c] = a[i][c] - back[c];
    }
    for (i = 0; i < s->n; ++i)
        for (c = 0; c < 3; ++c) s->v[i][c] = s->v[i][c] + h * a[i][c];
}

static int orc_state_finite(const orc_system* s)
{
    int i, c;
    for (i = 0; i < s->n; ++i)
        for (c = 0; c < 3; ++c)
            if (!orc_isfinite(s->Q[i][c]) || !orc_isfinite(s->v[i][c])) return 0;
    return 1;
}

/* n Wisdom-Holman steps (Eq. 2) with the drifts of neighbouring steps fused:
 * K(dt/2) on the first step after a synchronized state, K(dt) afterwards,
 * then J(dt/2) I(dt) [GR] J(dt/2).  The trailing K(dt/2) is only applied to
 * a copy for output (orc_synchronize), as in the paper's "keep unsynchronized"
 * mode (Sec. 3.5 list). */
static void orc_step(orc_system* s, long long n, const orc_options* opt)
{
    long long k;
    for (k = 0; k < n; ++k) {
        orc_real Qs[ORC_NMAX][3], vs[ORC_NMAX][3];
        int i, bad = 0;
        if (s->status) return;                          /* frozen */
        memcpy(Qs, s->Q, sizeof(Qs));
        memcpy(vs, s->v, sizeof(vs));
        {
            double hK = (s->nstep == 0) ? 0.5 * s->dt : s->dt;
            double rej = 0.0;
            if (opt->eject_factor > 0.0) {
                for (i = 0; i < s->n; ++i)
                    if (s->a0[i] > rej) rej = s->a0[i];
                rej *= opt->eject_factor;
            }
            for (i = 0; i < s->n; ++i) {
                orc_real beta;
                if (opt->eject_factor > 0.0 &&
                    s->Q[i][0] * s->Q[i][0] + s->Q[i][1] * s->Q[i][1] + s->Q[i][2] * s->Q[i][2] > rej * rej)
                    bad |= ORC_STATUS_EJECTED;
                orc_kepler_drift(s->m0, hK, s->Q[i], s->v[i], opt, &beta);
                if (!(beta > 0.0)) bad |= ORC_STATUS_HYPERBOLIC;
            }
        }
        if (opt->merge_jumps && !opt->gr_mode) {
            /* J commutes with I when there is no GR term (Sec. 3.1): J(dt) I(dt) */
            orc_jump(s, s->dt);
            if (orc_interaction(s, s->dt, opt)) bad |= ORC_STATUS_CLOSE_ENCOUNTER;
        } else {
            orc_jump(s, 0.5 * s->dt);
            if (orc_interaction(s, s->dt, opt)) bad |= ORC_STATUS_CLOSE_ENCOUNTER;
            if (opt->gr_mode) orc_gr_kick(s, s->dt, opt);
            orc_jump(s, 0.5 * s->dt);
        }
        if (!orc_state_finite(s)) bad |= ORC_STATUS_NONFINITE;
        if (bad) {
            memcpy(s->Q, Qs, sizeof(Qs));
            memcpy(s->v, vs, sizeof(vs));
            s->status |= bad;
            return;
        }
        s->nstep += 1;
    }
}

/* Synchronized copy for output: the pending K(dt/2) (Sec. 3.5 list). */
static void orc_synchronize(const orc_system* s, orc_system* out, const orc_options* opt)
{
    *out = *s;
    if (s->nstep > 0) {
        int i;
        for (i = 0; i < s->n; ++i) {
            orc_real beta;
            orc_kepler_drift(s->m0, 0.5 * s->dt, out->Q[i], out->v[i], opt, &beta);
        }
    }
}

/* Inertial -> democratic heliocentric (Sec. 3.1): Q_i = x_i - x_0 and
 * v_i = u_i - V_cm (so P_i = m_i v_i is measured from the barycentre);
 * M, X_cm and V_cm are kept for H_0 and for the way back.  m [1+n],
 * x, u [1+n][3], body 0 the star. */
static void orc_to_dh(orc_system* s, int n, const orc_mass* m, const orc_real* x, const orc_real* u,
                      double dt)
{
    int k, i, c;
    s->n = n;
    s->m0 = m[0];
    s->dt = dt;
    s->M = 0.0;
    for (k = 0; k <= n; ++k) s->M = s->M + m[k];
    for (c = 0; c < 3; ++c) {
        orc_real px = 0.0, pu = 0.0;
        for (k = 0; k <= n; ++k) {
            px = px + m[k] * x[3 * k + c];
            pu = pu + m[k] * u[3 * k + c];
        }
        s->Xcm[c] = px / s->M;
        s->Vcm[c] = pu / s->M;
    }
    for (i = 0; i < n; ++i) {
        double r2 = 0.0, w2 = 0.0;
        s->m[i] = m[1 + i];
        for (c = 0; c < 3; ++c) {
            s->Q[i][c] = x[3 * (1 + i) + c] - x[c];
            s->v[i][c] = u[3 * (1 + i) + c] - s->Vcm[c];
        }
        for (c = 0; c < 3; ++c) {
            double dx = orc_value(x[3 * (1 + i) + c]) - orc_value(x[c]);
            double du = orc_value(u[3 * (1 + i) + c]) - orc_value(u[c]);
            r2 += dx * dx;
            w2 += du * du;
        }
        /* heliocentric two-body osculating semi-major axis, mu = G (m_0 + m_i),
         * for the stop rules only (no derivative needed) */
        s->a0[i] = 1.0 / (2.0 / sqrt(r2) - w2 / (orc_mass_value(m[0]) + orc_mass_value(m[1 + i])));
    }
    s->nstep = 0;
    s->status = 0;
}

#endif /* ORC_CORE_C */
