/*
 * orc_ensemble.c -- CPU ORACLE, ensemble layer and exported C functions.
 * TEST INFRASTRUCTURE ONLY: loaded by the tests, smoke() and the benchmark's
 * CPU-baseline leg; never by the product.
 *
 * Holds S independent systems (the ensemble form of Sec. 4: independent runs
 * in parallel), converts inertial <-> democratic heliocentric coordinates
 * (Sec. 3.1, following Duncan et al. 1998), and exposes init / step / read /
 * energy / raw-state calls.  orc_run_threads() integrates contiguous system
 * ranges on plain POSIX threads (used only to time the oracle on all cores).
 *
 * Array layouts (S systems, Nmax planets, body 0 = star):
 *   masses [S][1+Nmax], pos/vel [S][1+Nmax][3] inertial frame,
 *   Q/v raw state [S][Nmax][3] democratic heliocentric.
 */
#include "orc_core.c"

#include <pthread.h>
#include <stdlib.h>

typedef struct {
    int S, Nmax;
    orc_options opt;
    orc_system* sys;
} orc_ensemble;

orc_ensemble* orc_create(int S, int Nmax, int gr_mode, double c_light, int halley_iters,
                         int halley_terms, int newton_iters, int newton_terms,
                         double encounter_hill, double eject_factor, int merge_jumps)
{
    orc_ensemble* e;
    if (S < 1 || Nmax < 1 || Nmax > ORC_NMAX) return NULL;
    if (halley_terms < 1 || halley_terms > ORC_TMAX || newton_terms < 1 || newton_terms > ORC_TMAX)
        return NULL;
    e = (orc_ensemble*)calloc(1, sizeof(orc_ensemble));
    if (!e) return NULL;
    e->sys = (orc_system*)calloc((size_t)S, sizeof(orc_system));
    if (!e->sys) { free(e); return NULL; }
    e->S = S;
    e->Nmax = Nmax;
    e->opt.gr_mode = gr_mode;
    e->opt.c_light = c_light;
    e->opt.halley_iters = halley_iters;
    e->opt.halley_terms = halley_terms;
    e->opt.newton_iters = newton_iters;
    e->opt.newton_terms = newton_terms;
    e->opt.encounter_hill = encounter_hill;
    e->opt.eject_factor = eject_factor;
    e->opt.merge_jumps = merge_jumps;
    return e;
}

void orc_destroy(orc_ensemble* e)
{
    if (!e) return;
    free(e->sys);
    free(e);
}

/* Democratic heliocentric -> inertial at time t = nstep * dt:
 * x_0 = X_cm + V_cm t - sum m_i Q_i / M, x_i = x_0 + Q_i,
 * u_0 = V_cm - sum m_i v_i / m_0, u_i = v_i + V_cm. */
static void orc_from_dh(const orc_system* s, double* x, double* u)
{
    double t = (double)s->nstep * s->dt;
    int i, c;
    for (c = 0; c < 3; ++c) {
        double sq = 0.0, sp = 0.0;
        for (i = 0; i < s->n; ++i) {
            sq += s->m[i] * s->Q[i][c];
            sp += s->m[i] * s->v[i][c];
        }
        x[c] = s->Xcm[c] + s->Vcm[c] * t - sq / s->M;
        u[c] = s->Vcm[c] - sp / s->m0;
        for (i = 0; i < s->n; ++i) {
            x[3 * (1 + i) + c] = x[c] + s->Q[i][c];
            u[3 * (1 + i) + c] = s->v[i][c] + s->Vcm[c];
        }
    }
}

int orc_init(orc_ensemble* e, const double* masses, const double* pos, const double* vel,
             const int* n_planets, const double* dt)
{
    int s;
    const int B = 1 + e->Nmax;
    for (s = 0; s < e->S; ++s) {
        int n = n_planets ? n_planets[s] : e->Nmax;
        if (n < 1 || n > e->Nmax || !(dt[s] > 0.0) || !(masses[(size_t)s * B] > 0.0)) return -1;
        orc_to_dh(&e->sys[s], n, masses + (size_t)s * B, pos + (size_t)s * B * 3,
                  vel + (size_t)s * B * 3, dt[s]);
    }
    return 0;
}

void orc_step_range(orc_ensemble* e, int s0, int s1, long long n)
{
    int s;
    for (s = s0; s < s1; ++s) orc_step(&e->sys[s], n, &e->opt);
}

void orc_step_all(orc_ensemble* e, long long n) { orc_step_range(e, 0, e->S, n); }

/* Synchronized inertial state, status and time; the live state is untouched. */
void orc_read(const orc_ensemble* e, double* pos, double* vel, int* status, double* t)
{
    int s;
    const int B = 1 + e->Nmax;
    for (s = 0; s < e->S; ++s) {
        orc_system sy;
        size_t o = (size_t)s * B * 3;
        orc_synchronize(&e->sys[s], &sy, &e->opt);
        memset(pos + o, 0, sizeof(double) * 3 * B);
        memset(vel + o, 0, sizeof(double) * 3 * B);
        orc_from_dh(&sy, pos + o, vel + o);
        if (status) status[s] = e->sys[s].status;
        if (t) t[s] = (double)e->sys[s].nstep * e->sys[s].dt;
    }
}

/* Total energy H = H_0 + H_K + H_I + H_J (Eq. 1) of the synchronized state,
 * plus sum_i m_i Phi(Q_i) when the GR potential is on. */
void orc_energy(const orc_ensemble* e, double* E)
{
    int s, i, j, c;
    for (s = 0; s < e->S; ++s) {
        orc_system sy;
        double H0 = 0.0, HK = 0.0, HI = 0.0, HJ, P[3] = {0.0, 0.0, 0.0}, HG = 0.0;
        orc_synchronize(&e->sys[s], &sy, &e->opt);
        for (c = 0; c < 3; ++c) H0 += 0.5 * sy.M * sy.Vcm[c] * sy.Vcm[c];
        for (i = 0; i < sy.n; ++i) {
            double v2 = 0.0, r2 = 0.0;
            for (c = 0; c < 3; ++c) {
                v2 += sy.v[i][c] * sy.v[i][c];
                r2 += sy.Q[i][c] * sy.Q[i][c];
                P[c] += sy.m[i] * sy.v[i][c];
            }
            HK += 0.5 * sy.m[i] * v2 - sy.m0 * sy.m[i] / sqrt(r2);
            if (e->opt.gr_mode)
                HG += -3.0 * sy.m[i] * sy.m0 * sy.m0 / (e->opt.c_light * e->opt.c_light * r2);
            for (j = i + 1; j < sy.n; ++j) {
                double d2 = 0.0;
                for (c = 0; c < 3; ++c) d2 += (sy.Q[i][c] - sy.Q[j][c]) * (sy.Q[i][c] - sy.Q[j][c]);
                HI -= sy.m[i] * sy.m[j] / sqrt(d2);
            }
        }
        HJ = (P[0] * P[0] + P[1] * P[1] + P[2] * P[2]) / (2.0 * sy.m0);
        E[s] = H0 + HK + HI + HJ + HG;
    }
}

/* Raw (unsynchronized) state for bitwise checkpoint / resume. */
void orc_get_raw(const orc_ensemble* e, double* Q, double* v, long long* nstep, int* status)
{
    int s, i, c;
    for (s = 0; s < e->S; ++s) {
        for (i = 0; i < e->Nmax; ++i)
            for (c = 0; c < 3; ++c) {
                size_t o = ((size_t)s * e->Nmax + i) * 3 + c;
                Q[o] = i < e->sys[s].n ? e->sys[s].Q[i][c] : 0.0;
                v[o] = i < e->sys[s].n ? e->sys[s].v[i][c] : 0.0;
            }
        nstep[s] = e->sys[s].nstep;
        status[s] = e->sys[s].status;
    }
}

void orc_set_raw(orc_ensemble* e, const double* Q, const double* v, const long long* nstep,
                 const int* status)
{
    int s, i, c;
    for (s = 0; s < e->S; ++s) {
        for (i = 0; i < e->sys[s].n; ++i)
            for (c = 0; c < 3; ++c) {
                size_t o = ((size_t)s * e->Nmax + i) * 3 + c;
                e->sys[s].Q[i][c] = Q[o];
                e->sys[s].v[i][c] = v[o];
            }
        e->sys[s].nstep = nstep[s];
        e->sys[s].status = status[s];
    }
}

/* ---- single sub-steps on one system, for the oracle's own pins ---------- */

void orc_apply_kepler(const orc_ensemble* e, double mu, double h, double* Q, double* v,
                      double* beta)
{
    orc_kepler_drift(mu, h, Q, v, &e->opt, beta);
}

void orc_apply_substep(orc_ensemble* e, int s, int which, double h)
{
    orc_system* sy = &e->sys[s];
    int i;
    double beta;
    switch (which) {
    case 0:
        for (i = 0; i < sy->n; ++i) orc_kepler_drift(sy->m0, h, sy->Q[i], sy->v[i], &e->opt, &beta);
        break;
    case 1: orc_jump(sy, h); break;
    case 2: orc_interaction(sy, h, &e->opt); break;
    case 3: orc_gr_kick(sy, h, &e->opt); break;
    default: break;
    }
}

void orc_stumpff(double z, int terms, double* c2, double* c3) { orc_stumpff_c2c3(z, terms, c2, c3); }

/* ---- all-core timing run -------------------------------------------------- */

typedef struct {
    orc_ensemble* e;
    int s0, s1;
    long long n;
} orc_job;

static void* orc_worker(void* arg)
{
    orc_job* j = (orc_job*)arg;
    orc_step_range(j->e, j->s0, j->s1, j->n);
    return NULL;
}

/* Step every system n times on `threads` POSIX threads, contiguous ranges. */
int orc_run_threads(orc_ensemble* e, long long n, int threads)
{
    pthread_t tid[512];
    orc_job job[512];
    int t, started = 0;
    if (threads < 1) threads = 1;
    if (threads > 512) threads = 512;
    if (threads > e->S) threads = e->S;
    for (t = 0; t < threads; ++t) {
        job[t].e = e;
        job[t].s0 = (int)((long long)e->S * t / threads);
        job[t].s1 = (int)((long long)e->S * (t + 1) / threads);
        job[t].n = n;
        if (pthread_create(&tid[t], NULL, orc_worker, &job[t]) != 0) break;
        ++started;
    }
    for (t = 0; t < started; ++t) pthread_join(tid[t], NULL);
    if (started < threads) {           /* finish what could not be started */
        for (t = started; t < threads; ++t) orc_worker(&job[t]);
    }
    return threads;
}
