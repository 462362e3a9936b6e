/*
 * tangent.cpp -- CPU ORACLE helper (test infrastructure only): forward-mode
 * derivatives of the oracle's map.  orc_core.c is compiled with a dual number
 * (value, derivative) for the state and the masses, so one pass gives the
 * exact directional derivative of the fixed-iteration map, rounding aside.
 *
 * orc_tangent_loss: one system, inertial initial conditions, n steps, loss
 * L = sum_i |Q_i - T_i|^2 over the planets' heliocentric positions of the
 * synchronized final state; the derivative of L along one input (a position,
 * velocity or mass component) is returned with L.
 */
#include <cmath>
#include <cstring>

struct Dual {
    double v, d;
    Dual() : v(0.0), d(0.0) {}
    Dual(double x) : v(x), d(0.0) {}
    Dual(double x, double dx) : v(x), d(dx) {}
};
static Dual operator+(Dual a, Dual b) { return Dual(a.v + b.v, a.d + b.d); }
static Dual operator-(Dual a, Dual b) { return Dual(a.v - b.v, a.d - b.d); }
static Dual operator*(Dual a, Dual b) { return Dual(a.v * b.v, a.d * b.v + a.v * b.d); }
static Dual operator/(Dual a, Dual b) { return Dual(a.v / b.v, (a.d * b.v - a.v * b.d) / (b.v * b.v)); }
static Dual operator-(Dual a) { return Dual(-a.v, -a.d); }
static Dual operator+(double a, Dual b) { return Dual(a) + b; }
static Dual operator-(double a, Dual b) { return Dual(a) - b; }
static Dual operator*(double a, Dual b) { return Dual(a) * b; }
static Dual operator/(double a, Dual b) { return Dual(a) / b; }
static Dual operator+(Dual a, double b) { return a + Dual(b); }
static Dual operator-(Dual a, double b) { return a - Dual(b); }
static Dual operator*(Dual a, double b) { return a * Dual(b); }
static Dual operator/(Dual a, double b) { return a / Dual(b); }
static bool operator>(Dual a, double b) { return a.v > b; }
static bool operator<(Dual a, double b) { return a.v < b; }
static Dual orc_sqrt(Dual x) { double r = std::sqrt(x.v); return Dual(r, x.d / (2.0 * r)); }
static int orc_isfinite(Dual x) { return std::isfinite(x.v) && std::isfinite(x.d) ? 1 : 0; }
static double orc_value(Dual x) { return x.v; }
static double orc_mass_value(Dual x) { return x.v; }

#define ORC_REAL Dual
#define ORC_MASS Dual
#include "orc_core.c"

extern "C" int orc_tangent_loss(int n, const double* m, const double* x, const double* u, double dt,
                                const double* target, long long nsteps, int gr_mode, double c_light,
                                int newton_terms, int merge_jumps, int kind, int body, int comp,
                                double* loss, double* dloss)
{
    if (n < 1 || n > ORC_NMAX || nsteps < 0) return -1;
    orc_options opt;
    opt.gr_mode = gr_mode;
    opt.c_light = c_light;
    opt.halley_iters = 2;
    opt.halley_terms = 4;
    opt.newton_iters = 2;
    opt.newton_terms = newton_terms;
    opt.encounter_hill = 0.0;
    opt.eject_factor = 0.0;
    opt.merge_jumps = merge_jumps;
    Dual md[ORC_NMAX + 1], xd[3 * (ORC_NMAX + 1)], ud[3 * (ORC_NMAX + 1)];
    for (int k = 0; k <= n; ++k) {
        md[k] = Dual(m[k], (kind == 2 && body == k) ? 1.0 : 0.0);
        for (int c = 0; c < 3; ++c) {
            xd[3 * k + c] = Dual(x[3 * k + c], (kind == 0 && body == k && comp == c) ? 1.0 : 0.0);
            ud[3 * k + c] = Dual(u[3 * k + c], (kind == 1 && body == k && comp == c) ? 1.0 : 0.0);
        }
    }
    orc_system s = orc_system();
    orc_to_dh(&s, n, md, xd, ud, dt);
    orc_step(&s, nsteps, &opt);
    if (s.status) return 1;
    orc_system out = orc_system();
    orc_synchronize(&s, &out, &opt);
    Dual L = 0.0;
    for (int i = 0; i < n; ++i)
        for (int c = 0; c < 3; ++c) {
            Dual e = out.Q[i][c] - target[3 * i + c];
            L = L + e * e;
        }
    *loss = L.v;
    *dloss = L.d;
    return 0;
}
