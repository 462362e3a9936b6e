/*
 * flopcount.cpp -- CPU ORACLE helper (test infrastructure only): counts the
 * floating-point operations of one steady-state Wisdom-Holman step of the
 * oracle (orc_core.c compiled with a counting number type).
 *
 * Counted: add/sub, mul, div, sqrt on values that depend on the state.
 * Products of constants (dt, masses, c) are plain doubles and not counted;
 * negation is not counted.  Prints: adds muls divs sqrts flops start, where
 * flops = adds + muls + divs + sqrts and start = the part of flops spent in
 * the Kepler solver's starting phase (initial guess and Halley steps).
 *
 * Usage: orc_flopcount N_PLANETS NEWTON_TERMS GR_MODE [HALLEY_ITERS (default 2)]
 */
#include <cmath>
#include <cstdio>
#include <cstdlib>

struct Counted {
    double v;
    static long long adds, muls, divs, sqrts, start;
    static int in_start;
    Counted() : v(0.0) {}
    Counted(double x) : v(x) {}
};
long long Counted::adds = 0, Counted::muls = 0, Counted::divs = 0, Counted::sqrts = 0;
long long Counted::start = 0;
int Counted::in_start = 0;

static void tally(long long& c) { ++c; if (Counted::in_start) ++Counted::start; }
static Counted operator+(Counted a, Counted b) { tally(Counted::adds); return Counted(a.v + b.v); }
static Counted operator-(Counted a, Counted b) { tally(Counted::adds); return Counted(a.v - b.v); }
static Counted operator*(Counted a, Counted b) { tally(Counted::muls); return Counted(a.v * b.v); }
static Counted operator/(Counted a, Counted b) { tally(Counted::divs); return Counted(a.v / b.v); }
static Counted operator-(Counted a) { return Counted(-a.v); }
static Counted operator+(double a, Counted b) { return Counted(a) + b; }
static Counted operator-(double a, Counted b) { return Counted(a) - b; }
static Counted operator*(double a, Counted b) { return Counted(a) * b; }
static Counted operator/(double a, Counted b) { return Counted(a) / b; }
static Counted operator+(Counted a, double b) { return a + Counted(b); }
static Counted operator-(Counted a, double b) { return a - Counted(b); }
static Counted operator*(Counted a, double b) { return a * Counted(b); }
static Counted operator/(Counted a, double b) { return a / Counted(b); }
static bool operator>(Counted a, double b) { return a.v > b; }
static bool operator<(Counted a, double b) { return a.v < b; }
static Counted orc_sqrt(Counted x) { tally(Counted::sqrts); return Counted(std::sqrt(x.v)); }
static int orc_isfinite(Counted x) { return std::isfinite(x.v) ? 1 : 0; }
static double orc_value(Counted x) { return x.v; }

#define ORC_REAL Counted
#define ORC_START_PHASE(on) (Counted::in_start = (on))
#include "orc_core.c"

int main(int argc, char** argv)
{
    if (argc < 4) { std::fprintf(stderr, "usage: %s N NEWTON_TERMS GR_MODE\n", argv[0]); return 2; }
    int n = std::atoi(argv[1]), nt = std::atoi(argv[2]), gr = std::atoi(argv[3]);
    int hi = argc > 4 ? std::atoi(argv[4]) : 2;
    if (n < 1 || n > ORC_NMAX || hi < 0 || hi > 16) return 2;
    orc_options opt;
    opt.gr_mode = gr; opt.c_light = 10065.32; opt.halley_iters = hi; opt.halley_terms = 4;
    opt.newton_iters = 2; opt.newton_terms = nt;
    opt.encounter_hill = 0.0; opt.eject_factor = 0.0; opt.merge_jumps = 0;
    orc_system s = orc_system();
    s.n = n; s.m0 = 1.0; s.dt = 0.01; s.M = 1.0; s.nstep = 1;   /* steady state: K(dt) */
    for (int i = 0; i < n; ++i) {
        double a = 1.0 + 0.5 * i, vc = std::sqrt(1.0 / a);
        s.m[i] = 1e-5;
        s.Q[i][0] = Counted(a * std::cos(0.7 * i)); s.Q[i][1] = Counted(a * std::sin(0.7 * i));
        s.Q[i][2] = Counted(0.01 * i);
        s.v[i][0] = Counted(-vc * std::sin(0.7 * i)); s.v[i][1] = Counted(vc * std::cos(0.7 * i));
        s.v[i][2] = Counted(0.0);
    }
    orc_step(&s, 1, &opt);
    if (s.status) { std::fprintf(stderr, "unexpected status %d\n", s.status); return 1; }
    long long fl = Counted::adds + Counted::muls + Counted::divs + Counted::sqrts;
    std::printf("%lld %lld %lld %lld %lld %lld\n", Counted::adds, Counted::muls, Counted::divs,
                Counted::sqrts, fl, Counted::start);
    return 0;
}
