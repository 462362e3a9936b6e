"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Tolerances (the target the integrator is held to): after 1 step, 1e-12
relative; after 1e4 steps, 1e-9 relative; "relative" per coordinate with each
system's largest |coordinate| as the scale for inertial output, and each
planet's own |Q_i|, |v_i| for the raw heliocentric state.  Run-to-run and
launch-split results are compared bit for bit.
"""
import os

import numpy as np
import pytest

from paper_2307_05683_gb300 import inputs

pytestmark = pytest.mark.gpu

CORES = os.cpu_count() or 1


@pytest.fixture(scope="module")
def whg():
    from paper_2307_05683_gb300 import build, whg as w
    build.build()
    w.load()
    return w


def gpu_run(whg, ens, n, chunks=None, **kw):
    it = whg.Integrator(ens.n_systems, ens.max_planets, **kw)
    it.init(ens)
    for k in (chunks or [n]):
        it.step(k)
    out = it.read_state() + it.get_raw() + (it.energy(),)
    it.close()
    return out


def oracle_run(orc, ens, n, gr_mode=1, newton_terms=8, c_light=None, **extra):
    kw = dict(gr_mode=gr_mode, newton_terms=newton_terms, **extra)
    if c_light is not None:
        kw["c_light"] = c_light
    o = orc.OracleEnsemble(ens.n_systems, ens.max_planets, **kw)
    o.init(ens)
    if n:
        o.run_threads(n, CORES)
    return o.read_state() + o.get_raw() + (o.energy(),)


def assert_parity(g, o, tol, n_planets):
    pos_g, vel_g, st_g, t_g, Q_g, v_g, ns_g, _, E_g = g
    pos_o, vel_o, st_o, t_o, Q_o, v_o, ns_o, _, E_o = o
    assert np.array_equal(st_g, st_o)
    assert np.array_equal(ns_g, ns_o)
    assert np.allclose(t_g, t_o, rtol=1e-15, atol=0)
    sx = np.abs(pos_o).max(axis=(1, 2))[:, None, None]
    su = np.abs(vel_o).max(axis=(1, 2))[:, None, None]
    assert (np.abs(pos_g - pos_o) / sx).max() <= tol
    assert (np.abs(vel_g - vel_o) / su).max() <= tol
    live = np.arange(Q_o.shape[1])[None, :] < n_planets[:, None]
    nq = np.linalg.norm(Q_o, axis=2)
    nv = np.linalg.norm(v_o, axis=2)
    eq = np.linalg.norm(Q_g - Q_o, axis=2)
    ev = np.linalg.norm(v_g - v_o, axis=2)
    assert (eq[live] / nq[live]).max() <= tol
    assert (ev[live] / nv[live]).max() <= tol
    assert np.all(Q_g[~live] == 0) and np.all(v_g[~live] == 0)
    # energy: undefined (non-finite) for the same frozen states; exactly 0 for
    # all-massless systems at rest
    assert np.array_equal(np.isfinite(E_g), np.isfinite(E_o))
    fin = np.isfinite(E_o)
    assert np.all(np.abs(E_g[fin] - E_o[fin]) <= max(tol, 1e-13) * np.abs(E_o[fin]) + 1e-300)


# ------------------------------------------------------ special functions --

def test_own_rcp_rsqrt_against_cuda(whg):
    import torch
    rng = np.random.default_rng(0)
    x = np.concatenate([10.0 ** rng.uniform(-300, 300, 200000),
                        10.0 ** rng.uniform(-6, 6, 200000),
                        1.0 + rng.uniform(-1e-9, 1e-9, 1000), [1.0, 2.0, 4.0, 0.5, 3.0]])
    xt = torch.tensor(x, dtype=torch.float64, device="cuda")
    out = torch.empty(12 * x.size, dtype=torch.float64, device="cuda")
    whg.whg_test_special(xt, out)
    r = out.cpu().numpy().reshape(12, -1)
    ulp_rcp = np.spacing(np.abs(r[1]))
    ulp_rsq = np.spacing(np.abs(r[3]))
    # CUDA's 1/x is correctly rounded; rsqrt is within 1 ulp of exact.
    assert (np.abs(r[0] - r[1]) / ulp_rcp).max() <= 1.0
    assert (np.abs(r[2] - r[3]) / ulp_rsq).max() <= 2.0
    assert np.mean(r[0] == r[1]) > 0.9
    # and against the exact value (long double reference) for the planetary range
    sel = (x > 1e-6) & (x < 1e6)
    xl = x[sel].astype(np.longdouble)
    exact_rsq = 1 / np.sqrt(xl)
    err = np.abs(r[2][sel].astype(np.longdouble) - exact_rsq) / np.spacing(np.abs(r[3][sel]))
    assert float(err.max()) <= 1.5


def test_integer_pipe_refinement_within_one_ulp_of_fp64_forms(whg):
    """The reciprocal and the reciprocal square roots form their whole
    correction (1 - x y and its square, or 1 - x y^2 and its square) on the
    integer pipe, leaving one FP64 FMA: within one ulp of the same
    refinements written with FP64 operations (fma(-x, y, 1), y*y, y^2*y)
    over each routine's domain (1/x normal; x^(-3/2) normal) and both signs
    for 1/x, equal to them for most arguments, and within 1.5 ulp (1/x: 1 ulp)
    of the exact values."""
    import torch
    rng = np.random.default_rng(4)
    mag = 10.0 ** rng.uniform(-307, 307, 400000)
    x = np.concatenate([mag, -mag[:100000], np.ldexp(1.0, np.arange(-1021, 1023)),
                        np.nextafter(np.ldexp(1.0, np.arange(-1021, 1023)), np.inf),
                        1.0 + rng.uniform(-1e-7, 1e-7, 20000)])
    xt = torch.tensor(x, dtype=torch.float64, device="cuda")
    out = torch.empty(12 * x.size, dtype=torch.float64, device="cuda")
    whg.whg_test_special(xt, out)
    r = out.cpu().numpy().reshape(12, -1)

    def ulps(a, b):            # |a - b| in units of the double spacing at b
        return np.abs(a - b) / np.spacing(np.abs(np.asarray(b, np.float64)))

    inv = np.abs(x) < 2.0 ** 1021                            # 1/x normal
    assert inv.sum() > 500000
    assert ulps(r[0][inv], r[6][inv]).max() <= 1.0 and np.mean(r[0][inv] == r[6][inv]) > 0.9   # rcp
    pos = (x > 0) & (x < 4.0e307)
    assert ulps(r[2][pos], r[7][pos]).max() <= 1.0 and np.mean(r[2][pos] == r[7][pos]) > 0.9   # rsqrt
    cube = (x > 2.0 ** -680) & (x < 2.0 ** 681)               # x^(-3/2) normal
    assert ulps(r[8][cube], r[9][cube]).max() <= 1.0 and np.mean(r[8][cube] == r[9][cube]) > 0.9
    sel = pos & (x > 1e-200) & (x < 1e200)
    xl = np.asarray(x[sel], np.longdouble)
    assert float(ulps(r[8][sel].astype(np.longdouble), xl ** np.longdouble(-1.5)).max()) <= 1.5
    assert float(ulps(r[2][sel].astype(np.longdouble), 1 / np.sqrt(xl)).max()) <= 1.5
    sel = inv & (np.abs(x) > 1e-200) & (np.abs(x) < 1e200)
    assert float(ulps(r[0][sel].astype(np.longdouble), 1 / np.asarray(x[sel], np.longdouble)).max()) <= 1.0
    # 1/x^2 (the GR term's factor) within 1.5 ulp of exact where it is normal
    sq = (x > 1e-150) & (x < 1e150)
    xq = np.asarray(x[sq], np.longdouble)
    assert float(ulps(r[10][sq].astype(np.longdouble), 1 / (xq * xq)).max()) <= 1.5
    # outside the domains the outcomes stay non-finite as in the FP64 forms: a
    # zero or subnormal argument gives the same infinite 1/x and x^(-3/2) (a
    # coincident pair of planets then freezes its system as non-finite), inf
    # and NaN give NaN (the FP64 form gives some non-finite value)
    sp = np.array([0.0, -0.0, 5e-324, -1e-310, np.inf, -np.inf, np.nan])
    spt = torch.tensor(sp, dtype=torch.float64, device="cuda")
    o = torch.empty(12 * sp.size, dtype=torch.float64, device="cuda")
    whg.whg_test_special(spt, o)
    q = o.cpu().numpy().reshape(12, -1)
    assert np.all(np.isinf(q[0][:4])) and np.array_equal(np.signbit(q[0][:4]), np.signbit(sp[:4]))
    assert np.all(np.isnan(q[0][4:]))
    assert np.array_equal(q[0][:4], q[6][:4]) and not np.any(np.isfinite(q[6][4:]))
    assert np.all(np.isinf(q[8][:3])) and np.array_equal(q[8][:3], q[9][:3])    # x^(-3/2) of 0, -0, 5e-324
    assert np.all(np.isinf(q[10][:3]))                                         # 1/x^2 of 0, -0, 5e-324


def test_own_fp32_conversions_against_cuda(whg):
    """The integer-pipe FP64 -> FP32 -> FP64 round trip used for the Kepler
    solver's FP32 starting phase: equal to CUDA's round-toward-zero
    conversion in the FP32 normal range (and a truncation there by direct
    check); signed zero below it, signed infinity above it and for inf/NaN."""
    import torch
    rng = np.random.default_rng(3)
    mag = 10.0 ** rng.uniform(-45, 45, 200000)
    x = np.concatenate([mag * rng.choice([-1.0, 1.0], mag.size),
                        np.ldexp(1.0, np.arange(-130, 130)), -np.ldexp(1.0, np.arange(-130, 130)),
                        np.nextafter(np.ldexp(1.0, np.arange(-126, 128)), 0.0),
                        [0.0, -0.0, 1e-300, -1e-300, 1e300, -1e300, np.inf, -np.inf, np.nan,
                         float(np.finfo(np.float32).max), float(np.finfo(np.float32).tiny)]])
    xt = torch.tensor(x, dtype=torch.float64, device="cuda")
    out = torch.empty(12 * x.size, dtype=torch.float64, device="cuda")
    whg.whg_test_special(xt, out)
    r = out.cpu().numpy().reshape(12, -1)
    own, rz = r[4], r[5]
    ax = np.abs(x)
    normal = np.isfinite(x) & (ax >= 2.0 ** -126) & (ax < 2.0 ** 128)
    assert np.array_equal(own[normal], rz[normal])
    f = own[normal]
    assert np.array_equal(f, f.astype(np.float32).astype(np.float64))          # FP32 values
    assert np.all(np.signbit(f) == np.signbit(x[normal])) and np.all(np.abs(f) <= ax[normal])
    gap = ax[normal] - np.abs(f)
    with np.errstate(over="ignore"):                    # the spacing above FLT_MAX is inf
        ulp = np.spacing(np.abs(f).astype(np.float32)).astype(np.float64)
    assert np.all(gap < ulp)
    tiny = np.isfinite(x) & (ax < 2.0 ** -126)
    assert np.all(own[tiny] == 0.0) and np.array_equal(np.signbit(own[tiny]), np.signbit(x[tiny]))
    big = ~np.isfinite(x) | (ax >= 2.0 ** 128)
    assert np.all(np.isinf(own[big]))
    fin_big = big & ~np.isnan(x)
    assert np.array_equal(np.signbit(own[fin_big]), np.signbit(x[fin_big]))


# ------------------------------------------------------------- parity --

@pytest.mark.parametrize("n,tol", [(1, 1e-12), (10000, 1e-9)])
def test_two_planet_systems(whg, orc, n, tol):
    """Two-planet systems (seeds 0..9), GR off: 1 step and the full 1e4 steps."""
    ens = inputs.two_planet_system(0, 10)
    g = gpu_run(whg, ens, n, gr_mode=0)
    o = oracle_run(orc, ens, n, gr_mode=0)
    assert_parity(g, o, tol, ens.n_planets)


@pytest.mark.parametrize("gr_mode", [0, 1, 2])
@pytest.mark.parametrize("n,tol", [(1, 1e-12), (100, 1e-11)])
def test_solar_ensemble_short(whg, orc, gr_mode, n, tol):
    ens = inputs.solar_ensemble(1, 96)
    g = gpu_run(whg, ens, n, gr_mode=gr_mode)
    o = oracle_run(orc, ens, n, gr_mode=gr_mode)
    assert_parity(g, o, tol, ens.n_planets)


def test_solar_ensemble_1e4_window(whg, orc):
    """Solar-System-shaped ensemble, GR on, 1e4-step window (256 systems)."""
    ens = inputs.solar_ensemble(2, 256)
    g = gpu_run(whg, ens, 10000, gr_mode=1)
    o = oracle_run(orc, ens, 10000, gr_mode=1)
    assert_parity(g, o, 1e-9, ens.n_planets)


def test_newton_terms_6(whg, orc):
    ens = inputs.solar_ensemble(3, 64)
    g = gpu_run(whg, ens, 500, gr_mode=1, newton_terms=6)
    o = oracle_run(orc, ens, 500, gr_mode=1, newton_terms=6)
    assert_parity(g, o, 1e-10, ens.n_planets)


@pytest.mark.parametrize("lanes", [0, 8])
def test_uneven_planet_counts(whg, orc, lanes):
    """2..8 planets per system in one ensemble (padding lanes), and forcing
    8 lanes per system.  Some of these closely spaced systems (8-12 mutual Hill
    radii) are chaotic: in the oracle alone a 1e-15 relative change of the
    initial positions grows to ~1e-9 within 2000 steps but stays ~3e-12 over
    500, so the comparison uses 500 steps."""
    ens = inputs.compact_ensemble(5, 200)
    g = gpu_run(whg, ens, 500, gr_mode=1, lanes_per_system=lanes)
    o = oracle_run(orc, ens, 500, gr_mode=1)
    assert_parity(g, o, 1e-10, ens.n_planets)


@pytest.mark.parametrize("nmax", [1, 2, 3, 4, 5])
def test_lanes_per_system_variants(whg, orc, nmax):
    """G = 1, 2, 4, 4 (one padding lane), 8 (three padding lanes)."""
    ens = inputs.compact_ensemble(6, 100)
    ens = inputs.Ensemble(ens.masses[:, :1 + nmax].copy(), ens.pos[:, :1 + nmax].copy(),
                          ens.vel[:, :1 + nmax].copy(), np.minimum(ens.n_planets, nmax), ens.dt)
    ens = inputs._assemble(1.0, ens.masses[:, 1:], ens.pos[:, 1:] - ens.pos[:, :1],
                           ens.vel[:, 1:] - ens.vel[:, :1], ens.n_planets, ens.dt, "")
    g = gpu_run(whg, ens, 500, gr_mode=1)
    o = oracle_run(orc, ens, 500, gr_mode=1)
    assert_parity(g, o, 1e-10, ens.n_planets)


def test_massless_test_particles(whg, orc):
    """Massless planets (drift-only problem of the paper's Fig. 1)."""
    ens = inputs.test_particle(np.linspace(0.3, 2.0, 40), np.linspace(0.0, 0.6, 40),
                               np.linspace(0, 6, 40))
    g = gpu_run(whg, ens, 3000, gr_mode=0)
    o = oracle_run(orc, ens, 3000, gr_mode=0)
    assert_parity(g, o, 1e-10, ens.n_planets)


# --------------------------------------------------- determinism, resume --

def test_bitwise_run_to_run_and_launch_split(whg):
    ens = inputs.solar_ensemble(4, 300)
    a = gpu_run(whg, ens, 2000, gr_mode=1)
    b = gpu_run(whg, ens, 2000, gr_mode=1)
    c = gpu_run(whg, ens, 2000, chunks=[1, 999, 1000], gr_mode=1)
    d = gpu_run(whg, ens, 2000, gr_mode=1, steps_per_launch=7)
    for x in (b, c, d):
        for u, v in zip(a, x):
            assert np.array_equal(u, v)


def test_keep_unsynchronized_reads_do_not_change_bits(whg):
    ens = inputs.solar_ensemble(5, 64)
    it = whg.Integrator(64, 8)
    it.init(ens)
    for _ in range(4):
        it.step(250)
        it.read_state()
        it.energy()
    raw_a = it.get_raw()
    it2 = whg.Integrator(64, 8)
    it2.init(ens)
    it2.step(1000)
    for u, v in zip(raw_a, it2.get_raw()):
        assert np.array_equal(u, v)
    # checkpoint into a fresh context and resume bit-identically
    it3 = whg.Integrator(64, 8)
    it3.init(ens)
    it3.set_raw(*raw_a)
    it.step(333)
    it3.step(333)
    for u, v in zip(it.get_raw(), it3.get_raw()):
        assert np.array_equal(u, v)


def test_device_pointer_api_matches_host_api(whg):
    import torch
    ens = inputs.solar_ensemble(6, 50)
    it = whg.Integrator(50, 8)
    it.init(ens)
    it.step(123)
    ref = it.read_state()
    dev = whg.Integrator(50, 8)
    t = lambda a, dt=torch.float64: torch.tensor(a, dtype=dt, device="cuda")
    whg.whg_init_device(dev.ctx, t(ens.masses), t(ens.pos), t(ens.vel),
                        t(ens.n_planets, torch.int32), t(ens.dt))
    dev.step(123)
    pos = torch.empty((50, 9, 3), dtype=torch.float64, device="cuda")
    vel = torch.empty_like(pos)
    st = torch.empty(50, dtype=torch.int32, device="cuda")
    tt = torch.empty(50, dtype=torch.float64, device="cuda")
    whg.whg_read_state_device(dev.ctx, pos, vel, st, tt)
    E = torch.empty(50, dtype=torch.float64, device="cuda")
    whg.whg_energy_device(dev.ctx, E)
    torch.cuda.synchronize()
    assert np.array_equal(pos.cpu().numpy(), ref[0])
    assert np.array_equal(vel.cpu().numpy(), ref[1])
    assert np.array_equal(st.cpu().numpy(), ref[2])
    assert np.array_equal(E.cpu().numpy(), it.energy())


# ------------------------------------------------------ edge cases, status --

def test_status_freeze_matches_oracle(whg, orc):
    """An unbound planet (HYPERBOLIC) and a coincident pair (NONFINITE) freeze
    their systems at the same step as the oracle; the others run on."""
    ens = inputs.two_planet_system(3, 4)
    ens.vel[1, 2] *= 3.0                       # unbound outer planet
    ens.pos[2, 2] = ens.pos[2, 1]
    ens.vel[2, 2] = ens.vel[2, 1]              # same position and velocity
    g = gpu_run(whg, ens, 50, gr_mode=0)
    o = oracle_run(orc, ens, 50, gr_mode=0)
    assert list(g[2]) == [0, 2, 1, 0]
    assert_parity(g, o, 1e-12, ens.n_planets)


def test_invalid_inputs_are_rejected(whg):
    ens = inputs.two_planet_system(0, 3)
    it = whg.Integrator(3, 2)
    with pytest.raises(whg.WhgError) as e:
        it.step(1)
    assert e.value.code == whg.WHG_ESTATE
    for bad in ("dt", "mass", "nan", "nplan", "onstar"):
        e2 = inputs.Ensemble(ens.masses.copy(), ens.pos.copy(), ens.vel.copy(),
                             ens.n_planets.copy(), ens.dt.copy())
        if bad == "dt":
            e2.dt[1] = 0.0
        elif bad == "mass":
            e2.masses[1, 2] = -1e-6
        elif bad == "nan":
            e2.vel[2, 1, 0] = np.nan
        elif bad == "nplan":
            e2.n_planets[0] = 3
        else:
            e2.pos[0, 1] = e2.pos[0, 0]
        with pytest.raises(whg.WhgError) as e:
            it.init(e2)
        assert e.value.code == whg.WHG_EINVAL
        assert "system" in whg.whg_last_error(it.ctx)
    with pytest.raises(whg.WhgError):
        whg.whg_create(0, 2)
    with pytest.raises(whg.WhgError):
        whg.whg_create(4, 9)


def test_device_init_marks_invalid_systems(whg):
    import torch
    ens = inputs.two_planet_system(1, 4)
    ens.dt[2] = -1.0
    it = whg.Integrator(4, 2)
    t = lambda a, dt=torch.float64: torch.tensor(a, dtype=dt, device="cuda")
    whg.whg_init_device(it.ctx, t(ens.masses), t(ens.pos), t(ens.vel), t(ens.n_planets, torch.int32),
                        t(ens.dt))
    it.step(10)
    _, _, st, tt = it.read_state()
    assert list(st) == [0, 0, whg.WHG_STATUS_INVALID, 0]
    assert tt[2] == 0.0 and tt[0] > 0


def test_zero_steps_and_single_system(whg, orc):
    ens = inputs.two_planet_system(7, 1)
    g = gpu_run(whg, ens, 0, gr_mode=0)
    assert np.allclose(g[0], ens.pos, rtol=0, atol=1e-15)
    o = oracle_run(orc, ens, 0, gr_mode=0)
    assert_parity(g, o, 1e-14, ens.n_planets)


@pytest.mark.parametrize("S", [1, 31, 33, 4097])
def test_ragged_system_counts(whg, orc, S):
    """System counts that leave a partial block / warp (padding systems)."""
    ens = inputs.solar_ensemble(8, S)
    g = gpu_run(whg, ens, 20, gr_mode=1)
    o = oracle_run(orc, ens, 20, gr_mode=1)
    assert_parity(g, o, 1e-12, ens.n_planets)


def test_full_size_ensemble_sampled(whg, orc):
    """2^20 systems (the largest sweep size), 20 steps; 512 sampled systems
    checked against the oracle one by one."""
    S = 1 << 20
    ens = inputs.solar_ensemble(9, 4096).tile(S)
    rng = np.random.default_rng(1)
    idx = np.sort(rng.choice(S, 512, replace=False))
    it = whg.Integrator(S, 8)
    it.init(ens)
    it.step(20)
    pos, vel, st, t = it.read_state()
    it.close()
    sub = ens.subset(idx)
    o = orc.OracleEnsemble(512, 8, gr_mode=1)
    o.init(sub)
    o.run_threads(20, CORES)
    po, vo, so, to = o.read_state()
    assert np.array_equal(st[idx], so)
    sx = np.abs(po).max(axis=(1, 2))[:, None, None]
    assert (np.abs(pos[idx] - po) / sx).max() <= 1e-12
    # systems that are copies of one another stay bitwise identical
    assert np.array_equal(pos[5], pos[5 + 4096])


def test_energy_error_statistics_match(whg, orc):
    """Relative energy errors over a 2e4-step run: same per-system values
    (to 1e-12 absolute) and the same distribution."""
    ens = inputs.solar_ensemble(10, 128)
    it = whg.Integrator(128, 8)
    it.init(ens)
    E0 = it.energy()
    it.step(20000)
    dEg = it.energy() / E0 - 1
    o = orc.OracleEnsemble(128, 8, gr_mode=1)
    o.init(ens)
    E0o = o.energy()
    o.run_threads(20000, CORES)
    dEo = o.energy() / E0o - 1
    assert np.abs(dEg - dEo).max() < 1e-12
    assert np.abs(dEg).max() < 1e-6


def test_energy_error_distributions_match_on_compact_systems(whg, orc):
    """512 compact systems (2-8 planets, 8-12 mutual Hill radii) over 5e4
    steps.  Many of them are chaotic, so per-system values from the GPU and
    the oracle may separate, but the distributions of log10 |E/E0 - 1| over
    the systems both leave running agree (two-sample Kolmogorov-Smirnov)."""
    stats = pytest.importorskip("scipy.stats")
    ens = inputs.compact_ensemble(21, 512)
    it = whg.Integrator(512, 8, gr_mode=1)
    it.init(ens)
    E0 = it.energy()
    it.step(50000)
    st = it.read_state()[2]
    dEg = it.energy() / E0 - 1
    it.close()
    o = orc.OracleEnsemble(512, 8, gr_mode=1)
    o.init(ens)
    E0o = o.energy()
    o.run_threads(50000, CORES)
    sto = o.read_state()[2]
    dEo = o.energy() / E0o - 1
    ok = (st == 0) & (sto == 0) & np.isfinite(dEg) & np.isfinite(dEo) & (dEg != 0) & (dEo != 0)
    assert ok.sum() >= 450
    res = stats.ks_2samp(np.log10(np.abs(dEg[ok])), np.log10(np.abs(dEo[ok])))
    assert res.pvalue > 0.01, res


# ------------------------------------------------------------ stop rules --

def test_ejection_stop_step_matches_oracle(whg, orc):
    """A test particle on an e = 0.9 orbit passes 1.5 a: the GPU stops it at
    the same step as the oracle (whose step is pinned to the two-body time)."""
    ens = inputs.test_particle(np.full(8, 1.0), np.full(8, 0.9), np.linspace(0.0, 1.0, 8), dt=0.01)
    it = whg.Integrator(8, 1, gr_mode=0, eject_factor=1.5)
    it.init(ens)
    it.step(1000)
    g = it.read_state()
    o = orc.OracleEnsemble(8, 1, gr_mode=0, eject_factor=1.5)
    o.init(ens)
    o.step(1000)
    r = o.read_state()
    assert np.all(g[2] == whg.WHG_STATUS_EJECTED)
    assert np.array_equal(g[2], r[2]) and np.array_equal(g[3], r[3])
    assert np.abs(g[0] - r[0]).max() < 1e-12


def test_close_encounter_stop_step_matches_oracle(whg, orc):
    """Two nearly massless planets on crossing orbits (as in the oracle's pin),
    in several phases: the same stop step as the oracle."""
    sys_list = []
    for k in range(6):
        x1, v1 = inputs.elements_to_state(1.0, 1.0, 0.0, 0.0, 0.0, 0.0, 0.3 + 0.1 * k)
        x2, v2 = inputs.elements_to_state(1.0, 1.3, 0.35, 0.0, 0.0, 0.0, 2.0)
        sys_list.append((np.stack([x1, x2]), np.stack([v1, v2])))
    x = np.stack([a for a, _ in sys_list])
    v = np.stack([b for _, b in sys_list])
    ens = inputs._assemble(1.0, np.full((6, 2), 1e-12), x, v, np.full(6, 2), np.full(6, 0.005), "")
    it = whg.Integrator(6, 2, gr_mode=0, close_encounter_hill=2000.0)
    it.init(ens)
    it.step(20000)
    g = it.read_state()
    o = orc.OracleEnsemble(6, 2, gr_mode=0, encounter_hill=2000.0)
    o.init(ens)
    o.step(20000)
    r = o.read_state()
    assert np.all(r[2] == whg.WHG_STATUS_CLOSE_ENCOUNTER)
    assert np.array_equal(g[2], r[2]) and np.array_equal(g[3], r[3])


def test_stop_rules_on_compact_ensemble(whg, orc):
    """Mixed planet counts with both stop rules on a short horizon where
    trajectories still agree: same statuses and stop steps as the oracle."""
    ens = inputs.compact_ensemble(12, 300)
    kw = dict(close_encounter_hill=6.0, eject_factor=3.0)
    g = gpu_run(whg, ens, 400, gr_mode=1, **kw)
    o = orc.OracleEnsemble(300, 8, gr_mode=1, encounter_hill=6.0, eject_factor=3.0)
    o.init(ens)
    o.run_threads(400, CORES)
    r = o.read_state() + o.get_raw() + (o.energy(),)
    assert (r[2] == whg.WHG_STATUS_CLOSE_ENCOUNTER).sum() >= 5
    assert_parity(g, r, 1e-10, ens.n_planets)


def test_device_init_mixed_planet_counts(whg, orc):
    """Device-pointer init of a mixed ensemble (the layout reads the planet
    counts back once) matches the host-pointer path bit for bit."""
    import torch
    ens = inputs.compact_ensemble(13, 120)
    a = whg.Integrator(120, 8)
    a.init(ens)
    a.step(300)
    ref = a.read_state()
    b = whg.Integrator(120, 8)
    t = lambda x, dt=torch.float64: torch.tensor(x, dtype=dt, device="cuda")
    whg.whg_init_device(b.ctx, t(ens.masses), t(ens.pos), t(ens.vel), t(ens.n_planets, torch.int32),
                        t(ens.dt))
    b.step(300)
    out = b.read_state()
    for u, v in zip(ref, out):
        assert np.array_equal(u, v)


@pytest.mark.parametrize("n,tol", [(1, 1e-12), (10000, 1e-9)])
def test_merged_jumps_match_oracle(whg, orc, n, tol):
    """Without GR, one J(dt) before I(dt) per step (Sec. 3.1), on both sides."""
    ens = inputs.two_planet_system(0, 10)
    g = gpu_run(whg, ens, n, gr_mode=0, merge_jumps=True)
    o = oracle_run(orc, ens, n, gr_mode=0, merge_jumps=True)
    assert_parity(g, o, tol, ens.n_planets)
    s = inputs.solar_ensemble(13, 64)
    assert_parity(gpu_run(whg, s, 500, gr_mode=0, merge_jumps=True),
                  oracle_run(orc, s, 500, gr_mode=0, merge_jumps=True), 1e-11, s.n_planets)


@pytest.mark.parametrize("case", ["two_planet_1", "two_planet_1e4", "solar_1", "solar_1e4", "compact",
                                  "particles", "status"])
def test_halley_fp32_matches_oracle(whg, orc, case):
    """halley_fp32 = 1: the Kepler solver's initial guess and Halley phase in
    FP32 (FP64 Newton phase), against the all-FP64 oracle at the same
    tolerances as the default all-FP64 path."""
    if case.startswith("two_planet"):
        ens, gr = inputs.two_planet_system(0, 10), 0
        n, tol = (1, 1e-12) if case.endswith("_1") else (10000, 1e-9)
    elif case.startswith("solar"):
        ens, gr = inputs.solar_ensemble(2, 256), 1
        n, tol = (1, 1e-12) if case.endswith("_1") else (10000, 1e-9)
    elif case == "compact":
        ens, n, tol, gr = inputs.compact_ensemble(5, 200), 500, 1e-10, 1
    elif case == "particles":
        ens = inputs.test_particle(np.linspace(0.3, 2.0, 40), np.linspace(0.0, 0.6, 40), np.linspace(0, 6, 40))
        n, tol, gr = 3000, 1e-10, 0
    else:
        ens = inputs.two_planet_system(3, 4)
        ens.vel[1, 2] *= 3.0
        ens.pos[2, 2] = ens.pos[2, 1]
        ens.vel[2, 2] = ens.vel[2, 1]
        n, tol, gr = 50, 1e-12, 0
    g = gpu_run(whg, ens, n, gr_mode=gr, halley_fp32=True)
    o = oracle_run(orc, ens, n, gr_mode=gr)
    assert_parity(g, o, tol, ens.n_planets)
    if case == "status":
        assert list(g[2]) == [0, 2, 1, 0]


def test_uneven_batch_full_size_sampled(whg, orc):
    """65,536 compact systems with 2..8 planets in one ensemble, both stop
    rules on (a pair closer than 1 mutual Hill radius, a planet beyond 100x
    the largest initial a), in the launch configuration the benchmark times
    (100-step launches replayed as CUDA graphs of 16).  400 steps; 512
    sampled systems checked one by one against the oracle (statuses, stop
    steps, states to 1e-10)."""
    S = 1 << 16
    ens = inputs.compact_ensemble(303, S)
    kw = dict(close_encounter_hill=1.0, eject_factor=100.0)
    it = whg.Integrator(S, 8, gr_mode=1, steps_per_launch=100, graph_launches=16, **kw)
    it.init(ens)
    it.step(400)
    pos, vel, st, t = it.read_state()
    Q, v, ns, _ = it.get_raw()
    it.close()
    rng = np.random.default_rng(5)
    idx = np.sort(rng.choice(S, 512, replace=False))
    sub = ens.subset(idx)
    o = orc.OracleEnsemble(512, 8, gr_mode=1, encounter_hill=1.0, eject_factor=100.0)
    o.init(sub)
    o.run_threads(400, CORES)
    ref = o.read_state() + o.get_raw() + (o.energy(),)
    it2 = whg.Integrator(512, 8, gr_mode=1, **kw)        # the same systems alone, for the energy
    it2.init(sub)
    it2.step(400)
    E = it2.energy()
    it2.close()
    g = (pos[idx], vel[idx], st[idx], t[idx], Q[idx], v[idx], ns[idx], None, E)
    assert_parity(g, ref, 1e-10, sub.n_planets)
    assert set(np.unique(st)) <= {0, whg.WHG_STATUS_CLOSE_ENCOUNTER, whg.WHG_STATUS_EJECTED,
                                  whg.WHG_STATUS_CLOSE_ENCOUNTER | whg.WHG_STATUS_EJECTED}


@pytest.mark.parametrize("case", ["solar_1", "solar_1e4", "compact", "stop_rules"])
def test_full_rotation_schedule_matches_oracle(whg, orc, case):
    """interaction_schedule = 1 (all L-1 rotations, no third-law reactions):
    the same map as the oracle at the default path's tolerances, and the same
    close-encounter stops."""
    kw, okw = {}, {}
    if case.startswith("solar"):
        ens = inputs.solar_ensemble(2, 256)
        n, tol = (1, 1e-12) if case == "solar_1" else (10000, 1e-9)
    elif case == "compact":
        ens, n, tol = inputs.compact_ensemble(5, 200), 500, 1e-10
    else:
        ens, n, tol = inputs.compact_ensemble(12, 300), 400, 1e-10
        kw = dict(close_encounter_hill=6.0, eject_factor=3.0)
        okw = dict(encounter_hill=6.0, eject_factor=3.0)
    g = gpu_run(whg, ens, n, gr_mode=1, interaction_schedule=1, **kw)
    o = oracle_run(orc, ens, n, gr_mode=1, **okw)
    assert_parity(g, o, tol, ens.n_planets)


def test_bench_workload_sampled():
    """The benchmark's own workload and launch configuration: its 4096
    Solar-System-shaped systems (bench.rank_workload, rank 0) advanced by one
    1e4-step launch (the bench's chunk); 128 sampled systems against the
    oracle to 1e-9, every system finite and running."""
    import types
    import bench
    from paper_2307_05683_gb300 import build, whg
    import oracle as orc_mod
    build.build()
    orc_mod.build()
    args = types.SimpleNamespace(seed=2024, systems=4096)
    ens = bench.rank_workload(args, 0)
    it = whg.Integrator(4096, 8, gr_mode=1)
    it.init(ens)
    l0 = it.launches
    it.step(10000)
    assert it.launches - l0 == 1
    pos, vel, st, t = it.read_state()
    it.close()
    assert np.all(st == 0) and np.all(np.isfinite(pos)) and np.all(np.isfinite(vel))
    idx = np.sort(np.random.default_rng(11).choice(4096, 128, replace=False))
    sub = ens.subset(idx)
    o = orc_mod.OracleEnsemble(128, 8, gr_mode=1)
    o.init(sub)
    o.run_threads(10000, CORES)
    po, vo, so, to = o.read_state()
    assert np.array_equal(st[idx], so) and np.allclose(t[idx], to, rtol=1e-15, atol=0)
    sx = np.abs(po).max(axis=(1, 2))[:, None, None]
    su = np.abs(vo).max(axis=(1, 2))[:, None, None]
    assert (np.abs(pos[idx] - po) / sx).max() <= 1e-9
    assert (np.abs(vel[idx] - vo) / su).max() <= 1e-9
