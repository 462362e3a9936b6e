"""Pins for the oracle's sub-steps and the full Wisdom-Holman map (Eq. 2).

Independent references only: inertial-frame energy and angular momentum
written out here, brute-force pair sums at 40 digits (mpmath), finite
differences of the GR potential, the textbook GR perihelion precession rate,
time reversibility, second-order convergence, and a high-order Runge-Kutta
integration (scipy DOP853) of the inertial N-body equations.
"""
import mpmath as mp
import numpy as np
import pytest

from paper_2307_05683_gb300 import inputs

mp.mp.dps = 40
C = inputs.C_LIGHT


def inertial_energy(m, x, u, gr_c=None):
    """Sum of kinetic energies minus all pair potentials (+ 1/r^2 GR term)."""
    E = 0.5 * np.sum(m[:, None] * u * u)
    for k in range(len(m)):
        for l in range(k + 1, len(m)):
            E -= m[k] * m[l] / np.linalg.norm(x[k] - x[l])
    if gr_c is not None:
        for i in range(1, len(m)):
            E -= 3.0 * m[i] * m[0] ** 2 / (gr_c ** 2 * np.sum((x[i] - x[0]) ** 2))
    return E


def inertial_L(m, x, u):
    return np.sum(m[:, None] * np.cross(x, u), axis=0)


def dh_L(m, Q, v):
    return np.sum(m[:, None] * np.cross(Q, v), axis=0)


def make(orc, ens, **kw):
    o = orc.OracleEnsemble(ens.n_systems, ens.max_planets, **kw)
    o.init(ens)
    return o


# ------------------------------------------------------------- coordinates --

def test_dh_round_trip_and_energy(orc):
    ens = inputs.solar_ensemble(3, 4)
    for gr in (0, 1):
        o = make(orc, ens, gr_mode=gr)
        pos, vel, st, t = o.read_state()
        assert np.all(st == 0) and np.all(t == 0)
        scale = np.abs(ens.pos).max()
        assert np.abs(pos - ens.pos).max() < 4e-16 * scale * 8
        assert np.abs(vel - ens.vel).max() < 4e-16 * np.abs(ens.vel).max() * 8
        E = o.energy()
        for s in range(ens.n_systems):
            Ei = inertial_energy(ens.masses[s], ens.pos[s], ens.vel[s], C if gr else None)
            assert E[s] == pytest.approx(Ei, rel=1e-13)


def test_dh_coordinates_definition(orc):
    """Q_i = x_i - x_0 and v_i = u_i - V_cm (Sec. 3.1)."""
    ens = inputs.two_planet_system(1, 3)
    o = make(orc, ens)
    Q, v, ns, st = o.get_raw()
    for s in range(3):
        m = ens.masses[s]
        vcm = (m[:, None] * ens.vel[s]).sum(0) / m.sum()
        assert np.allclose(Q[s], ens.pos[s, 1:] - ens.pos[s, 0], rtol=0, atol=1e-15)
        assert np.allclose(v[s], ens.vel[s, 1:] - vcm, rtol=0, atol=1e-15)


# ---------------------------------------------------------------- sub-steps --

def test_jump_step(orc):
    """Eq. 6: every Q_i moves by (h/m_0) sum_j m_j v_j; v is bit-unchanged."""
    ens = inputs.solar_ensemble(5, 2)
    o = make(orc, ens)
    Q0, v0, _, _ = o.get_raw()
    h = 0.037
    o.substep(1, "jump", h)
    Q1, v1, _, _ = o.get_raw()
    assert np.array_equal(v1, v0) and np.array_equal(Q1[0], Q0[0])
    m = ens.masses[1, 1:]
    shift = h / ens.masses[1, 0] * (m[:, None] * v0[1]).sum(0)
    d = Q1[1] - Q0[1]
    ulp = np.spacing(np.abs(Q0[1]).max())          # d is a difference of two positions
    assert np.abs(d - shift[None, :]).max() <= 2 * ulp
    assert np.abs(d - d[0]).max() <= 2 * ulp


def test_interaction_step_brute_force(orc):
    """Eq. 5 against all ordered pairs at 40 digits; third law sum_i m_i dv_i = 0."""
    ens = inputs.solar_ensemble(9, 1)
    o = make(orc, ens)
    Q, v0, _, _ = o.get_raw()
    h = 0.02
    o.substep(0, "interaction", h)
    _, v1, _, _ = o.get_raw()
    m = ens.masses[0, 1:]
    for i in range(8):
        acc = [mp.mpf(0)] * 3
        for j in range(8):
            if j == i:
                continue
            d = [mp.mpf(Q[0, i, c]) - mp.mpf(Q[0, j, c]) for c in range(3)]
            r3 = mp.sqrt(sum(x * x for x in d)) ** 3
            for c in range(3):
                acc[c] -= mp.mpf(m[j]) * d[c] / r3
        v_ref = np.array([float(mp.mpf(v0[0, i, c]) + h * acc[c]) for c in range(3)])
        ulp = np.spacing(np.abs(v0[0, i]).max())
        assert np.abs(v1[0, i] - v_ref).max() <= 2 * ulp
    # third law: total planet momentum changes only by rounding of each v_i
    mom = (m[:, None] * (v1[0] - v0[0])).sum(0)
    assert np.abs(mom).max() <= 2 * np.sum(m * np.spacing(np.abs(v0[0]).max(axis=1)))


@pytest.mark.parametrize("mode", [1, 2])
def test_gr_kick_is_minus_grad_potential(orc, mode):
    """GR kick = h * (-grad Phi), Phi = -3 (G m_0)^2 / (c^2 r^2) per unit mass,
    by central finite differences; mode 2 subtracts sum_j (m_j/m_0) a_j."""
    ens = inputs.solar_ensemble(4, 1)
    c = 50.0
    o = make(orc, ens, gr_mode=mode, c_light=c)
    Q, v0, _, _ = o.get_raw()
    h = 0.05
    o.substep(0, "gr", h)
    _, v1, _, _ = o.get_raw()
    m0, m = ens.masses[0, 0], ens.masses[0, 1:]

    def phi(q):
        return -3.0 * m0 ** 2 / (c ** 2 * (q @ q))

    acc = np.zeros((8, 3))
    for i in range(8):
        for k in range(3):
            eps = 1e-6 * np.linalg.norm(Q[0, i])
            dq = np.zeros(3)
            dq[k] = eps
            acc[i, k] = -(phi(Q[0, i] + dq) - phi(Q[0, i] - dq)) / (2 * eps)
    if mode == 2:
        acc = acc - (m[:, None] / m0 * acc).sum(0)[None, :]
    err = np.linalg.norm(v1[0] - v0[0] - h * acc, axis=1)
    tol = 1e-8 * np.linalg.norm(h * acc, axis=1) + 4 * np.spacing(np.abs(v0[0]).max(axis=1))
    assert np.all(err <= tol)


def _omega_from_lrl(Q, v, mu=1.0):
    L = np.cross(Q, v)
    A = np.cross(v, L) / mu - Q / np.linalg.norm(Q)
    return np.arctan2(A[1], A[0])


def test_gr_perihelion_precession_rate(orc):
    """A massless planet under the GR term precesses at the textbook rate
    3 (G m_0)^{3/2} / (c^2 a^{5/2} (1 - e^2)) (the rate the 1/r^2 potential of
    Nobili & Roxburgh is built to reproduce)."""
    a, e, cl = 0.387, 0.2, 1000.0
    P = 2 * np.pi * a ** 1.5
    n = 200 * 30
    ens = inputs.test_particle(a, e, 0.0, dt=P / 30)
    rates = {}
    for mode in (0, 1):
        o = make(orc, ens, gr_mode=mode, c_light=cl)
        _, _, _, t0 = o.read_state()
        w0 = _omega_from_lrl(*[x[0, 0] for x in o.get_raw()[:2]])
        o.step(n)
        pos, vel, st, t = o.read_state()
        w1 = _omega_from_lrl(pos[0, 1] - pos[0, 0], vel[0, 1] - vel[0, 0])
        rates[mode] = (w1 - w0) / t[0]
    expect = 3.0 / (cl ** 2 * a ** 2.5 * (1 - e * e))
    assert abs(rates[0]) < 1e-3 * expect
    assert rates[1] == pytest.approx(expect, rel=5e-3)


# ------------------------------------------------------------------ the map --

def test_fused_drifts_equal_eq2_composition(orc):
    """n fused steps + output sync == n applications of
    K(dt/2) J(dt/2) I(dt) J(dt/2) K(dt/2) built from single sub-steps (Eq. 2)."""
    ens = inputs.solar_ensemble(11, 1)
    for gr in (0, 1):
        a = make(orc, ens, gr_mode=gr)
        b = make(orc, ens, gr_mode=gr)
        dt = ens.dt[0]
        n = 50
        a.step(n)
        for _ in range(n):
            b.substep(0, "kepler", dt / 2)
            b.substep(0, "jump", dt / 2)
            b.substep(0, "interaction", dt)
            if gr:
                b.substep(0, "gr", dt)
            b.substep(0, "jump", dt / 2)
            b.substep(0, "kepler", dt / 2)
        pa, va, _, _ = a.read_state()
        Qb, vb, _, _ = b.get_raw()
        Qa = pa[0, 1:] - pa[0, 0]
        assert np.abs(Qa - Qb[0]).max() < 1e-13 * np.abs(Qb).max()


@pytest.mark.parametrize("n,tol", [(100, 1e-13), (1000, 1e-11)])
def test_time_reversibility(orc, n, tol):
    """n steps, sync, flip velocities, n steps, flip back: the start again
    (backward integration by flipping velocities, Sec. 3.5 list).  The residual
    is roundoff, which grows along the orbit roughly like n^2."""
    for seed in range(3):
        ens = inputs.two_planet_system(seed, 1)
        o = make(orc, ens)
        o.step(n)
        pos, vel, _, _ = o.read_state()
        back = inputs.Ensemble(ens.masses, pos, -vel, ens.n_planets, ens.dt)
        o2 = make(orc, back)
        o2.step(n)
        p2, v2, _, _ = o2.read_state()
        assert np.abs(p2 - ens.pos).max() < tol * np.abs(ens.pos).max()
        assert np.abs(-v2 - ens.vel).max() < tol * np.abs(ens.vel).max()


def test_angular_momentum_conserved_by_each_substep(orc):
    ens = inputs.solar_ensemble(2, 1)
    o = make(orc, ens, gr_mode=1)
    m = ens.masses[0, 1:]
    Q, v, _, _ = o.get_raw()
    L0 = dh_L(m, Q[0], v[0])
    for which, h in [("kepler", 0.07), ("jump", 0.035), ("interaction", 0.07), ("gr", 0.07)]:
        o.substep(0, which, h)
        Q, v, _, _ = o.get_raw()
        assert np.abs(dh_L(m, Q[0], v[0]) - L0).max() < 1e-15 * np.linalg.norm(L0) * 20, which


def test_total_L_conserved_and_matches_inertial(orc):
    ens = inputs.solar_ensemble(6, 1)
    o = make(orc, ens, gr_mode=1)
    L0 = inertial_L(ens.masses[0], ens.pos[0], ens.vel[0])
    o.step(2000)
    pos, vel, st, _ = o.read_state()
    L1 = inertial_L(ens.masses[0], pos[0], vel[0])
    assert st[0] == 0
    assert np.abs(L1 - L0).max() < 1e-13 * np.linalg.norm(L0)


def test_energy_error_second_order_and_bounded(orc):
    """Energy error O(eps dt^2) (Sec. 3.1): halving dt cuts the peak error ~4x;
    no secular growth between the first and second half of the run."""
    ens = inputs.two_planet_system(4, 1)
    peaks = []
    for div in (1, 2):
        e2 = inputs.Ensemble(ens.masses, ens.pos, ens.vel, ens.n_planets, ens.dt / div)
        o = make(orc, e2)
        E0 = o.energy()[0]
        errs = []
        for _ in range(200):
            o.step(15 * div)
            errs.append(abs(o.energy()[0] / E0 - 1))
        errs = np.array(errs)
        peaks.append(errs.max())
        assert errs[100:].max() < 1.5 * errs[:100].max() + 1e-14
    assert 3.0 < peaks[0] / peaks[1] < 5.5
    assert peaks[0] < 1e-6


def _nbody_rhs(t, y, m):
    n = len(m)
    x = y[:3 * n].reshape(n, 3)
    a = np.zeros_like(x)
    for k in range(n):
        for l in range(n):
            if k != l:
                d = x[l] - x[k]
                a[k] += m[l] * d / np.linalg.norm(d) ** 3
    return np.concatenate([y[3 * n:], a.ravel()])


@pytest.mark.parametrize("seed", [0, 1])
def test_against_high_order_integrator(orc, seed):
    """2 planets over 5 inner orbits vs DOP853 (rtol 1e-13) on the inertial
    equations: the WH position error scales as dt^2 and stays small."""
    from scipy.integrate import solve_ivp
    ens = inputs.two_planet_system(seed, 1)
    ens.masses[0, 1:] = [3e-4, 1e-4]          # resolvable coupling, same orbits
    ens = inputs.Ensemble(*inputs._assemble(1.0, ens.masses[:, 1:],
                                            ens.pos[:, 1:] - ens.pos[:, :1],
                                            ens.vel[:, 1:] - ens.vel[:, :1],
                                            ens.n_planets, ens.dt, "").__dict__.values())
    m = ens.masses[0]
    T = 5 * 2 * np.pi
    y0 = np.concatenate([ens.pos[0].ravel(), ens.vel[0].ravel()])
    ref = solve_ivp(_nbody_rhs, (0, T), y0, method="DOP853", rtol=1e-13, atol=1e-15,
                    args=(m,)).y[:, -1]
    xr = ref[:9].reshape(3, 3)
    errs = []
    for div in (30, 60):
        dt = 2 * np.pi / div
        nsteps = int(round(T / dt))
        e2 = inputs.Ensemble(ens.masses, ens.pos, ens.vel, ens.n_planets, np.array([dt]))
        o = make(orc, e2)
        o.step(nsteps)
        pos, _, _, _ = o.read_state()
        errs.append(np.abs(pos[0] - xr).max())
    assert errs[0] < 2e-5
    assert 3.0 < errs[0] / errs[1] < 5.0


def test_keep_unsynchronized_is_bitwise_reproducible(orc):
    """Reading (synchronizing a copy) mid-run leaves the final bits unchanged,
    and a raw checkpoint resumes bit-identically (Sec. 3.5 list)."""
    ens = inputs.solar_ensemble(8, 3)
    a = make(orc, ens, gr_mode=1)
    b = make(orc, ens, gr_mode=1)
    a.step(300)
    for _ in range(3):
        b.step(100)
        b.read_state()
        b.energy()
    ra, rb = a.get_raw(), b.get_raw()
    for x, y in zip(ra, rb):
        assert np.array_equal(x, y)
    c = make(orc, ens, gr_mode=1)
    c.set_raw(*b.get_raw())
    a.step(77)
    c.step(77)
    assert np.array_equal(a.read_state()[0], c.read_state()[0])


def test_nonfinite_step_rolls_back_and_freezes(orc):
    """Two planets with the same position and velocity: the interaction gives
    non-finite values;
    that system is rolled back and frozen (NONFINITE), the other runs on."""
    ens = inputs.two_planet_system(0, 2)
    ens.pos[1, 2] = ens.pos[1, 1]
    ens.vel[1, 2] = ens.vel[1, 1]
    o = make(orc, ens)
    o.step(10)
    pos, vel, st, t = o.read_state()
    assert st[0] == 0 and st[1] == 1
    assert t[0] == pytest.approx(10 * ens.dt[0]) and t[1] == 0.0
    assert np.array_equal(pos[1], o.read_state()[0][1])
    assert np.all(np.isfinite(pos[1]))


def test_merged_jumps_are_the_same_map_without_gr(orc):
    """Sec. 3.1: without GR the jump commutes with the interaction, so
    J(dt/2) I(dt) J(dt/2) and J(dt) I(dt) are the same map (rounding aside);
    with the GR term the option is ignored."""
    ens = inputs.solar_ensemble(12, 3)
    a = make(orc, ens, gr_mode=0)
    b = make(orc, ens, gr_mode=0, merge_jumps=True)
    a.step(500)
    b.step(500)
    pa, va, _, _ = a.read_state()
    pb, vb, _, _ = b.read_state()
    assert np.abs(pa - pb).max() < 1e-12 * np.abs(pa).max()
    assert not np.array_equal(pa, pb)                    # a different operation order
    c = make(orc, ens, gr_mode=1)
    d = make(orc, ens, gr_mode=1, merge_jumps=True)
    c.step(100)
    d.step(100)
    for x, y in zip(c.get_raw(), d.get_raw()):
        assert np.array_equal(x, y)
