"""Pins for the oracle's optional ensemble stopping rules (close encounter,
ejection): the step at which a system is stopped must match the step
predicted from exact two-body orbits (the bodies involved are massless or
nearly so, so the map reduces to exact Kepler drifts).

Timing of the checks: the ejection check runs at the start of each step's
drift, on the unsynchronized state, which is at time 0 for the first step and
(k - 1/2) dt for step k >= 1; the close-encounter check runs in the
interaction step of step k, at time (k + 1/2) dt.  A stopped step is rolled
back, so the system reports k completed steps.
"""
import mpmath as mp
import numpy as np

from paper_2307_05683_gb300 import inputs

mp.mp.dps = 30


def kepler_pos(a, e, M0, t, mu=1.0):
    n = np.sqrt(mu / a ** 3)
    M = M0 + n * t
    E = float(mp.findroot(lambda E: E - e * mp.sin(E) - M, M))
    return np.array([a * (np.cos(E) - e), a * np.sqrt(1 - e * e) * np.sin(E), 0.0])


def test_ejection_step_matches_two_body_crossing(orc):
    a, e, factor, dt = 1.0, 0.9, 1.5, 0.01
    ens = inputs.test_particle(a, e, 0.0, dt=dt)            # starts at pericentre
    o = orc.OracleEnsemble(1, 1, gr_mode=0, eject_factor=factor)
    o.init(ens)
    o.step(1000)
    _, _, st, t = o.read_state()
    assert st[0] == 16
    k = int(round(t[0] / dt))                               # completed steps
    # analytic: r(t) = a (1 - e cos E) crosses factor * a at E* ...
    Estar = np.arccos((1 - factor) / e)
    tstar = (Estar - e * np.sin(Estar)) / np.sqrt(1.0 / a ** 3)
    # ... and the stop happens at the first drift start with (k - 1/2) dt > t*
    kexp = int(np.floor(tstar / dt + 0.5)) + 1
    assert k == kexp
    assert (k - 0.5) * dt > tstar > (k - 1.5) * dt


def test_close_encounter_step_matches_two_body_prediction(orc):
    dt, K = 0.005, 2000.0
    m = 1e-12
    # two nearly massless planets on crossing orbits: a circular one and an
    # eccentric one whose orbit cuts through it
    a1, e1, M1 = 1.0, 0.0, 0.3
    a2, e2, M2 = 1.3, 0.35, 2.0
    x1, v1 = inputs.elements_to_state(1.0, a1, e1, 0.0, 0.0, 0.0, M1)
    x2, v2 = inputs.elements_to_state(1.0, a2, e2, 0.0, 0.0, 0.0, M2)
    ens = inputs._assemble(1.0, np.array([[m, m]]), np.stack([x1, x2])[None],
                           np.stack([v1, v2])[None], np.array([2]), np.array([dt]), "")
    o = orc.OracleEnsemble(1, 2, gr_mode=0, encounter_hill=K)
    o.init(ens)
    o.step(20000)
    _, _, st, t = o.read_state()
    assert st[0] == 8
    k = int(round(t[0] / dt))
    # prediction with exact Kepler orbits (mu = G m_0, as the drift uses; the
    # interaction and jump are ~1e-12 and cannot move the crossing by a step)
    a01 = 1.0 / (2.0 / np.linalg.norm(x1) - v1 @ v1 / (1.0 + m))
    a02 = 1.0 / (2.0 / np.linalg.norm(x2) - v2 @ v2 / (1.0 + m))
    rh = K * ((2 * m) / 3.0) ** (1.0 / 3.0) * 0.5 * (a01 + a02)
    kexp = None
    margin = []
    for j in range(20000):
        tj = (j + 0.5) * dt
        d = np.linalg.norm(kepler_pos(a1, e1, M1, tj) - kepler_pos(a2, e2, M2, tj))
        margin.append(abs(d / rh - 1))
        if d < rh:
            kexp = j
            break
    assert kexp is not None and min(margin[-3:]) > 1e-6     # not a knife-edge case
    assert k == kexp


def test_stop_rules_off_change_nothing(orc):
    ens = inputs.compact_ensemble(3, 20)
    a = orc.OracleEnsemble(20, 8, gr_mode=1)
    b = orc.OracleEnsemble(20, 8, gr_mode=1, encounter_hill=0.0, eject_factor=0.0)
    a.init(ens)
    b.init(ens)
    a.step(300)
    b.step(300)
    for x, y in zip(a.get_raw(), b.get_raw()):
        assert np.array_equal(x, y)


def test_compact_ensemble_stop_rules_trigger(orc):
    """Closely packed systems run long enough: some stop by close encounter,
    statuses are single stop-rule bits, and stopped systems keep finite state."""
    ens = inputs.compact_ensemble(4, 200)
    o = orc.OracleEnsemble(200, 8, gr_mode=1, encounter_hill=1.0, eject_factor=100.0)
    o.init(ens)
    o.run_threads(50000, 8)
    pos, vel, st, t = o.read_state()
    assert set(np.unique(st)) <= {0, 2, 8, 16}
    assert (st == 8).sum() >= 1
    assert np.all(np.isfinite(pos))
