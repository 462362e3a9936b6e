"""Pins for the oracle's forward-mode (tangent) derivatives, which serve as the
reference gradient of the adjoint: central finite differences of the plain
oracle, and the exact invariances of a loss on heliocentric positions
(translating all bodies, or boosting all velocities, changes nothing)."""
import numpy as np
import pytest

from paper_2307_05683_gb300 import inputs


def _loss(orc, m, x, u, n, dt, T, steps, gr):
    o = orc.OracleEnsemble(1, n, gr_mode=gr)
    ens = inputs.Ensemble(m[None], x[None], u[None], np.array([n], np.int32), np.array([dt]))
    o.init(ens)
    o.step(steps)
    pos, _, st, _ = o.read_state()
    assert st[0] == 0
    Q = pos[0, 1:] - pos[0, 0]
    return float(((Q - T) ** 2).sum())


@pytest.mark.parametrize("gr", [0, 1])
def test_tangent_matches_central_differences(orc, gr):
    ens = inputs.two_planet_system(3, 1)
    m, x, u, dt = ens.masses[0], ens.pos[0], ens.vel[0], ens.dt[0]
    rng = np.random.default_rng(0)
    T = x[1:] - x[0] + rng.normal(0, 0.05, (2, 3))
    steps = 300
    L, gx, gu, gm = orc.tangent_gradient(m, x, u, 2, dt, T, steps, gr_mode=gr)
    assert L == pytest.approx(_loss(orc, m, x, u, 2, dt, T, steps, gr), rel=1e-15)
    for name, arr, g in (("x", x, gx), ("u", u, gu)):
        for k in range(3):
            for c in range(3):
                h = 1e-7
                ap, am = arr.copy(), arr.copy()
                ap[k, c] += h
                am[k, c] -= h
                if name == "x":
                    fd = (_loss(orc, m, ap, u, 2, dt, T, steps, gr) - _loss(orc, m, am, u, 2, dt, T, steps, gr)) / (2 * h)
                else:
                    fd = (_loss(orc, m, x, ap, 2, dt, T, steps, gr) - _loss(orc, m, x, am, 2, dt, T, steps, gr)) / (2 * h)
                assert abs(fd - g[k, c]) <= 1e-6 * np.abs(g).max(), (name, k, c, fd, g[k, c])
    for k in range(3):
        # the star (m0 = 1) takes h = 1e-7; planet masses are ~1e-6, where a small
        # relative step drowns in the loss's rounding (below ~1e-3 m the central
        # difference is noise-limited), and they enter almost linearly: 1e-2 m
        h = 1e-7 if k == 0 else 1e-2 * m[k]
        mp, mm = m.copy(), m.copy()
        mp[k] += h
        mm[k] -= h
        fd = (_loss(orc, mp, x, u, 2, dt, T, steps, gr) - _loss(orc, mm, x, u, 2, dt, T, steps, gr)) / (2 * h)
        assert abs(fd - gm[k]) <= 1e-6 * abs(gm[k]) + 1e-9 * np.abs(gx).max(), (k, fd, gm[k])


def test_tangent_invariances(orc):
    ens = inputs.solar_ensemble(4, 1)
    m, x, u, dt = ens.masses[0], ens.pos[0], ens.vel[0], ens.dt[0]
    T = x[1:] - x[0]
    L, gx, gu, gm = orc.tangent_gradient(m, x, u, 8, dt, T, 200, gr_mode=1)
    assert np.abs(gx.sum(0)).max() <= 1e-11 * np.abs(gx).max()
    assert np.abs(gu.sum(0)).max() <= 1e-11 * np.abs(gu).max()
    # the star's mass enters the dynamics; the loss is not blind to it
    assert abs(gm[0]) > 0
