"""CPU checks of the seeded input generators (paper_2307_05683_gb300/inputs.py).

The generators feed both the CUDA path and the oracle, so a mistake in them
would go unnoticed by parity tests. Each check here is fixed by two-body
mechanics or by the recipe a generator states, not by the generator's code:
vis-viva energy, angular momentum, Kepler's equation, the barycentric frame,
mutual-Hill-radius spacing and the stated parameter ranges.
"""
import numpy as np
import pytest

from paper_2307_05683_gb300 import inputs


def _elements(seed, n=400):
    rng = np.random.default_rng(seed)
    mu = 10.0 ** rng.uniform(-1, 1, n)
    a = 10.0 ** rng.uniform(-1, 1.5, n)
    e = rng.uniform(0.0, 0.95, n)
    inc = rng.uniform(0.01, np.pi - 0.01, n)
    Om, om, M = rng.uniform(0, 2 * np.pi, (3, n))
    return mu, a, e, inc, Om, om, M


def test_elements_to_state_two_body_invariants():
    """Energy -mu/(2a), |h| = sqrt(mu a (1-e^2)), inclination, node and |e| vector."""
    mu, a, e, inc, Om, om, M = _elements(1)
    x, v = inputs.elements_to_state(mu, a, e, inc, Om, om, M)
    r = np.linalg.norm(x, axis=1)
    energy = 0.5 * (v * v).sum(1) - mu / r
    np.testing.assert_allclose(energy, -mu / (2 * a), rtol=1e-11)
    h = np.cross(x, v)
    hn = np.linalg.norm(h, axis=1)
    np.testing.assert_allclose(hn, np.sqrt(mu * a * (1 - e * e)), rtol=1e-11)
    np.testing.assert_allclose(np.arccos(h[:, 2] / hn), inc, atol=1e-10)
    # ascending node direction z x h points at angle Omega in the reference plane
    np.testing.assert_allclose(np.cos(np.arctan2(h[:, 0], -h[:, 1]) - Om), 1.0, atol=1e-10)
    evec = np.cross(v, h) / mu[:, None] - x / r[:, None]
    np.testing.assert_allclose(np.linalg.norm(evec, axis=1), e, atol=1e-10)


def test_elements_to_state_mean_anomaly():
    """The eccentric anomaly recovered from r and x.v satisfies Kepler's equation
    E - e sin E = M (mod 2 pi)."""
    mu, a, e, inc, Om, om, M = _elements(2)
    x, v = inputs.elements_to_state(mu, a, e, inc, Om, om, M)
    r = np.linalg.norm(x, axis=1)
    ecosE = 1.0 - r / a
    esinE = (x * v).sum(1) / np.sqrt(mu * a)
    E = np.arctan2(esinE, ecosE)
    Mrec = E - esinE
    np.testing.assert_allclose(np.cos(Mrec - M), 1.0, atol=1e-10)


def test_elements_to_state_circular_special_case():
    """e = i = Omega = omega = 0: a point on a circle moving at sqrt(mu/a)."""
    phi = np.linspace(0, 2 * np.pi, 7)
    x, v = inputs.elements_to_state(2.0, 3.0, 0.0, 0.0, 0.0, 0.0, phi)
    np.testing.assert_allclose(x, np.stack([3 * np.cos(phi), 3 * np.sin(phi), 0 * phi], 1), atol=1e-14)
    vc = np.sqrt(2.0 / 3.0)
    np.testing.assert_allclose(v, np.stack([-vc * np.sin(phi), vc * np.cos(phi), 0 * phi], 1), atol=1e-14)


@pytest.mark.parametrize("make", [
    lambda: inputs.two_planet_system(3, 50),
    lambda: inputs.solar_ensemble(4, 50),
    lambda: inputs.compact_ensemble(5, 200),
])
def test_barycentric_frame_and_padding(make):
    """Total momentum and mass-weighted position vanish; unused slots are zero;
    the heliocentric planet orbits are bound with the recipe's semi-major axes
    positive; dt > 0."""
    ens = make()
    m = ens.masses
    np.testing.assert_allclose((m[..., None] * ens.pos).sum(1), 0.0, atol=1e-15)
    np.testing.assert_allclose((m[..., None] * ens.vel).sum(1), 0.0, atol=1e-18)
    slot = np.arange(ens.max_planets)[None, :] < ens.n_planets[:, None]
    assert np.all(m[:, 0] == 1.0)
    assert np.all(m[:, 1:][~slot] == 0) and np.all(m[:, 1:][slot] > 0)
    assert np.all(ens.pos[:, 1:][~slot] == 0) and np.all(ens.vel[:, 1:][~slot] == 0)
    assert np.all(ens.dt > 0) and ens.dt.dtype == np.float64
    assert ens.n_planets.dtype == np.int32
    xh = ens.pos[:, 1:] - ens.pos[:, :1]
    vh = ens.vel[:, 1:] - ens.vel[:, :1]
    mu = m[:, :1] + m[:, 1:]
    eps = 0.5 * (vh * vh).sum(-1) - mu / np.maximum(np.linalg.norm(xh, axis=-1), 1e-300)
    assert np.all(eps[slot] < 0)


def test_solar_ensemble_recipe():
    """Masses and semi-major axes within 6 sigma of the template (sigma 1e-3
    relative); dt = P_Mercury / 20 from the perturbed a and mass."""
    ens = inputs.solar_ensemble(6, 300)
    mp = ens.masses[:, 1:]
    assert np.all(np.abs(mp / inputs.SOLAR_MASSES - 1) < 6e-3)
    xh = ens.pos[:, 1:] - ens.pos[:, :1]
    vh = ens.vel[:, 1:] - ens.vel[:, :1]
    mu = 1.0 + mp
    a = 1.0 / (2.0 / np.linalg.norm(xh, axis=-1) - (vh * vh).sum(-1) / mu)
    assert np.all(np.abs(a / inputs.SOLAR_A - 1) < 6e-3)
    P = 2 * np.pi * np.sqrt(a[:, 0] ** 3 / mu[:, 0])
    np.testing.assert_allclose(ens.dt, P / 20.0, rtol=1e-10)
    # Mercury's period is about 88 days
    assert np.all(np.abs(ens.dt * 20 / inputs.DAY - 87.97) < 1.0)


def test_compact_ensemble_hill_spacing():
    """Planet counts span 2..8; consecutive live planets sit 8..12 mutual Hill
    radii apart, R_H = ((m_k + m_k+1)/3)^(1/3) (a_k + a_k+1)/2; a_1 = 0.1."""
    ens = inputs.compact_ensemble(7, 2000)
    assert set(np.unique(ens.n_planets)) == set(range(2, 9))
    xh = ens.pos[:, 1:] - ens.pos[:, :1]
    vh = ens.vel[:, 1:] - ens.vel[:, :1]
    mp = ens.masses[:, 1:]
    slot = np.arange(8)[None, :] < ens.n_planets[:, None]
    with np.errstate(divide="ignore", invalid="ignore"):
        a = 1.0 / (2.0 / np.linalg.norm(xh, axis=-1) - (vh * vh).sum(-1) / (1.0 + mp))
        rh = ((mp[:, :-1] + mp[:, 1:]) / 3.0) ** (1.0 / 3.0) * (a[:, :-1] + a[:, 1:]) / 2
        delta = ((a[:, 1:] - a[:, :-1]) / rh)[slot[:, 1:]]
    np.testing.assert_allclose(a[:, 0], 0.1, rtol=1e-10)
    assert np.all((mp[slot] > 1e-7 * (1 - 1e-12)) & (mp[slot] < 1e-4))
    assert delta.min() >= 8.0 - 1e-6 and delta.max() <= 12.0 + 1e-6
    np.testing.assert_allclose(ens.dt, 2 * np.pi * 0.1 ** 1.5 / 20.0, rtol=1e-15)


def test_seeded_and_subset_tile():
    """Same seed, same bits; another seed differs; subset/tile copy rows."""
    a, b = inputs.compact_ensemble(11, 64), inputs.compact_ensemble(11, 64)
    for f in ("masses", "pos", "vel", "n_planets", "dt"):
        assert np.array_equal(getattr(a, f), getattr(b, f))
    assert not np.array_equal(a.pos, inputs.compact_ensemble(12, 64).pos)
    t = a.tile(150)
    assert t.n_systems == 150 and np.array_equal(t.pos[64:128], a.pos)
    s = a.subset([5, 2])
    assert np.array_equal(s.vel[1], a.vel[2]) and s.n_planets[0] == a.n_planets[5]


def test_test_particle_drift_problem():
    """One massless planet per system: the star stays at the origin at rest and
    the planet's orbit has the requested a and e."""
    ens = inputs.test_particle([1.0, 2.5], [0.1, 0.9], [0.3, 2.0], m0=1.0)
    assert ens.masses[:, 1].tolist() == [0.0, 0.0]
    assert np.all(ens.pos[:, 0] == 0) and np.all(ens.vel[:, 0] == 0)
    x, v = ens.pos[:, 1], ens.vel[:, 1]
    r = np.linalg.norm(x, axis=1)
    a = 1.0 / (2.0 / r - (v * v).sum(1))
    np.testing.assert_allclose(a, [1.0, 2.5], rtol=1e-12)
    h = np.linalg.norm(np.cross(x, v), axis=1)
    np.testing.assert_allclose(np.sqrt(1 - h * h / a), [0.1, 0.9], rtol=1e-10)
