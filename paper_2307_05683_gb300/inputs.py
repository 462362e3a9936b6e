"""Seeded synthetic planetary ensembles (initial conditions only).

This module produces inertial-frame masses, positions and velocities for
ensembles of independent star + planet systems, plus a per-system timestep.
It holds none of the integrator's arithmetic: it places bodies on two-body
orbits from orbital elements and moves each system to its barycentric frame.
Both the CUDA path and the CPU oracle are fed from here.

Units: G = 1, masses in solar masses, lengths in AU, time in units of
yr/(2 pi) (one day = K_GAUSS code units).

Layout of an Ensemble (S systems, Nmax planets, body 0 is the star):
    masses  [S, 1+Nmax]     float64
    pos     [S, 1+Nmax, 3]  float64, inertial (barycentric) frame
    vel     [S, 1+Nmax, 3]  float64
    n_planets [S]           int32   (slots >= n_planets are zero-filled)
    dt      [S]             float64 (> 0)
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

K_GAUSS = 0.01720209895           # code time units per day (Gaussian constant)
DAY = K_GAUSS
YEAR = 365.25 * K_GAUSS
C_LIGHT_AU_PER_DAY = 173.1446326742403
C_LIGHT = C_LIGHT_AU_PER_DAY / K_GAUSS  # speed of light in code units (~10065.32)

# Eight-planet template, Mercury .. Neptune: standard public planetary masses
# (solar masses), semi-major axes (AU), eccentricities and inclinations (deg).
SOLAR_MASSES = np.array([1.660e-7, 2.448e-6, 3.040e-6, 3.227e-7,
                         9.548e-4, 2.859e-4, 4.366e-5, 5.151e-5])
SOLAR_A = np.array([0.3871, 0.7233, 1.0000, 1.5237, 5.2026, 9.5549, 19.218, 30.110])
SOLAR_E = np.array([0.2056, 0.0068, 0.0167, 0.0934, 0.0489, 0.0565, 0.0457, 0.0113])
SOLAR_I_DEG = np.array([7.00, 3.39, 0.00, 1.85, 1.30, 2.49, 0.77, 1.77])


@dataclass
class Ensemble:
    masses: np.ndarray
    pos: np.ndarray
    vel: np.ndarray
    n_planets: np.ndarray
    dt: np.ndarray
    recipe: str = ""

    @property
    def n_systems(self) -> int:
        return int(self.masses.shape[0])

    @property
    def max_planets(self) -> int:
        return int(self.masses.shape[1] - 1)

    def subset(self, idx) -> "Ensemble":
        idx = np.asarray(idx)
        return Ensemble(self.masses[idx].copy(), self.pos[idx].copy(), self.vel[idx].copy(),
                        self.n_planets[idx].copy(), self.dt[idx].copy(), self.recipe)

    def tile(self, n_systems: int) -> "Ensemble":
        """Repeat systems cyclically up to n_systems (used for large sweeps)."""
        idx = np.arange(n_systems) % self.n_systems
        return self.subset(idx)


def _solve_eccentric_anomaly(M: np.ndarray, e: np.ndarray) -> np.ndarray:
    """E - e sin E = M for elliptic orbits (Newton, fixed 60 iterations)."""
    E = np.where(e < 0.8, M, np.pi * np.ones_like(M))
    for _ in range(60):
        E = E - (E - e * np.sin(E) - M) / (1.0 - e * np.cos(E))
    return E


def elements_to_state(mu, a, e, inc, Omega, omega, M):
    """Heliocentric position/velocity from elliptic orbital elements (arrays)."""
    mu, a, e, inc, Omega, omega, M = np.broadcast_arrays(
        *[np.asarray(v, dtype=np.float64) for v in (mu, a, e, inc, Omega, omega, M)])
    E = _solve_eccentric_anomaly(np.mod(M, 2 * np.pi), e)
    cE, sE = np.cos(E), np.sin(E)
    b = a * np.sqrt(1.0 - e * e)
    xp = a * (cE - e)
    yp = b * sE
    n = np.sqrt(mu / a ** 3)
    r = a * (1.0 - e * cE)
    vxp = -a * n * sE * a / r
    vyp = b * n * cE * a / r
    cO, sO = np.cos(Omega), np.sin(Omega)
    co, so = np.cos(omega), np.sin(omega)
    ci, si = np.cos(inc), np.sin(inc)
    # rotation R = Rz(Omega) Rx(inc) Rz(omega) applied to the in-plane vector
    r11 = cO * co - sO * so * ci
    r12 = -cO * so - sO * co * ci
    r21 = sO * co + cO * so * ci
    r22 = -sO * so + cO * co * ci
    r31 = so * si
    r32 = co * si
    x = np.stack([r11 * xp + r12 * yp, r21 * xp + r22 * yp, r31 * xp + r32 * yp], axis=-1)
    v = np.stack([r11 * vxp + r12 * vyp, r21 * vxp + r22 * vyp, r31 * vxp + r32 * vyp], axis=-1)
    return x, v


def _assemble(m0, mp, xh, vh, n_planets, dt, recipe) -> Ensemble:
    """Star at the heliocentric origin, then shift every system to its barycentre."""
    S, N = mp.shape
    masses = np.zeros((S, 1 + N))
    masses[:, 0] = m0
    masses[:, 1:] = mp
    pos = np.zeros((S, 1 + N, 3))
    vel = np.zeros((S, 1 + N, 3))
    pos[:, 1:] = xh
    vel[:, 1:] = vh
    slot = np.arange(N)[None, :] < n_planets[:, None]
    masses[:, 1:] *= slot
    pos[:, 1:] *= slot[..., None]
    vel[:, 1:] *= slot[..., None]
    mt = masses.sum(axis=1)
    xc = (masses[..., None] * pos).sum(axis=1) / mt[:, None]
    vc = (masses[..., None] * vel).sum(axis=1) / mt[:, None]
    live = np.concatenate([np.ones((S, 1), bool), slot], axis=1)
    pos = (pos - xc[:, None, :]) * live[..., None]
    vel = (vel - vc[:, None, :]) * live[..., None]
    return Ensemble(masses, pos, vel, n_planets.astype(np.int32), np.asarray(dt, np.float64), recipe)


def two_planet_system(seed: int, n_systems: int = 1) -> Ensemble:
    """Star of mass 1 + 2 planets: masses log-uniform 1e-6..1e-3, a = 1.0 and 1.6,
    e ~ Rayleigh(0.02), i ~ Rayleigh(0.01 rad), angles uniform; dt = P_inner/30."""
    rng = np.random.default_rng(seed)
    S, N = n_systems, 2
    mp = 10.0 ** rng.uniform(-6, -3, size=(S, N))
    a = np.broadcast_to(np.array([1.0, 1.6]), (S, N))
    e = rng.rayleigh(0.02, size=(S, N))
    inc = rng.rayleigh(0.01, size=(S, N))
    ang = rng.uniform(0, 2 * np.pi, size=(3, S, N))
    xh, vh = elements_to_state(1.0 + mp, a, e, inc, ang[0], ang[1], ang[2])
    P_in = 2 * np.pi * np.sqrt(a[:, 0] ** 3 / (1.0 + mp[:, 0]))
    return _assemble(1.0, mp, xh, vh, np.full(S, N), P_in / 30.0,
                     f"two_planet seed={seed} S={S}")


def solar_ensemble(seed: int, n_systems: int, dt_per_inner_period: float = 20.0) -> Ensemble:
    """Solar-System-shaped ensemble: the 8-planet template with masses and a
    scaled by (1 + N(0, 1e-3)), e and i = |template +- Rayleigh(1e-3)|,
    angles uniform; dt = P_Mercury / 20 per system."""
    rng = np.random.default_rng(seed)
    S, N = n_systems, 8
    mp = SOLAR_MASSES[None, :] * (1.0 + rng.normal(0.0, 1e-3, size=(S, N)))
    a = SOLAR_A[None, :] * (1.0 + rng.normal(0.0, 1e-3, size=(S, N)))
    sgn = rng.choice([-1.0, 1.0], size=(2, S, N))
    e = np.abs(SOLAR_E[None, :] + sgn[0] * rng.rayleigh(1e-3, size=(S, N)))
    inc = np.abs(np.deg2rad(SOLAR_I_DEG)[None, :] + sgn[1] * rng.rayleigh(1e-3, size=(S, N)))
    ang = rng.uniform(0, 2 * np.pi, size=(3, S, N))
    xh, vh = elements_to_state(1.0 + mp, a, e, inc, ang[0], ang[1], ang[2])
    P_in = 2 * np.pi * np.sqrt(a[:, 0] ** 3 / (1.0 + mp[:, 0]))
    return _assemble(1.0, mp, xh, vh, np.full(S, N), P_in / dt_per_inner_period,
                     f"solar_ensemble seed={seed} S={S} dt=P_in/{dt_per_inner_period:g}")


def compact_ensemble(seed: int, n_systems: int) -> Ensemble:
    """Compact systems: planet count uniform in 2..8, masses log-uniform
    1e-7..1e-4, a_1 = 0.1 and consecutive spacings of 8..12 mutual Hill radii,
    e ~ Rayleigh(0.01), i ~ Rayleigh(0.005); dt = P(0.1)/20."""
    rng = np.random.default_rng(seed)
    S, N = n_systems, 8
    npl = rng.integers(2, 9, size=S)
    mp = 10.0 ** rng.uniform(-7, -4, size=(S, N))
    a = np.zeros((S, N))
    a[:, 0] = 0.1
    delta = rng.uniform(8.0, 12.0, size=(S, N))
    for k in range(N - 1):
        hk = ((mp[:, k] + mp[:, k + 1]) / 3.0) ** (1.0 / 3.0)
        a[:, k + 1] = a[:, k] * (1 + delta[:, k] * hk / 2) / (1 - delta[:, k] * hk / 2)
    e = rng.rayleigh(0.01, size=(S, N))
    inc = rng.rayleigh(0.005, size=(S, N))
    ang = rng.uniform(0, 2 * np.pi, size=(3, S, N))
    xh, vh = elements_to_state(1.0 + mp, a, e, inc, ang[0], ang[1], ang[2])
    dt = np.full(S, 2 * np.pi * np.sqrt(0.1 ** 3) / 20.0)
    return _assemble(1.0, mp, xh, vh, npl, dt, f"compact seed={seed} S={S}")


def test_particle(a, e, phase, inc=0.0, Omega=0.0, omega=0.0, m0=1.0, dt=5 * DAY) -> Ensemble:
    """One massless planet per system on an (a, e) orbit with mean anomaly
    `phase` around a star of mass m0 (the drift-only problem)."""
    a, e, phase = np.broadcast_arrays(np.atleast_1d(np.asarray(a, float)),
                                      np.atleast_1d(np.asarray(e, float)),
                                      np.atleast_1d(np.asarray(phase, float)))
    S = a.shape[0]
    xh, vh = elements_to_state(m0, a, e, inc, Omega, omega, phase)
    return _assemble(m0, np.zeros((S, 1)), xh[:, None, :], vh[:, None, :],
                     np.ones(S, np.int32), np.full(S, dt), "test_particle")
