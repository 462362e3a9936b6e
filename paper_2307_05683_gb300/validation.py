"""Validation sweeps of the Kepler solver on the GPU (the paper's Fig. 1 and
Appendix A experiments, on synthetic test particles).

accuracy_map: massless test particles on (a, e) orbits with random phases,
integrated with the library's production kernel (one single-planet system per
particle, 5-day step, 10 years); returns the relative semi-major axis error
and the status of every particle (Sec. 3.2, Fig. 1).

iteration_search: the same test at Mercury's a for every solver
configuration (Halley iterations, Halley series terms, Newton iterations,
Newton series terms) through the library's whg_kepler_sweep diagnostic
kernel; returns the worst relative a error per configuration (Appendix A).

Units: G = 1, solar masses, AU, time in yr/(2 pi).
"""
from __future__ import annotations

import itertools

import numpy as np

from . import inputs, whg


def semi_major_axis(Q, v, mu=1.0):
    r = np.linalg.norm(Q, axis=-1)
    return 1.0 / (2.0 / r - (v * v).sum(axis=-1) / mu)


def pericentre_timescale(a, e, mu=1.0):
    """T_f = (2 pi / n) (1 - e)^2 / sqrt(1 - e^2) (Eq. 4)."""
    n = np.sqrt(mu / np.asarray(a) ** 3)
    e = np.asarray(e)
    return 2 * np.pi / n * (1 - e) ** 2 / np.sqrt(1 - e * e)


def accuracy_map(a_values, e_values, n_phases=8, years=10.0, dt_days=5.0, seed=0, halley_fp32=False):
    """Relative a error after `years` of massless particles (production kernel;
    halley_fp32=True runs the solver's starting phase in FP32).
    Returns (err [na, ne, n_phases], status [na, ne, n_phases])."""
    a_values = np.asarray(a_values, float)
    e_values = np.asarray(e_values, float)
    rng = np.random.default_rng(seed)
    A, E = np.meshgrid(a_values, e_values, indexing="ij")
    A = np.repeat(A[..., None], n_phases, axis=2)
    E = np.repeat(E[..., None], n_phases, axis=2)
    M = rng.uniform(0, 2 * np.pi, A.shape)
    dt = dt_days * inputs.DAY
    n = int(round(years * 365.25 / dt_days))
    ens = inputs.test_particle(A.ravel(), E.ravel(), M.ravel(), dt=dt)
    it = whg.Integrator(ens.n_systems, 1, gr_mode=0, halley_fp32=halley_fp32)
    it.init(ens)
    it.step(n)
    pos, vel, st, _ = it.read_state()
    it.close()
    Q = pos[:, 1] - pos[:, 0]
    V = vel[:, 1] - vel[:, 0]
    Q0 = ens.pos[:, 1] - ens.pos[:, 0]
    V0 = ens.vel[:, 1] - ens.vel[:, 0]
    err = semi_major_axis(Q, V) / semi_major_axis(Q0, V0) - 1.0
    return err.reshape(A.shape), st.reshape(A.shape)


def iteration_search(configs, e_values, n_phases=8, a=0.387, years=10.0, dt_days=5.0, seed=0):
    """Worst |relative a error| per solver configuration (h_iters, h_terms,
    n_iters, n_terms) over the eccentricities and random phases (whg_kepler_sweep)."""
    import torch
    configs = [tuple(int(x) for x in c) for c in configs]
    rng = np.random.default_rng(seed)
    E = np.repeat(np.asarray(e_values, float), n_phases)
    M = rng.uniform(0, 2 * np.pi, E.size)
    q0, v0 = inputs.elements_to_state(1.0, a, E, 0.0, 0.0, 0.0, M)
    P = E.size
    C = len(configs)
    q = np.tile(q0, (C, 1))
    v = np.tile(v0, (C, 1))
    cfg = np.repeat(np.asarray(configs, np.int32), P, axis=0)
    dev = lambda x, dt=torch.float64: torch.tensor(x, dtype=dt, device="cuda")
    qo = torch.empty((C * P, 3), dtype=torch.float64, device="cuda")
    vo = torch.empty_like(qo)
    steps = int(round(years * 365.25 / dt_days))
    whg.whg_kepler_sweep(dev(q), dev(v), dev(cfg, torch.int32), 1.0, dt_days * inputs.DAY, steps, qo, vo)
    qf, vf = qo.cpu().numpy(), vo.cpu().numpy()
    err = np.abs(semi_major_axis(qf, vf) / semi_major_axis(q, v) - 1.0).reshape(C, P)
    err = np.where(np.isfinite(err), err, np.inf)
    return {c: float(err[i].max()) for i, c in enumerate(configs)}


def default_search_grid():
    """Halley iterations 0..3 (terms 2..8), Newton iterations 0..6 (terms 4..10)."""
    out = []
    for hi, ni, nt in itertools.product(range(4), range(7), range(4, 11)):
        for ht in (range(2, 9) if hi else [4]):
            out.append((hi, ht, ni, nt))
    return out


def solar_copies(n_systems: int, seed: int = 0, dt_days: float = 5.0, perturb_m: float = 1.0):
    """One Solar-System-shaped system (the 8-planet template, angles from
    `seed`) copied n_systems times, Mercury's x moved by +-perturb_m metres in
    each copy (a random sign and size up to perturb_m), dt = dt_days."""
    base = inputs.solar_ensemble(seed, 1)
    rng = np.random.default_rng(seed + 1)
    ens = base.tile(n_systems)
    au_m = 1.495978707e11
    ens.pos[:, 1, 0] += rng.uniform(-1.0, 1.0, n_systems) * perturb_m / au_m
    ens.dt[:] = dt_days * inputs.DAY
    return ens


def energy_error_run(ens, total_steps: int, samples: int = 20, gr_mode: int = 1, **options):
    """Relative energy error |E(t)/E(0) - 1| of every system at `samples`
    evenly spaced times (whg_energy on the synchronized state); `options`
    go to the Integrator (e.g. halley_fp32=True).
    Returns (times [samples], errors [samples, S], status [S])."""
    it = whg.Integrator(ens.n_systems, ens.max_planets, gr_mode=gr_mode, **options)
    it.init(ens)
    E0 = it.energy()
    chunk = max(1, total_steps // samples)
    times, errs = [], []
    done = 0
    for _ in range(samples):
        it.step(chunk)
        done += chunk
        times.append(done * float(ens.dt[0]))
        errs.append(np.abs(it.energy() / E0 - 1.0))
    _, _, st, _ = it.read_state()
    it.close()
    return np.asarray(times), np.asarray(errs), st
