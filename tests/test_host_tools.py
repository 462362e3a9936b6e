"""CPU checks of the host-side logic of the autotuner and the validation tools
(no GPU: timing is replaced by a stub, no kernel is launched)."""
import json

import numpy as np

from paper_2307_05683_gb300 import autotune, inputs, validation


def test_candidates_uniform_and_mixed():
    """A uniform 8-planet ensemble tries only per-count packing; a mixed one
    also the 8-lane layout. Queue launches only with one-warp blocks."""
    solar = list(autotune.candidates(inputs.solar_ensemble(0, 4)))
    mixed = list(autotune.candidates(inputs.compact_ensemble(0, 64)))
    assert {c["lanes_per_system"] for c in solar} == {0}
    assert {c["lanes_per_system"] for c in mixed} == {0, 8}
    for cands in (solar, mixed):
        assert all(c["block_size"] == 32 for c in cands if c["queue_steps"])
        keys = [tuple(sorted(c.items())) for c in cands]
        assert len(keys) == len(set(keys))
    # 3 blocks x 2 launch lengths x 2 graph settings x 2 schedules without the
    # queue, plus 1 block x 2 x 2 x 2 with it, per packing
    assert len(solar) == 24 + 8 and len(mixed) == 2 * (24 + 8)
    three = inputs.compact_ensemble(1, 64).subset(np.arange(64))
    three.masses = three.masses[:, :4]
    three.pos, three.vel = three.pos[:, :4], three.vel[:, :4]
    three.n_planets = np.minimum(three.n_planets, 3)
    assert {c["lanes_per_system"] for c in autotune.candidates(three)} == {0, 4}


def test_cache_key_separates_shapes():
    a = inputs.compact_ensemble(2, 64)
    b = inputs.compact_ensemble(3, 64)
    k = autotune._key(a, 1, 8, "GPU")
    assert k == autotune._key(a, 1, 8, "GPU")
    assert k != autotune._key(a, 0, 8, "GPU") and k != autotune._key(a, 1, 6, "GPU")
    assert k != autotune._key(a, 1, 8, "other")
    assert (k == autotune._key(b, 1, 8, "GPU")) == np.array_equal(
        np.bincount(a.n_planets, minlength=9), np.bincount(b.n_planets, minlength=9))


def test_tune_picks_fastest_and_caches(tmp_path, monkeypatch):
    """tune() keeps the candidate with the highest measured rate, writes it to
    the cache, and answers from the cache without timing on the next call."""
    import torch
    monkeypatch.setattr(torch.cuda, "get_device_name", lambda *a: "stub")
    calls = []

    def fake_time(ens, cfg, gr_mode, newton_terms, window_s=0.05):
        calls.append(cfg)
        return 1.0 + cfg["block_size"] + 1000 * cfg["queue_steps"] + cfg["interaction_schedule"]

    monkeypatch.setattr(autotune, "time_config", fake_time)
    ens = inputs.solar_ensemble(0, 8)
    path = str(tmp_path / "sub" / "tune.json")
    best = autotune.tune(ens, cache_path=path)
    n = len(list(autotune.candidates(ens)))
    assert len(calls) == n and best["tried"] == n
    assert best["queue_steps"] == 100 and best["block_size"] == 32 and best["interaction_schedule"] == 1
    assert best["system_steps_per_s"] == 1.0 + 32 + 100000 + 1
    stored = json.load(open(path))
    assert list(stored.values())[0]["queue_steps"] == 100
    calls.clear()
    again = autotune.tune(ens, cache_path=path)
    assert calls == [] and again == best
    autotune.tune(ens, cache_path=path, force=True)
    assert len(calls) == n
    # a corrupt cache file is ignored and rewritten
    open(path, "w").write("{not json")
    calls.clear()
    autotune.tune(ens, cache_path=path)
    assert len(calls) == n and json.load(open(path))


def test_launch_space_is_results_neutral_and_skips_long_graph_timings(tmp_path, monkeypatch):
    """space="launch" (the size sweep's tuning) tries only block size, work
    queue and graph replay of short launches -- dimensions that leave results
    bit for bit unchanged -- and skips the graph candidate once two replays
    would take more than 20 timing windows (large ensembles)."""
    import torch
    monkeypatch.setattr(torch.cuda, "get_device_name", lambda *a: "stub")
    cands = list(autotune.candidates(inputs.solar_ensemble(0, 8), "launch"))
    assert all(set(c) == {"block_size", "queue_steps", "steps_per_launch", "graph_launches"} for c in cands)
    assert any(c["graph_launches"] for c in cands) and all(c["block_size"] == 32 for c in cands
                                                          if c["queue_steps"])
    timed = []
    monkeypatch.setattr(autotune, "time_config",
                        lambda ens, cfg, g, nt, window_s=0.05: timed.append(cfg) or 1.0 + cfg["graph_launches"])
    base = inputs.solar_ensemble(0, 16)
    small = autotune.tune(base.tile(1 << 14), cache_path=None, space="launch")
    assert small["graph_launches"] == 16 and small["tried"] == len(cands)
    timed.clear()
    large = autotune.tune(base.tile(1 << 18), cache_path=None, space="launch")
    assert large["tried"] == len(cands) - 1 and not any(c["graph_launches"] for c in timed)
    # a queue candidate is timed over at least 4 units, where launches use the queue
    queued = [c for c in cands if c["queue_steps"]][0]
    assert autotune.min_steps(base.tile(1 << 18), queued, 0.05) >= 4 * queued["queue_steps"]


def test_pericentre_timescale_eq4():
    """e = 0 gives the orbital period; the factor (1-e)^2/sqrt(1-e^2) shrinks
    it toward high eccentricity (Eq. 4)."""
    np.testing.assert_allclose(validation.pericentre_timescale(1.0, 0.0), 2 * np.pi, rtol=1e-15)
    np.testing.assert_allclose(validation.pericentre_timescale(4.0, 0.0, mu=2.0),
                               2 * np.pi * np.sqrt(64 / 2.0), rtol=1e-15)
    e = np.array([0.5, 0.9])
    np.testing.assert_allclose(validation.pericentre_timescale(1.0, e),
                               2 * np.pi * np.array([0.25 / np.sqrt(0.75), 0.01 / np.sqrt(0.19)]), rtol=1e-14)


def test_semi_major_axis_vis_viva():
    q, v = inputs.elements_to_state(1.5, np.array([0.4, 2.0]), np.array([0.1, 0.6]), 0.2, 0.3, 0.4,
                                    np.array([1.0, 4.0]))
    np.testing.assert_allclose(validation.semi_major_axis(q, v, mu=1.5), [0.4, 2.0], rtol=1e-12)


def test_default_search_grid():
    """Halley 0..3 iterations (2..8 terms; one entry with 0 iterations),
    Newton 0..6 iterations with 4..10 terms; the paper's (2, 4, 2, 8) is in it."""
    grid = validation.default_search_grid()
    assert len(grid) == len(set(grid)) == (1 + 3 * 7) * 7 * 7
    assert (2, 4, 2, 8) in grid and (2, 4, 2, 6) in grid
    assert all(0 <= h <= 3 and 2 <= ht <= 8 and 0 <= n <= 6 and 4 <= nt <= 10 for h, ht, n, nt in grid)


def test_solar_copies_perturbation():
    """Copies differ from the template only in Mercury's x, by at most
    perturb_m metres, and step with the requested dt."""
    base = inputs.solar_ensemble(5, 1)
    ens = validation.solar_copies(100, seed=5, dt_days=4.0, perturb_m=2.0)
    assert ens.n_systems == 100
    dx = (ens.pos - base.pos)
    dx[:, 1, 0] = 0.0
    assert np.all(dx == 0) and np.all(ens.vel == base.vel) and np.all(ens.masses == base.masses)
    shift_m = (ens.pos[:, 1, 0] - base.pos[0, 1, 0]) * 1.495978707e11
    assert np.all(np.abs(shift_m) <= 2.0 * (1 + 1e-6)) and np.std(shift_m) > 0.5
    np.testing.assert_array_equal(ens.dt, 4.0 * inputs.DAY)



def test_integrator_refuses_misshaped_host_arrays():
    """Integrator.init and set_raw check every host array's shape against the
    context's S and N before any library call (no GPU needed to reach the check)."""
    import pytest
    from paper_2307_05683_gb300 import whg
    it = object.__new__(whg.Integrator)
    it.S, it.N, it.ctx = 4, 2, None
    good = inputs.two_planet_system(0, 4)
    for bad in (inputs.two_planet_system(0, 3), inputs.solar_ensemble(0, 4)):
        with pytest.raises(ValueError):
            it.init(bad)
    short = inputs.two_planet_system(0, 4)
    short.dt = short.dt[:3]
    with pytest.raises(ValueError, match="dt"):
        it.init(short)
    Q = np.zeros((4, 2, 3))
    with pytest.raises(ValueError, match="v"):
        it.set_raw(Q, np.zeros((4, 3, 3)), np.zeros(4, np.int64), np.zeros(4, np.int32))
    with pytest.raises(ValueError, match="status"):
        it.set_raw(Q, Q, np.zeros(4, np.int64), np.zeros(5, np.int32))
    it._check_shapes((("masses", good.masses, (4, 3)), ("pos", good.pos, (4, 3, 3))))
    with pytest.raises(ValueError):
        whg.whg_get_raw(None, Q, Q, np.zeros(4, np.int32), np.zeros(4, np.int32))
