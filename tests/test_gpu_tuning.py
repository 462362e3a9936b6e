"""CUDA-graph replay of step launches and the autotuner."""
import json
import os

import numpy as np
import pytest

from paper_2307_05683_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def whg():
    from paper_2307_05683_gb300 import build, whg as w
    build.build()
    w.load()
    return w


def _run(whg, ens, n, **kw):
    it = whg.Integrator(ens.n_systems, ens.max_planets, **kw)
    it.init(ens)
    it.step(n)
    out = it.read_state() + it.get_raw() + (it.launches,)
    it.close()
    return out


def test_graph_replay_is_bitwise_identical(whg):
    ens = inputs.compact_ensemble(41, 300)
    direct = _run(whg, ens, 1000, steps_per_launch=10)
    graph = _run(whg, ens, 1000, steps_per_launch=10, graph_launches=8)
    for a, b in zip(direct[:-1], graph[:-1]):
        assert np.array_equal(a, b)
    assert direct[-1] == graph[-1]                   # 2 + 100 step launches either way


def test_graph_is_captured_again_after_init(whg):
    a = inputs.solar_ensemble(42, 64)
    b = inputs.solar_ensemble(43, 64)
    it = whg.Integrator(64, 8, steps_per_launch=5, graph_launches=4)
    it.init(a)
    it.step(100)
    it.init(b)                                       # new state, same context
    it.step(100)
    got = it.read_state()
    it.close()
    ref = _run(whg, b, 100)
    for x, y in zip(got, ref[:4]):
        assert np.array_equal(x, y)


def test_autotuner_picks_a_valid_configuration_and_caches_it(whg, tmp_path):
    from paper_2307_05683_gb300 import autotune
    ens = inputs.compact_ensemble(44, 2048)
    cache = str(tmp_path / "tune.json")
    best = autotune.tune(ens, cache_path=cache, window_s=0.01)
    assert best["lanes_per_system"] in (0, 8) and best["block_size"] in (32, 64, 128)
    assert best["system_steps_per_s"] > 0 and best["tried"] == len(list(autotune.candidates(ens)))
    assert os.path.exists(cache) and len(json.load(open(cache))) == 1
    again = autotune.tune(ens, cache_path=cache, window_s=0.01)
    assert again == best
    # the tuned configuration integrates the same map (packing only reorders sums)
    it = autotune.integrator(ens, cache_path=cache)
    it.init(ens)
    it.step(200)
    p, v, st, t = it.read_state()
    it.close()
    ref = _run(whg, ens, 200)
    sx = np.abs(ref[0]).max(axis=(1, 2))[:, None, None]
    assert np.array_equal(st, ref[2])
    assert (np.abs(p - ref[0]) / sx).max() <= 1e-12


def test_fp64_masked_lanes_cost_full_pipe_time():
    """The lane layout fills all 32 lanes of a warp with planets (floor(32/L)
    systems per warp) rather than spreading a small ensemble over more,
    partly filled warps: on this GPU an FP64 warp instruction takes the same
    pipe time whatever the number of active lanes."""
    from paper_2307_05683_gb300 import build, whg
    build.build()
    t32 = whg.whg_probe_fp64_lanes(4, 32, 4000)
    t8 = whg.whg_probe_fp64_lanes(4, 8, 4000)
    assert t32 > 0 and t8 >= 0.9 * t32, (t8, t32)


def test_fp64_issue_rate_is_the_same_for_every_instruction_kind():
    """A stream of DFMA, DMUL or DADD, alone or interleaved with integer or
    FP32 work, issues at the same number of FP64 lane-operations per SM clock
    (about 1.68 on GB300, under the nominal 2): no kind of FP64 instruction
    is cheaper, so the step kernel's cost is its FP64 instruction count."""
    from paper_2307_05683_gb300 import build, whg
    build.build()
    rates = [whg.whg_probe_fp64_kind(k, 8, 4000) for k in range(5)]
    assert all(1.0 < r <= 2.05 for r in rates), rates
    assert max(rates) <= 1.05 * min(rates), rates


@pytest.mark.parametrize("graphs,lanes", [(0, 0), (4, 0), (0, 8)])
def test_repacking_stopped_systems_is_bitwise_neutral(whg, graphs, lanes):
    """repack_frozen regroups running systems ahead of stopped ones inside
    each planet-count bucket (or the one lane group, lanes_per_system = 8);
    every output (state, status, step counts, energy, raw state) stays bit
    for bit the same, with and without graph replay.  A tight close-encounter
    rule stops many systems on the way."""
    ens = inputs.compact_ensemble(45, 700)
    kw = dict(close_encounter_hill=8.0, eject_factor=3.0, steps_per_launch=25, graph_launches=graphs,
              lanes_per_system=lanes)
    plain = _run(whg, ens, 1500, repack_frozen=False, **kw)
    auto = _run(whg, ens, 1500, **kw)                 # default: on, since a stop rule is on
    it = whg.Integrator(ens.n_systems, 8, repack_frozen=True, **kw)
    it.init(ens)
    for n in (700, 800):                              # two calls: the repack state carries over
        it.step(n)
    rep = it.read_state() + it.get_raw() + (it.launches,)
    E = it.energy()
    it.close()
    st = plain[2]
    assert 50 < int((st != 0).sum()) < ens.n_systems - 50      # both kinds present
    for a, b in zip(plain[:-1], rep[:-1]):
        assert np.array_equal(a, b)
    ref = whg.Integrator(ens.n_systems, 8, **kw)
    ref.init(ens)
    ref.step(1500)
    assert np.array_equal(ref.energy(), E, equal_nan=True)
    ref.close()
    assert rep[-1] > plain[-1]                        # the repack kernels are counted
    assert auto[-1] == rep[-1]
    for a, b in zip(auto[:-1], rep[:-1]):
        assert np.array_equal(a, b)
    # without a stop rule the default does not repack: the same launches as off
    assert _run(whg, ens, 600, steps_per_launch=25)[-1] == _run(whg, ens, 600, steps_per_launch=25,
                                                                 repack_frozen=False)[-1]


@pytest.mark.parametrize("extra", [{}, {"graph_launches": 4, "steps_per_launch": 250},
                                   {"repack_frozen": True, "steps_per_launch": 250}])
def test_work_queue_is_bitwise_identical(whg, extra):
    """queue_steps moves warp-groups between SMs in units of steps; each
    system's arithmetic is unchanged, so every output matches the default
    path bit for bit (mixed planet counts, stop rules, graphs, repacking)."""
    ens = inputs.compact_ensemble(46, 900)
    kw = dict(close_encounter_hill=8.0, eject_factor=3.0, **extra)
    plain = _run(whg, ens, 1500, queue_steps=0, **kw)
    queued = _run(whg, ens, 1500, queue_steps=37, **kw)
    assert int((plain[2] != 0).sum()) > 50
    for a, b in zip(plain[:-1], queued[:-1]):
        assert np.array_equal(a, b)


def test_work_queue_bench_size_is_bitwise_identical(whg):
    """4096 Solar-System-shaped systems (1024 warp-groups over 152 SMs),
    3000 steps in 100-step units against one plain launch."""
    ens = inputs.solar_ensemble(47, 4096)
    plain = _run(whg, ens, 3000, queue_steps=0)
    queued = _run(whg, ens, 3000, queue_steps=100)
    for a, b in zip(plain[:-1], queued[:-1]):
        assert np.array_equal(a, b)
    small = inputs.solar_ensemble(48, 64)
    it = whg.Integrator(64, 8, queue_steps=10)
    it.init(small)
    it.step(0)
    it.step(5)                                       # below 4 units: a plain launch
    it.step(45)                                      # 5 units, the last one partial
    it.synchronize()
    got = it.read_state()
    it.close()
    ref = _run(whg, small, 50, queue_steps=0)
    for a, b in zip(got, ref[:4]):
        assert np.array_equal(a, b)


def test_work_queue_wait_gives_up_and_context_stays_usable(whg):
    """Failure path of the work queue without a fault: every unit waits for
    a predecessor that never runs; each wait gives up after a few thousand
    polls, sets the error flag that the host reads, and leaves the state and
    the context usable (the next steps equal those of a fresh context)."""
    ens = inputs.solar_ensemble(49, 256)
    it = whg.Integrator(256, 8, queue_steps=50)
    it.init(ens)
    assert whg.whg_test_queue_timeout(it.ctx, 1 << 12) == 1
    it.synchronize()                                 # the flag was reported and cleared
    it.step(400)                                     # 8 units: a queue launch
    it.synchronize()
    got = it.read_state()
    it.close()
    ref = _run(whg, ens, 400, queue_steps=0)
    for a, b in zip(got, ref[:4]):
        assert np.array_equal(a, b)
    off = whg.Integrator(8, 8, queue_steps=0)
    off.init(inputs.solar_ensemble(50, 8))
    with pytest.raises(whg.WhgError):
        whg.whg_test_queue_timeout(off.ctx, 10)
    off.close()
