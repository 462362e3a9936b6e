"""Autotuner for the launch configuration of an ensemble.

Times candidate configurations of the library on the current GPU for the
given ensemble shape (system count, planet-count histogram, GR mode, series
length) and keeps the fastest in a JSON cache:

* lane packing: systems grouped by planet count with n lanes each (0), or one
  lane group for all systems (the power of two >= max planets),
* CUDA block size (32, 64 or 128 threads),
* steps per launch (automatic, or shorter launches),
* CUDA-graph replay of step launches (off, or 16 launches per graph),
* interaction schedule (third-law rotations, or all L-1 rotations),
* work queue (100-step units, or one warp per warp-group for a whole launch).

Block size, launch length and graphs never change results; the packing and
the schedule only change the order of the sums (rounding).  The timing uses CUDA
events around whg_step on the library's stream after a warm-up call of the
same length.
"""
from __future__ import annotations

import itertools
import json
import os
import time

import numpy as np

from . import whg

DEFAULT_CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_build", "autotune.json")


def _key(ens, gr_mode: int, newton_terms: int, device: str) -> str:
    hist = np.bincount(np.asarray(ens.n_planets), minlength=9).tolist()
    return f"{device}|S={ens.n_systems}|N={ens.max_planets}|hist={hist}|gr={gr_mode}|nt={newton_terms}"


def candidates(ens, space: str = "full"):
    """Configurations to time.  space "full": every dimension above.
    space "launch": only the dimensions that leave results bit for bit
    unchanged (block size, work queue, and short launches replayed as CUDA
    graphs against automatic launch lengths), with the default packing and
    interaction schedule."""
    if space == "launch":
        yield from ({"block_size": b, "queue_steps": q, "steps_per_launch": 0, "graph_launches": 0}
                    for b, q in ((32, 100), (32, 0), (64, 0)))
        yield {"block_size": 32, "queue_steps": 0, "steps_per_launch": 100, "graph_launches": 16}
        return
    nmax = ens.max_planets
    uniform = 1
    while uniform < nmax:
        uniform <<= 1
    lanes = [0] if uniform == nmax and np.all(ens.n_planets == nmax) else [0, uniform]
    for L, block, spl, graph, sched, queue in itertools.product(lanes, (32, 64, 128), (0, 64), (0, 16), (0, 1),
                                                                (0, 100)):
        if queue and block != 32:                    # queue launches always use one-warp blocks
            continue
        yield {"lanes_per_system": L, "block_size": block, "steps_per_launch": spl, "graph_launches": graph,
               "interaction_schedule": sched, "queue_steps": queue}


def min_steps(ens, cfg: dict, window_s: float) -> int:
    """Steps timed for one configuration: about window_s of work at ~2e8
    system-steps/s, at least two whole graph replays when graphs are on, and
    at least the 4 units per warp-group from which a launch uses the work
    queue when the queue is on (else the timing would measure plain
    launches)."""
    n = max(16, int(2.0e8 * window_s / ens.n_systems))
    if cfg.get("steps_per_launch"):
        n = max(n, 2 * cfg["steps_per_launch"] * max(1, cfg.get("graph_launches", 0)))
    if cfg.get("queue_steps") and not cfg.get("steps_per_launch"):
        n = max(n, 4 * cfg["queue_steps"])
    return n


def time_config(ens, cfg: dict, gr_mode: int, newton_terms: int, window_s: float = 0.05) -> float:
    """system-steps/s of one configuration over a window of about window_s."""
    import torch
    S = ens.n_systems
    stream = torch.cuda.Stream()
    it = whg.Integrator(S, ens.max_planets, gr_mode=gr_mode, newton_terms=newton_terms,
                        stream=stream.cuda_stream, **cfg)
    try:
        it.init(ens)
        n = min_steps(ens, cfg, window_s)
        it.step(n)
        it.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        it.step(n)
        e1.record(stream)
        e1.synchronize()
        return S * n / (e0.elapsed_time(e1) / 1e3)
    finally:
        it.close()


def tune(ens, gr_mode: int = 1, newton_terms: int = 8, cache_path: str | None = DEFAULT_CACHE,
         window_s: float = 0.05, force: bool = False, space: str = "full") -> dict:
    """Best configuration for this ensemble shape (from the cache if present).
    Returns the option values plus the measured rate under "system_steps_per_s".
    Candidates whose shortest timing (two graph replays, or the work queue's
    4 units) would exceed 20 windows of work are skipped: at that size one
    launch is long enough that replaying it as a graph saves nothing, and
    the warp-groups fill so many waves that the queue has little to
    balance."""
    import torch
    device = torch.cuda.get_device_name()
    key = _key(ens, gr_mode, newton_terms, device) + ("" if space == "full" else f"|space={space}")
    cache = {}
    if cache_path and os.path.exists(cache_path):
        try:
            cache = json.load(open(cache_path))
        except (OSError, ValueError):
            cache = {}
    if not force and key in cache:
        return dict(cache[key])
    results = []
    budget = 20 * max(16, int(2.0e8 * window_s / ens.n_systems))
    for cfg in candidates(ens, space):
        if min_steps(ens, cfg, window_s) > budget:
            continue
        results.append((time_config(ens, cfg, gr_mode, newton_terms, window_s), cfg))
    rate, best = max(results, key=lambda r: r[0])
    entry = dict(best, system_steps_per_s=rate, tried=len(results), when=time.strftime("%Y-%m-%dT%H:%M:%S"))
    if cache_path:
        os.makedirs(os.path.dirname(cache_path), exist_ok=True)
        cache[key] = entry
        tmp = cache_path + f".{os.getpid()}.tmp"
        with open(tmp, "w") as f:
            json.dump(cache, f, indent=1, sort_keys=True)
        os.replace(tmp, cache_path)
    return entry


def integrator(ens, gr_mode: int = 1, newton_terms: int = 8, **kw) -> "whg.Integrator":
    """An Integrator with the tuned launch configuration for this ensemble."""
    best = tune(ens, gr_mode, newton_terms, **kw)
    cfg = {k: best[k] for k in ("lanes_per_system", "block_size", "steps_per_launch", "graph_launches",
                                "interaction_schedule", "queue_steps") if k in best}
    return whg.Integrator(ens.n_systems, ens.max_planets, gr_mode=gr_mode, newton_terms=newton_terms, **cfg)
