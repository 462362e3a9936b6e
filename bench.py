#!/usr/bin/env python
"""Benchmark: FP64 system-steps/s of the Wisdom-Holman ensemble integrator.

Workload (default): 4096 Solar-System-shaped systems (star + 8 planets, the
8-planet template with masses and semi-major axes scaled by 1 + N(0, 1e-3),
e and i perturbed by Rayleigh(1e-3), angles seeded), dt = P_Mercury / 20, GR
term on.  One benchmark step = one whg_step call advancing every system by
--chunk integrator steps (default 1e4; 100 benchmark steps = the full 1e6
steps).  The state lives in registers during a launch, so there is no
per-step memory traffic to cache (with the default work queue it is reloaded
from L2 every 100 steps); L2 is flushed (256 MB write) between timed steps
anyway.

Prints ONE JSON line.  --impl reference times the CPU oracle instead (rank 0).
Multi-GPU (torchrun): each rank integrates its own ensemble of the same size
(weak scaling, no data-path collective; a barrier and a max-reduction of the
elapsed times only).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2307_05683_gb300 import inputs  # noqa: E402

METRIC = "8-planet FP64 system-steps/s on 1 GB300"
UNIT = "system-steps/s"

# Algorithmic FP64 operations per system-step (steady state, fused drift),
# counted by the oracle's counting build (add/sub, mul, div, sqrt each one
# operation); key (planets, newton_terms, gr_mode).  A CPU test keeps this
# table equal to the oracle's count.
ALG_FLOPS = {(8, 8, 1): 3464, (8, 8, 0): 3336, (8, 6, 1): 3272, (8, 8, 2): 3536}
# Of these, the Kepler solver's starting phase (initial guess and the two
# Halley steps, 8 drifts): with the halley_fp32 option they run on the FP32
# pipe, and that option's FP64 roofline counts ALG_FLOPS - START_FLOPS.
START_FLOPS = {(8, 8, 1): 776, (8, 8, 0): 776, (8, 6, 1): 776, (8, 8, 2): 776}
# The same count for systems of n = 1..8 planets (8-term series, GR on), for
# ensembles of mixed planet counts; a CPU test keeps it equal to the oracle's.
ALG_FLOPS_BY_PLANETS = {1: 349, 2: 722, 3: 1119, 4: 1540, 5: 1985, 6: 2454, 7: 2947, 8: 3464}


def fp64_flops(gr_mode: int, halley_fp32: bool, newton_terms: int = 8) -> int:
    key = (8, newton_terms, gr_mode)
    return ALG_FLOPS[key] - (START_FLOPS[key] if halley_fp32 else 0)

# FP64 peak from the unit counts and clocks: 152 SMs x 2 FP64 FMA lanes per
# clock (1.25 TFLOP/s nominal / (152 x 2.07 GHz x 2)) x 2 flops x 2.07 GHz.
SMS, FP64_LANES_PER_SM_CLK, SM_MAX_HZ = 152, 2, 2.07e9
FP64_PEAK_TFLOPS = SMS * FP64_LANES_PER_SM_CLK * 2 * SM_MAX_HZ / 1e12

PROFILE = os.path.join(ROOT, "profiles", "k_step_solar4096.md")


def parse_args():
    p = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=100)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["whg", "reference"], default="whg")
    p.add_argument("--systems", type=int, default=4096)
    p.add_argument("--chunk", type=int, default=10000, help="integrator steps per benchmark step")
    p.add_argument("--gr-mode", type=int, default=1)
    p.add_argument("--halley-fp32", type=int, choices=[0, 1], default=0,
                   help="Kepler solver's initial guess and Halley steps in FP32 (1, an option) "
                        "or FP64 (0, the library default: every step in FP64)")
    p.add_argument("--block-size", type=int, default=0)
    p.add_argument("--e2e-steps", type=int, default=5)
    p.add_argument("--cpu-seconds", type=float, default=15.0, help="CPU work of the oracle sample")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--seed", type=int, default=2024)
    p.add_argument("--only", choices=["adjoint", "sweep", "uneven"], default=None,
                   help="run just this one of the extra measurements on one GPU and print its JSON "
                        "(a short command for profiling its kernels); no benchmark line")
    return p.parse_args()


def workload(args) -> dict:
    return {"workload": f"{args.systems} Solar-System-shaped systems, star + 8 planets, FP64, "
                        f"dt = P_Mercury/20, GR term {'on' if args.gr_mode else 'off'}",
            "systems_per_gpu": args.systems, "planets": 8,
            "integrator_steps_per_bench_step": args.chunk,
            "gr_mode": args.gr_mode, "newton_terms": 8, "halley_terms": 4,
            "kepler_solver": ("initial guess + 2 Halley steps (4-term series) in FP32, 2 Newton steps "
                              "(8-term series) and f, g in FP64" if args.halley_fp32 else
                              "initial guess, 2 Halley steps (4-term series), 2 Newton steps (8-term series) "
                              "and f, g all in FP64"),
            "l2": "state register-resident during each 100-step work unit (reloaded from L2 between units); "
                  "256 MB L2 flush between timed steps"}


# ------------------------------------------------------------ environment --

def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def rank_workload(args, rank: int):
    """Weak scaling: every rank integrates its own ensemble of args.systems
    systems (seed + rank); no system is shared between ranks."""
    return inputs.solar_ensemble(args.seed + rank, args.systems)


def max_over_ranks(x: float, dist=None, device=None) -> float:
    """Maximum of a per-rank float over all ranks (the slowest rank sets the
    elapsed time of a weak-scaling step); identity without a process group."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(world: int, systems: int, chunk: int, steps: int, max_ms: float) -> float:
    """Whole-job system-steps/s: all ranks' system-steps over the slowest rank's time."""
    return world * systems * chunk * steps / (max_ms / 1e3)


def code_only(text: str) -> str:
    """C/CUDA source without comments and with whitespace runs collapsed (the
    code a compiler sees; string literals in these files hold no comment
    markers)."""
    text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
    text = re.sub(r"//[^\n]*", " ", text)
    return " ".join(text.split())


def kernel_source_hash() -> str:
    """Hash of the code that defines the step kernel (device code and its
    instantiation with 8-term Newton-phase series), comments excluded."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2307_05683_gb300", "csrc")
    for name in ("whg_device.cuh", "whg_kernels_nt8.cu"):
        h.update(name.encode())
        h.update(code_only(open(os.path.join(csrc, name)).read()).encode())
    return h.hexdigest()[:16]


def profiled_traffic():
    """DRAM bytes per k_step launch from the committed ncu summary, or None if
    the kernels changed since it was taken."""
    if not os.path.exists(PROFILE):
        return None
    text = open(PROFILE).read()
    m = re.search(r"kernel_source_sha256_16:\s*([0-9a-f]+)", text)
    t = re.search(r"dram_bytes_per_launch:\s*([0-9.eE+]+)", text)
    if not m or not t or m.group(1) != kernel_source_hash():
        return None
    return float(t.group(1))


class ClockSampler:
    """nvidia-smi samples every 200 ms while the timed region runs."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, ValueError):
            self.proc = None
        time.sleep(0.3)

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
                power.append(float(f[3]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "power_w_max": max(power) if power else None,
                "samples": len(sm), "reasons": sorted(reasons)}


# ------------------------------------------------------------ CPU oracle --

def cpu_model() -> str:
    """Host CPU model name (lscpu, else /proc/cpuinfo, else the machine type)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform
    return platform.machine()


def oracle_rate(ens, gr_mode: int, target_cpu_seconds: float, threads: int):
    """Time the oracle (as it stands) on `threads` host threads over a bounded
    sample of the ensemble: all systems, a step count sized for about
    target_cpu_seconds of CPU work.  Returns (system-steps/s, sample text)."""
    import oracle
    oracle.build()
    S = ens.n_systems
    pilot = ens.subset(np.arange(min(S, 64)))
    o = oracle.OracleEnsemble(pilot.n_systems, 8, gr_mode=gr_mode)
    o.init(pilot)
    t0 = time.perf_counter()
    o.step(20)
    per_core = pilot.n_systems * 20 / (time.perf_counter() - t0)
    n = max(10, int(target_cpu_seconds * per_core / S))
    o = oracle.OracleEnsemble(S, 8, gr_mode=gr_mode)
    o.init(ens)
    t0 = time.perf_counter()
    used = o.run_threads(n, threads)
    dt = time.perf_counter() - t0
    return S * n / dt, f"{S} systems x {n} steps on {used} threads ({dt:.1f} s wall)", used


def measure_adjoint(whg, torch, systems=1024, steps=10000, every=100, seed=4242):
    """Cost of the adjoint on the gradient workload: 1024 Solar-System-shaped
    systems, 1e4 steps, checkpoints every 100 steps, loss on the final
    heliocentric positions.  Returns CUDA-event times of a plain forward
    (whg_step), the checkpointed forward and the backward (adjoint kernels)."""
    ens = inputs.solar_ensemble(seed, systems)
    rng = np.random.default_rng(seed)
    T = ens.pos[:, 1:] - ens.pos[:, :1] + rng.normal(0, 0.05, ens.pos[:, 1:].shape)
    dev = lambda a, dt=torch.float64: torch.tensor(a, dtype=dt, device="cuda")
    stream = torch.cuda.Stream()
    res = {}
    with torch.cuda.stream(stream):
        m, x, u, npl, dt, tgt = (dev(ens.masses), dev(ens.pos), dev(ens.vel), dev(ens.n_planets, torch.int32),
                                 dev(ens.dt), dev(T))
        loss = torch.empty(systems, dtype=torch.float64, device="cuda")
        gx = torch.empty_like(x)
        gu = torch.empty_like(x)
        gm = torch.empty_like(m)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(6)]
        # the contexts are reused, as a training loop would: the first round
        # warms up and pays the one-time allocation of checkpoints and tapes
        a = whg.Integrator(systems, 8, gr_mode=1, stream=stream.cuda_stream)
        b = whg.Integrator(systems, 8, gr_mode=1, stream=stream.cuda_stream)
        for rep in range(2):
            whg.whg_init_device(a.ctx, m, x, u, npl, dt)
            whg.whg_init_device(b.ctx, m, x, u, npl, dt)
            stream.synchronize()
            ev[0].record(stream)
            a.step(steps)
            ev[1].record(stream)
            whg.whg_adjoint_forward(b.ctx, steps, every, tgt, loss)
            ev[2].record(stream)
            whg.whg_adjoint_backward(b.ctx, None, gx, gu, gm)
            ev[3].record(stream)
            stream.synchronize()
        layout = whg.whg_adjoint_layout(b.ctx)
        a.close()
        b.close()
        fwd = ev[0].elapsed_time(ev[1])
        afw = ev[1].elapsed_time(ev[2])
        bwd = ev[2].elapsed_time(ev[3])
    res = {"workload": f"{systems} Solar-System-shaped systems, {steps} steps, checkpoint every {every}, "
                       "loss = sum |Q_i(T) - target_i|^2",
           "forward_ms": round(fwd, 3), "adjoint_forward_ms": round(afw, 3),
           "adjoint_backward_ms": round(bwd, 3),
           "backward_over_forward": round(bwd / fwd, 3),
           "gradient_over_forward": round((afw + bwd) / fwd, 3),
           "finite_gradients": bool(torch.isfinite(gx).all().item() and torch.isfinite(gm).all().item()),
           "schedule": layout}
    return res


def time_rate(whg, torch, ens, window_s: float, stream, min_steps: int = 32, **kw) -> tuple[float, int]:
    """System-steps/s of one Integrator configuration on `ens`, CUDA events
    on the library's stream over a window of about window_s (and at least
    min_steps steps) after a warm-up call of the same length."""
    S = ens.n_systems
    it = whg.Integrator(S, ens.max_planets, stream=stream.cuda_stream, **kw)
    try:
        it.init(ens)
        n = max(min_steps, int(2.4e8 * window_s / S))
        it.step(n)
        it.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        it.step(n)
        e1.record(stream)
        e1.synchronize()
        return S * n / (e0.elapsed_time(e1) / 1e3), n
    finally:
        it.close()


def measure_uneven(whg, torch, systems=1 << 16, steps=20000, seed=303):
    """Uneven batch: compact systems with 2..8 planets in one ensemble, both
    stop rules on (a pair closer than 1 mutual Hill radius, a planet beyond
    100x the largest initial a), 100-step launches replayed as CUDA graphs of
    16, GR on.  Systems packed by planet count (n lanes each, 8 for n = 7;
    the default, which with a stop rule on also regroups stopped systems
    behind running ones after every graph replay), the same without that
    regrouping (repack_frozen = 0), and 8 lanes for every system.
    Rates count every system for every
    step (a frozen system counts but costs nothing once its whole warp is
    frozen); CUDA events on the library's stream after a warm-up of 1600
    steps.  The FP64 fraction counts the algorithmic flops of each system's
    planet count (idle lanes do none), every system every step."""
    ens = inputs.compact_ensemble(seed, systems)
    stream = torch.cuda.Stream()
    flops = float(np.mean([ALG_FLOPS_BY_PLANETS[int(n)] for n in ens.n_planets]))
    out = {"workload": f"{systems} compact systems, 2..8 planets, stop rules on (1 mutual Hill radius, "
                       f"100 x largest initial a), GR on, 100-step launches in graphs of 16, {steps} steps",
           "algorithmic_flops_per_system_step": round(flops, 1)}
    for name, lanes, repack in (("packed", 0, None), ("packed_no_repack", 0, False), ("lanes8", 8, None)):
        it = whg.Integrator(systems, 8, gr_mode=1, lanes_per_system=lanes, steps_per_launch=100,
                            graph_launches=16, close_encounter_hill=1.0, eject_factor=100.0,
                            repack_frozen=repack, stream=stream.cuda_stream)
        it.init(ens)
        it.step(1600)
        it.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        it.step(steps)
        e1.record(stream)
        e1.synchronize()
        ms = e0.elapsed_time(e1)
        _, _, st, _ = it.read_state()
        it.close()
        rate = systems * steps / (ms / 1e3)
        out[name] = {"system_steps_per_s": round(rate, 1), "stopped": int((st != 0).sum()),
                     "frac": round(rate * flops / 1e12 / FP64_PEAK_TFLOPS, 4)}
    return out


def throughput_sweep(whg, torch, sizes=tuple(1 << k for k in range(14, 21)), window_s=1.0, min_steps=1000,
                     seed=77):
    """System-steps/s and FP64 fraction against ensemble size (Solar-System-
    shaped systems, GR on, default solver).  At each size the autotuner picks
    the launch configuration among those that leave results bit for bit
    unchanged (block size, work queue, automatic launch lengths or 100-step
    launches replayed as CUDA graphs of 16; 0.05 s per candidate), then that
    configuration is timed with CUDA events over a window of at least
    window_s and min_steps steps after a warm-up call of the same length
    (step time does not depend on the coordinates, so a window stands for
    the nominal 1e7-step run)."""
    from paper_2307_05683_gb300 import autotune
    base = inputs.solar_ensemble(seed, 4096)
    out = []
    stream = torch.cuda.Stream()
    for S in sizes:
        ens = base.tile(S)
        best = autotune.tune(ens, gr_mode=1, cache_path=None, window_s=0.05, space="launch")
        cfg = {k: best[k] for k in ("block_size", "queue_steps", "steps_per_launch", "graph_launches")}
        rate, n = time_rate(whg, torch, ens, window_s, stream, min_steps=min_steps, gr_mode=1, **cfg)
        out.append({"systems": S, "steps": n, "system_steps_per_s": round(rate, 1),
                    "frac": round(rate * fp64_flops(1, False) / 1e12 / FP64_PEAK_TFLOPS, 4),
                    "config": cfg, "candidates_timed": best["tried"]})
    return out


def solver_comparison(whg, torch, ens, gr_mode: int, window_s=1.0):
    """The bench workload with the whole Kepler solver in FP64 (the paper's
    arithmetic) beside the default FP32 starting phase, same timing method."""
    stream = torch.cuda.Stream()
    out = {}
    for h32 in (False, True):
        rate, n = time_rate(whg, torch, ens, window_s, stream, gr_mode=gr_mode, halley_fp32=h32)
        fl = fp64_flops(gr_mode, h32)
        out["fp32_start" if h32 else "all_fp64"] = {
            "system_steps_per_s": round(rate, 1), "steps": n, "fp64_flops_per_system_step": fl,
            "frac": round(rate * fl / 1e12 / FP64_PEAK_TFLOPS, 4)}
    return out


# ------------------------------------------------------------ GPU arm --

def run_whg(args):
    import torch
    from paper_2307_05683_gb300 import build, whg

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group(backend="nccl", device_id=torch.device("cuda", local))
    build.build()
    S, chunk = args.systems, args.chunk
    ens = rank_workload(args, rank)
    stream = torch.cuda.Stream()
    it = whg.Integrator(S, 8, gr_mode=args.gr_mode, block_size=args.block_size,
                        halley_fp32=bool(args.halley_fp32), stream=stream.cuda_stream)
    it.init(ens)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            it.step(chunk)
        stream.synchronize()
        launches_per_step = None
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(args.steps)]
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        gpu_idx = local
        cvd = os.environ.get("CUDA_VISIBLE_DEVICES", "")
        if cvd and cvd.split(",")[0].strip().isdigit():
            gpu_idx = int(cvd.split(",")[local].strip())
        clocks = ClockSampler(gpu_idx)
        clocks.start()
        l0 = it.launches
        for k in range(args.steps):
            flush.add_(1.0)
            ev[k][0].record(stream)
            it.step(chunk)
            ev[k][1].record(stream)
        stream.synchronize()
        torch.cuda.synchronize()
        launches = it.launches - l0
        clock_info = clocks.stop()
        if dist:
            dist.barrier()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total_ms = float(sum(step_ms))
    worst = max_over_ranks(total_ms, dist, "cuda")
    value = job_throughput(world, S, chunk, args.steps, worst)
    launches_per_step = launches / args.steps

    # end to end through the public API: pinned host inputs -> init (H2D) ->
    # step -> read_state (D2H), wall clock.
    pinned = {}
    for name in ("masses", "pos", "vel", "dt"):
        a = getattr(ens, name)
        t = torch.empty(a.shape, dtype=torch.float64, pin_memory=True)
        t.numpy()[...] = a
        pinned[name] = t
    npl = torch.empty(S, dtype=torch.int32, pin_memory=True)
    npl.numpy()[...] = ens.n_planets
    out = {k: torch.empty(s, dtype=d, pin_memory=True) for k, s, d in
           (("pos", (S, 9, 3), torch.float64), ("vel", (S, 9, 3), torch.float64),
            ("status", (S,), torch.int32), ("t", (S,), torch.float64))}
    h2d = sum(v.numel() * v.element_size() for v in pinned.values()) + npl.numel() * 4
    d2h = sum(v.numel() * v.element_size() for v in out.values())
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.e2e_steps):
        whg.whg_init(it.ctx, pinned["masses"].numpy(), pinned["pos"].numpy(), pinned["vel"].numpy(),
                     npl.numpy(), pinned["dt"].numpy())
        it.step(chunk)
        whg.whg_read_state(it.ctx, out["pos"].numpy(), out["vel"].numpy(), out["status"].numpy(),
                           out["t"].numpy())
    e2e_s = max_over_ranks(time.perf_counter() - t0, dist, "cuda")
    e2e_value = job_throughput(world, S, chunk, args.e2e_steps, 1e3 * e2e_s)
    bad = int((out["status"].numpy() != 0).sum())

    if rank != 0:
        it.close()
        if dist:
            dist.destroy_process_group()
        return

    flops = fp64_flops(args.gr_mode, bool(args.halley_fp32))
    kernel_ms = total_ms / args.steps / max(launches_per_step, 1.0)
    achieved = flops * S * (chunk / max(launches_per_step, 1.0)) / (kernel_ms / 1e3) / 1e12
    adjoint = measure_adjoint(whg, torch) if world == 1 else None
    sweep = throughput_sweep(whg, torch) if world == 1 else None
    solvers = solver_comparison(whg, torch, ens, args.gr_mode) if world == 1 else None
    uneven = measure_uneven(whg, torch) if world == 1 else None
    roofline = {"bound": "alu", "achieved": round(achieved, 4), "peak": round(FP64_PEAK_TFLOPS, 4),
                "unit": "TFLOP/s", "frac": round(achieved / FP64_PEAK_TFLOPS, 4),
                "traffic": profiled_traffic(),
                "kernel": "k_step_queue<8,1> via queue_unit (FP64 pipe)",
                "algorithmic_flops_per_system_step": flops,
                "fp32_flops_per_system_step": START_FLOPS[(8, 8, args.gr_mode)] if args.halley_fp32 else 0,
                "peak_basis": "recipe unit counts x clocks: 152 SMs x 2 FP64 FMA/clk x 2 x 2.07 GHz"}
    line = {"metric": METRIC, "value": round(value, 1), "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(total_ms / args.steps, 4),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded Solar-System-shaped ensemble)",
            "config": workload(args),
            "roofline": roofline,
            "e2e": {"value": round(e2e_value, 1), "unit": UNIT, "h2d_bytes_per_step": int(h2d),
                    "d2h_bytes_per_step": int(d2h), "steps": args.e2e_steps,
                    "api": "whg_init(host) + whg_step + whg_read_state(host)"},
            "gpu_launches": int(launches),
            "adjoint": adjoint,
            "sweep": sweep,
            "solver_comparison": solvers,
            "uneven_batch": uneven,
            "clocks": clock_info,
            "systems_flagged": bad}
    it.close()
    if world == 1 and not args.no_cpu_baseline:
        threads = os.cpu_count() or 1
        rate, sample, used = oracle_rate(ens, args.gr_mode, args.cpu_seconds, threads)
        line["cpu_baseline"] = {"value": round(rate, 1), "unit": UNIT, "cores": used, "kind": "oracle",
                                "sample": sample, "per_core": round(rate / max(used, 1), 1),
                                "cpu_model": cpu_model()}
    if dist:
        dist.destroy_process_group()
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------ reference arm --

def run_reference(args):
    """The CPU oracle as it stands, on all host cores, rank 0 only."""
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import oracle
    oracle.build()
    S = args.systems
    ens = inputs.solar_ensemble(args.seed, S)
    threads = os.cpu_count() or 1
    o = oracle.OracleEnsemble(S, 8, gr_mode=args.gr_mode)
    o.init(ens)
    t0 = time.perf_counter()
    o.run_threads(5, threads)
    rate0 = S * 5 / (time.perf_counter() - t0)
    # each reference step: every system advanced by n_ref steps, ~1 s of wall time,
    # so --steps K --warmup W ends within a few minutes for K ~ 100
    n_ref = max(1, int(rate0 * 1.0 / S))
    for _ in range(args.warmup):
        o.run_threads(n_ref, threads)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        o.run_threads(n_ref, threads)
    wall = time.perf_counter() - t0
    value = S * n_ref * args.steps / wall
    sample = f"{S} systems x {n_ref} steps per benchmark step on {threads} threads"
    line = {"impl": "reference", "metric": METRIC, "value": round(value, 1), "unit": UNIT,
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(1e3 * wall / args.steps, 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded Solar-System-shaped ensemble)", "config": workload(args),
            "note": "the oracle runs the whole Kepler solver in FP64",
            "cpu_baseline": {"value": round(value, 1), "unit": UNIT, "cores": threads, "kind": "oracle",
                             "sample": sample, "per_core": round(value / max(threads, 1), 1),
                             "cpu_model": cpu_model()},
            "e2e": {"value": round(value, 1), "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_only(args):
    import torch
    from paper_2307_05683_gb300 import build, whg
    torch.cuda.set_device(0)
    build.build()
    whg.load()
    fn = {"adjoint": measure_adjoint, "sweep": throughput_sweep, "uneven": measure_uneven}[args.only]
    print(json.dumps({args.only: fn(whg, torch)}), flush=True)


def main():
    args = parse_args()
    if args.impl == "reference":
        run_reference(args)
    elif args.only:
        run_only(args)
    else:
        run_whg(args)


if __name__ == "__main__":
    main()
