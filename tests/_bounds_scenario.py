"""Run every kernel of the library once on small inputs and print the index-
check flags of each context as JSON (run with WHG_LIBRARY pointing at the
debug build; used by test_gpu_debug_bounds.py)."""
import json

import numpy as np
import torch

from paper_2307_05683_gb300 import inputs, whg

flags = {}

ens = inputs.compact_ensemble(7, 300)                       # planet counts 2..8, stop rules
it = whg.Integrator(300, 8, gr_mode=1, close_encounter_hill=6.0, eject_factor=3.0, repack_frozen=True,
                    steps_per_launch=100, graph_launches=4, queue_steps=25)
it.init(ens)
it.step(900)
it.read_state()
it.energy()
Q, v, ns, st = it.get_raw()
it.set_raw(Q, v, ns, st)
it.step(150)
it.read_state()
flags["mixed_stop_repack_graph_queue"] = whg.whg_debug_bounds(it.ctx)
it.close()

sol = inputs.solar_ensemble(3, 70)
it = whg.Integrator(70, 8, gr_mode=0, lanes_per_system=8, interaction_schedule=1, halley_fp32=True,
                    merge_jumps=True, queue_steps=0)
it.init(sol)
it.step(300)
it.read_state()
it.energy()
flags["options"] = whg.whg_debug_bounds(it.ctx)
it.close()

dev = lambda a, dt=torch.float64: torch.tensor(a, dtype=dt, device="cuda")
it = whg.Integrator(300, 8, gr_mode=2, newton_terms=6)
whg.whg_init_device(it.ctx, dev(ens.masses), dev(ens.pos), dev(ens.vel), dev(ens.n_planets, torch.int32),
                    dev(ens.dt))
target = ens.pos[:, 1:] - ens.pos[:, :1]
loss = torch.empty(300, dtype=torch.float64, device="cuda")
whg.whg_adjoint_forward(it.ctx, 250, 50, dev(target), loss)
gx = torch.empty((300, 9, 3), dtype=torch.float64, device="cuda")
gu = torch.empty_like(gx)
gm = torch.empty((300, 9), dtype=torch.float64, device="cuda")
whg.whg_adjoint_backward(it.ctx, None, gx, gu, gm)
flags["device_init_adjoint"] = whg.whg_debug_bounds(it.ctx)
# a tape per segment, computed beside the forward half, and a second backward
# call with weights (the tape pool of the SM-split schedule)
whg.whg_init_device(it.ctx, dev(ens.masses), dev(ens.pos), dev(ens.vel), dev(ens.n_planets, torch.int32),
                    dev(ens.dt))
whg.whg_adjoint_schedule(it.ctx, -1, -1)
whg.whg_adjoint_forward(it.ctx, 250, 50, dev(target), loss)
whg.whg_adjoint_backward(it.ctx, None, gx, gu, gm)
whg.whg_adjoint_backward(it.ctx, dev(np.linspace(0.5, 2.0, 300)), gx, gu, gm)
flags["adjoint_tape_pool"] = whg.whg_debug_bounds(it.ctx)
it.close()

# the allocation-free entry point: mixed planet counts with stop rules, then
# systems of at most 3 planets, packed 8 per warp (4 lanes each by default)
c = inputs.compact_ensemble(8, 200)
small = inputs.Ensemble(c.masses[:, :4].copy(), c.pos[:, :4].copy(), c.vel[:, :4].copy(),
                        np.minimum(c.n_planets, 3).astype(np.int32), c.dt.copy())
for e, N, extra in ((ens, 8, dict(close_encounter_hill=6.0, eject_factor=3.0)), (small, 3, {})):
    opt = whg.whg_default_options()
    for k, v in extra.items():
        setattr(opt, k, v)
    S = e.n_systems
    pos = torch.empty((S, 1 + N, 3), dtype=torch.float64, device="cuda")
    whg.whg_integrate_noalloc(S, N, opt, dev(e.masses), dev(e.pos), dev(e.vel),
                              dev(e.n_planets, torch.int32), dev(e.dt), 300, pos, torch.empty_like(pos),
                              torch.empty(S, dtype=torch.int32, device="cuda"),
                              torch.empty(S, dtype=torch.float64, device="cuda"))
flags["noalloc_mixed_and_packed"] = whg.whg_noalloc_debug_bounds()

print(json.dumps(flags))
