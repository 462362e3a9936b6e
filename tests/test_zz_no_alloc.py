"""whg_integrate_noalloc: the allocation-free entry point, for callers that
cannot allocate device memory (frameworks that pool all GPU memory up front,
hosts that forbid device allocation while running, loops that cannot pay for
cudaMalloc's device-wide synchronization).

Calls in a row through the C ABI, each compared with the context-based
entry points (whg_create / whg_init / whg_step / whg_read_state) on the same
inputs, within the parity tolerance of the other tests (1e-12 relative to the
system's scale).  Later calls are smaller than the first, so results that
depended on contents left behind in the shared scratch array would show.
Device free memory must not change across a call.  Kept in its own file so
that it is collected last.
"""
import numpy as np
import pytest

from paper_2307_05683_gb300 import inputs

pytestmark = pytest.mark.gpu


def _lanes_for(max_planets):
    """The lane group the allocation-free call gives every system by default:
    one lane per planet, 8 lanes for 7 planets."""
    return 8 if max_planets == 7 else max_planets


def _context_path(whg, ens, n, **opts):
    # same lane group for every system as the allocation-free call uses
    it = whg.Integrator(ens.n_systems, ens.max_planets, gr_mode=1,
                        lanes_per_system=_lanes_for(ens.max_planets), **opts)
    it.init(ens)
    it.step(n)
    out = it.read_state()
    it.close()
    return out


def _first_planets(ens, k):
    """The same systems cut to their first k planets (a packed lane group)."""
    return inputs.Ensemble(ens.masses[:, :k + 1].copy(), ens.pos[:, :k + 1].copy(),
                           ens.vel[:, :k + 1].copy(), np.minimum(ens.n_planets, k).astype(np.int32),
                           ens.dt.copy())


def test_noalloc_matches_context_entry_points_calls_in_a_row():
    """Three calls in a row: 8-lane systems, 3-planet systems packed ten to a
    warp (lanes_per_system 0), and mixed planet counts with both stop rules
    on (status and stop times must agree bit for bit)."""
    import torch
    from paper_2307_05683_gb300 import build, whg

    build.build()
    whg.load()
    torch.cuda.init()
    stop = dict(close_encounter_hill=6.0, eject_factor=3.0)
    cases = [(inputs.solar_ensemble(21, 3000), 700, {}),
             (_first_planets(inputs.compact_ensemble(24, 1500), 3), 500, {}),
             (inputs.compact_ensemble(22, 900), 400, stop)]
    for call, (ens, n, extra) in enumerate(cases):
        S, N = ens.n_systems, ens.max_planets
        ref_pos, ref_vel, ref_st, ref_t = _context_path(whg, ens, n, **extra)
        if extra:
            assert (ref_st != 0).any()       # the stop rules really stop some systems
        dev = lambda a, dt=torch.float64: torch.tensor(a, dtype=dt, device="cuda")
        m, x, u = dev(ens.masses), dev(ens.pos), dev(ens.vel)
        npl, dt = dev(ens.n_planets, torch.int32), dev(ens.dt)
        pos = torch.full((S, 1 + N, 3), np.nan, dtype=torch.float64, device="cuda")
        vel = torch.full_like(pos, np.nan)
        st = torch.full((S,), -1, dtype=torch.int32, device="cuda")
        tt = torch.full((S,), np.nan, dtype=torch.float64, device="cuda")
        opt = whg.whg_default_options()
        opt.gr_mode = 1
        for k, v in extra.items():
            setattr(opt, k, v)
        stream = torch.cuda.current_stream()
        torch.cuda.synchronize()
        free_before = torch.cuda.mem_get_info()[0]
        whg.whg_integrate_noalloc(S, N, opt, m, x, u, npl, dt, n, pos, vel, st, tt,
                                  stream=stream.cuda_stream)
        torch.cuda.synchronize()
        free_after = torch.cuda.mem_get_info()[0]
        if call > 0:           # the first call may load the library's device image
            assert free_after == free_before
        p, v = pos.cpu().numpy(), vel.cpu().numpy()
        sx = np.abs(ref_pos).max(axis=(1, 2))[:, None, None]
        su = np.abs(ref_vel).max(axis=(1, 2))[:, None, None]
        assert np.array_equal(st.cpu().numpy(), ref_st)
        assert np.array_equal(tt.cpu().numpy(), ref_t)
        assert (np.abs(p - ref_pos) / sx).max() <= 1e-12
        assert (np.abs(v - ref_vel) / su).max() <= 1e-12


def test_noalloc_rejects_sizes_beyond_its_scratch():
    import torch
    from paper_2307_05683_gb300 import build, whg

    build.build()
    S = whg.WHG_NOALLOC_MAX_LANES // 8 + 1          # one system too many at 8 lanes each
    ens = inputs.solar_ensemble(23, 4).tile(S)
    dev = lambda a, dt=torch.float64: torch.tensor(a, dtype=dt, device="cuda")
    pos = torch.empty((S, 9, 3), dtype=torch.float64, device="cuda")
    with pytest.raises(whg.WhgError) as e:
        whg.whg_integrate_noalloc(S, 8, None, dev(ens.masses), dev(ens.pos), dev(ens.vel),
                                  None, dev(ens.dt), 10, pos, torch.empty_like(pos))
    assert e.value.code == whg.WHG_EINVAL
    assert "scratch" in whg.whg_last_error(None)
