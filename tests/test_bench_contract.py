"""Host-side pieces of bench.py (no GPU): the algorithmic flop table equals the
oracle's counting build, and the peak arithmetic."""
import importlib

import pytest


def test_alg_flops_table_matches_oracle_count(orc):
    bench = importlib.import_module("bench")
    for (n, nt, gr), flops in bench.ALG_FLOPS.items():
        c = orc.count_flops(n, nt, gr)
        assert c["flops"] == flops
        assert c["start_phase"] == bench.START_FLOPS[(n, nt, gr)]
        assert bench.fp64_flops(gr, True, nt) == flops - c["start_phase"]
        assert bench.fp64_flops(gr, False, nt) == flops


def test_flops_by_planet_count_match_oracle(orc):
    """The per-planet-count table (mixed ensembles' roofline) equals the
    oracle's counting build for 1..8 planets, 8-term series, GR on."""
    bench = importlib.import_module("bench")
    assert sorted(bench.ALG_FLOPS_BY_PLANETS) == list(range(1, 9))
    for n, flops in bench.ALG_FLOPS_BY_PLANETS.items():
        assert orc.count_flops(n, 8, 1)["flops"] == flops, n
    assert bench.ALG_FLOPS_BY_PLANETS[8] == bench.ALG_FLOPS[(8, 8, 1)]


def test_start_phase_count_follows_the_halley_iterations(orc):
    """The starting-phase tally grows by one Halley step's flops per extra
    iteration and is the initial guess alone without Halley steps, so it
    covers exactly the guess and the Halley steps."""
    c = [orc.count_flops(8, 8, 1, halley_iters=k) for k in range(4)]
    per_step = c[1]["start_phase"] - c[0]["start_phase"]
    assert per_step > 0 and c[0]["start_phase"] > 0                 # guess alone without Halley
    assert all(c[k + 1]["start_phase"] - c[k]["start_phase"] == per_step for k in range(3))
    # the rest of the step does not depend on the Halley iterations
    assert len({x["flops"] - x["start_phase"] for x in c}) == 1
    assert c[2]["start_phase"] % 8 == 0                             # same work in each of 8 drifts


def test_fp64_peak_from_unit_counts():
    bench = importlib.import_module("bench")
    assert bench.FP64_PEAK_TFLOPS == pytest.approx(1.2586, rel=1e-4)
    assert bench.FP64_PEAK_TFLOPS == pytest.approx(1.25, rel=0.01)   # nominal FP64 figure


def test_kernel_source_hash_is_stable():
    bench = importlib.import_module("bench")
    assert bench.kernel_source_hash() == bench.kernel_source_hash()
    assert len(bench.kernel_source_hash()) == 16


def test_reference_arm_prints_the_contract_line(orc):
    """bench.py --impl reference (the oracle on the host cores) prints one JSON
    line with the arm's metric and the reference-arm keys."""
    import json
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "0",
                          "--systems", "64"], cwd=root, capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    bench = importlib.import_module("bench")
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["unit"] == bench.UNIT
    assert d["value"] > 0 and d["higher_is_better"] is True and d["dtype"] == "f64"
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"]
    assert cb["per_core"] > 0 and isinstance(cb["cpu_model"], str) and cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}


def test_kernel_hash_ignores_comments_only():
    bench = importlib.import_module("bench")
    a = "int f(int x) { // doubles x\n  return 2 * x; /* plain */ }"
    b = "int f(int x) {\n  return 2 * x;\n}  // other words"
    c = "int f(int x) { return 3 * x; }"
    assert bench.code_only(a) == bench.code_only(b) != bench.code_only(c)


def _hand_count(n, nt, gr, halley_iters=2):
    """Flops of one steady-state step (K(dt) J I [GR] J) counted by hand from
    the operations each sub-step needs; masses, dt and c are constants (their
    products are not counted), as in the counting build.
    Kepler drift per planet (Sec. 3.2, Eq. 3):
      prologue r0 (3 mul, 2 add, sqrt), eta0 and v^2 (5 each), beta (div, add),
      zeta0 (mul, add): 20;
      initial guess h/r0: 1;
      Stiefel functions with T terms (series through z^T): X^2, z (2), two
      Horner series of T steps (4 each), G0..G3 (8): 4T + 10;
      Halley step (T = 4): 26 + F 6 + F' 5 + F'' 3 + update 8 = 48;
      Newton step: 4 nt + 10 + F 6 + F' 5 + update 2 = 4 nt + 23;
      final G_n (4 nt + 10), r 5, f 3, g 2, fdot 3, gdot 3, new Q and v 18.
    Jump (Sec. 3.4, Eq. 6), per planet and jump: sum m v (6), Q update (6).
    Interaction (Sec. 3.3, Eq. 5), per pair: difference 3, r^2 5, r^3 2,
      two mass factors 2, both accelerations 12; per planet v += h a: 6.
    GR per planet: r^2 5, 1/r^4 factor 2, a 3, kick 6; mode 2 adds the
      back-reaction sum (6) and its subtraction (3)."""
    kepler = 20 + 1 + 48 * halley_iters + 2 * (4 * nt + 23) + (4 * nt + 10) + 34
    per_planet = kepler + 2 * 12 + 6 + (16 if gr else 0) + (9 if gr == 2 else 0)
    return n * per_planet + 24 * n * (n - 1) // 2, n * (1 + 48 * halley_iters)


@pytest.mark.parametrize("gr", [0, 1, 2])
@pytest.mark.parametrize("nt", [6, 8])
def test_flop_count_matches_hand_count(orc, gr, nt):
    """The counting build of the oracle (the roofline's algorithmic flops)
    agrees with a hand count of every sub-step for 1..8 planets and 0..3
    Halley steps; 3464 for 8 planets, 8-term series and GR on."""
    for n in range(1, 9):
        for hi in (0, 1, 2, 3):
            c = orc.count_flops(n, nt, gr, halley_iters=hi)
            assert (c["flops"], c["start_phase"]) == _hand_count(n, nt, gr, hi), (n, nt, gr, hi)
    assert _hand_count(8, 8, 1) == (3464, 776) and _hand_count(8, 8, 0)[0] == 3336
