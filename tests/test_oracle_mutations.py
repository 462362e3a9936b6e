"""Planted mistakes in the oracle: every one must fail a pin.

Each entry below changes one expression of a temporary copy of the oracle's C
source into a plausible mistake (a dropped term, a wrong sign, index or
operand).  The copy is compiled on its own and the oracle's pin tests
(tests/test_oracle_kepler.py, test_oracle_map.py, test_oracle_stop_rules.py)
are run against it in a subprocess (ORC_LIBRARY selects the library).  The
test requires every mutant to fail at least one pin, and the unchanged copy,
built the same way, to pass them all.  The one check that compares the
oracle with itself (fused drifts against single sub-steps) is left out; the
remaining pins are independent of the oracle (closed forms, brute force,
conservation laws, exact orbits, a high-order reference integration), so
this shows that they constrain each part of the map.  The dual-number build
that gives the adjoint's reference gradients gets the same treatment for its
derivative rules, against its own pins (central differences of the plain
oracle, invariances of the loss).  CPU only.
"""
import concurrent.futures
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PINS = ["tests/test_oracle_kepler.py", "tests/test_oracle_map.py", "tests/test_oracle_stop_rules.py"]
# compares the oracle's fused step with its own single sub-steps, so it is left
# out: a mistake must be caught by a pin from outside the oracle
SELF_CHECKS = ["tests/test_oracle_map.py::test_fused_drifts_equal_eq2_composition"]

# name: (file, original text, planted mistake) -- what the original computes
MUTATIONS = {
    # Kepler drift, Sec. 3.2 / Eq. 3 (mu = G m_0, universal variables)
    "kepler_mu_includes_planet": ("orc_core.c", "orc_kepler_drift(s->m0, hK,", "orc_kepler_drift(s->m0 + s->m[i], hK,"),
    "beta_without_factor_2": ("orc_core.c", "orc_real beta = 2.0 * mu / r0 - v2;", "orc_real beta = mu / r0 - v2;"),
    "halley_denominator_sign": ("orc_core.c", "(2.0 * Fp * Fp - F * Fpp)", "(2.0 * Fp * Fp + F * Fpp)"),
    "newton_step_sign": ("orc_core.c", "X = X - F / Fp;", "X = X + F / Fp;"),
    "stumpff_series_index": ("orc_core.c", "s2 = orc_inv_factorial(2 * k + 2) - z * s2;",
                             "s2 = orc_inv_factorial(2 * k + 1) - z * s2;"),
    "c1_from_c2": ("orc_core.c", "G[1] = X * (1.0 - z * c3);", "G[1] = X * (1.0 - z * c2);"),
    "f_over_r_not_r0": ("orc_core.c", "orc_real f = 1.0 - mu * G[2] / r0;", "orc_real f = 1.0 - mu * G[2] / r;"),
    "g_uses_G2": ("orc_core.c", "orc_real g = h - mu * G[3];", "orc_real g = h - mu * G[2];"),
    "fdot_sign": ("orc_core.c", "orc_real fd = -mu * G[1] / (r * r0);", "orc_real fd = mu * G[1] / (r * r0);"),
    "gdot_over_r0": ("orc_core.c", "orc_real gd = 1.0 - mu * G[2] / r;", "orc_real gd = 1.0 - mu * G[2] / r0;"),
    # Jump, Sec. 3.4 / Eq. 6
    "jump_sign": ("orc_core.c", "s->Q[i][c] = s->Q[i][c] + h / s->m0 * Psum[c];",
                  "s->Q[i][c] = s->Q[i][c] - h / s->m0 * Psum[c];"),
    "jump_without_masses": ("orc_core.c", "Psum[c] = Psum[c] + s->m[i] * s->v[i][c];",
                            "Psum[c] = Psum[c] + s->v[i][c];"),
    # Interaction, Sec. 3.3 / Eq. 5
    "interaction_sign": ("orc_core.c", "a[i][c] = a[i][c] - ki * d[c];", "a[i][c] = a[i][c] + ki * d[c];"),
    "interaction_own_mass": ("orc_core.c", "ki = s->m[j] / r3;", "ki = s->m[i] / r3;"),
    "reaction_wrong_mass": ("orc_core.c", "kj = s->m[i] / r3;", "kj = s->m[j] / r3;"),
    "inverse_square_not_cube": ("orc_core.c", "r3 = r2 * orc_sqrt(r2);", "r3 = r2;"),
    # GR term, Sec. 3.3
    "gr_factor_3": ("orc_core.c", "-6.0 * m0 * m0", "-3.0 * m0 * m0"),
    "gr_mode2_back_reaction_sign": ("orc_core.c", "a[i][c] = a[i][c] - back[c];", "a[i][c] = a[i][c] + back[c];"),
    # Step composition, Sec. 3.1 / Eq. 2 and the output sync (Sec. 3.5 list)
    "first_drift_full_step": ("orc_core.c", "(s->nstep == 0) ? 0.5 * s->dt : s->dt", "s->dt"),
    "second_jump_missing": ("orc_core.c", "if (opt->gr_mode) orc_gr_kick(s, s->dt, opt);\n            orc_jump(s, 0.5 * s->dt);",
                            "if (opt->gr_mode) orc_gr_kick(s, s->dt, opt);"),
    "merged_jump_half": ("orc_core.c", "orc_jump(s, s->dt);\n            if (orc_interaction",
                         "orc_jump(s, 0.5 * s->dt);\n            if (orc_interaction"),
    "no_output_sync": ("orc_core.c", "if (s->nstep > 0) {\n        int i;", "if (0) {\n        int i;"),
    "no_rollback": ("orc_core.c", "memcpy(s->Q, Qs, sizeof(Qs));", "(void)Qs;"),
    # Democratic heliocentric coordinates (Sec. 3.1) and their inverse
    "v_relative_to_star": ("orc_core.c", "s->v[i][c] = u[3 * (1 + i) + c] - s->Vcm[c];",
                           "s->v[i][c] = u[3 * (1 + i) + c] - u[c];"),
    "star_velocity_over_M": ("orc_ensemble.c", "u[c] = s->Vcm[c] - sp / s->m0;", "u[c] = s->Vcm[c] - sp / s->M;"),
    # Energy, Eq. 1
    "energy_without_HJ": ("orc_ensemble.c", "HJ = (P[0] * P[0] + P[1] * P[1] + P[2] * P[2]) / (2.0 * sy.m0);",
                          "HJ = 0.0;"),
    "energy_HI_sign": ("orc_ensemble.c", "HI -= sy.m[i] * sy.m[j] / sqrt(d2);", "HI += sy.m[i] * sy.m[j] / sqrt(d2);"),
    # Stop rules (an ensemble option, not the paper's map)
    "hill_radius_without_3": ("orc_core.c", "/ (3.0 * orc_mass_value(s->m0))", "/ (orc_mass_value(s->m0))"),
    "eject_radius_unscaled": ("orc_core.c", "rej *= opt->eject_factor;", "rej *= 1.0;"),
}

# Derivative rules of the dual-number build that gives the adjoint's reference
# gradients (oracle/tangent.cpp); pinned by tests/test_oracle_tangent.py.
TANGENT_PINS = ["tests/test_oracle_tangent.py"]
TANGENT_MUTATIONS = {
    "product_rule_one_term": ("tangent.cpp", "a.d * b.v + a.v * b.d)", "a.d * b.v)"),
    "quotient_rule_sign": ("tangent.cpp", "(a.d * b.v - a.v * b.d) / (b.v * b.v)", "(a.d * b.v + a.v * b.d) / (b.v * b.v)"),
    "sqrt_derivative_factor": ("tangent.cpp", "Dual(r, x.d / (2.0 * r))", "Dual(r, x.d / r)"),
    "negation_derivative": ("tangent.cpp", "return Dual(-a.v, -a.d);", "return Dual(-a.v, a.d);"),
    "mass_direction_seed": ("tangent.cpp", "md[k] = Dual(m[k], (kind == 2 && body == k) ? 1.0 : 0.0);",
                            "md[k] = Dual(m[k], 0.0);"),
}


def _build(name, workdir):
    """Copy the oracle's C sources, plant one mistake (name "unchanged":
    none), compile; returns the library path."""
    import oracle
    src = os.path.join(workdir, name)
    os.makedirs(src)
    for f in os.listdir(os.path.join(ROOT, "oracle")):
        if f.endswith((".c", ".cpp", ".h")):
            shutil.copy(os.path.join(ROOT, "oracle", f), src)
    tangent = name in TANGENT_MUTATIONS or name == "unchanged_tangent"
    if not name.startswith("unchanged"):
        f, old, new = (TANGENT_MUTATIONS if tangent else MUTATIONS)[name]
        path = os.path.join(src, f)
        text = open(path).read()
        assert text.count(old) == 1, f"{name}: the original text must occur exactly once in {f}"
        open(path, "w").write(text.replace(old, new))
    if tangent:
        lib = os.path.join(src, "liborc_tangent.so")
        oracle.compile_tangent(src, lib)
    else:
        lib = os.path.join(src, "liborc.so")
        oracle.compile_library(src, lib)
    return lib


def _run_pins(lib, tangent=False):
    env = dict(os.environ, **({"ORC_TANGENT_LIBRARY": lib} if tangent else {"ORC_LIBRARY": lib}))
    pins = TANGENT_PINS if tangent else PINS
    deselect = [a for t in SELF_CHECKS for a in ("--deselect", t)]
    r = subprocess.run([sys.executable, "-m", "pytest", *pins, *deselect, "-x", "-q", "-m", "not gpu",
                        "-p", "no:cacheprovider"], cwd=ROOT, env=env, capture_output=True, text=True,
                       timeout=600)
    failed = [ln.split(" ")[1] for ln in r.stdout.splitlines() if ln.startswith("FAILED ")]
    return r.returncode, failed, r.stdout[-400:]


def test_every_planted_mistake_fails_a_pin(tmp_path, orc):
    names = ["unchanged", "unchanged_tangent", *MUTATIONS, *TANGENT_MUTATIONS]
    workers = max(2, min(8, os.cpu_count() or 2))

    def one(name):
        tangent = name in TANGENT_MUTATIONS or name == "unchanged_tangent"
        return name, _run_pins(_build(name, str(tmp_path)), tangent)

    with concurrent.futures.ThreadPoolExecutor(max_workers=workers) as ex:
        results = dict(ex.map(one, names))
    for control in ("unchanged", "unchanged_tangent"):
        rc, failed, tail = results.pop(control)
        assert rc == 0, f"the unchanged copy ({control}) must pass every pin:\n{tail}"
    survivors = {n: tail for n, (rc, failed, tail) in results.items() if rc != 1 or not failed}
    assert not survivors, "planted mistakes that no pin caught: " + ", ".join(survivors)


@pytest.mark.parametrize("name", sorted(MUTATIONS) + sorted(TANGENT_MUTATIONS))
def test_mutation_text_is_present(name):
    """Each planted mistake still finds its original text (the list follows
    the oracle's source)."""
    f, old, new = {**MUTATIONS, **TANGENT_MUTATIONS}[name]
    assert open(os.path.join(ROOT, "oracle", f)).read().count(old) == 1 and old != new
