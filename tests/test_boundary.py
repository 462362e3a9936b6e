"""The C ABI: include/whg.h declarations, the built library's exports, and the
Python binding's names.  CPU only (no CUDA calls are made)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "whg.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(whg_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib_path():
    from paper_2307_05683_gb300 import build
    return build.build()


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ["whg_create", "whg_init", "whg_step", "whg_read_state", "whg_energy",
              "whg_get_raw", "whg_set_raw", "whg_last_error", "whg_destroy"]:
        assert n in names


def test_library_exports_every_declared_symbol(lib_path):
    out = subprocess.check_output(["nm", "-D", "--defined-only", lib_path], text=True)
    exported = set(re.findall(r"\bT (whg_[a-z0-9_]+)", out))
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, missing
    lib = ctypes.CDLL(lib_path)
    for n in declared_functions():
        assert getattr(lib, n) is not None


def test_binding_covers_the_header(lib_path):
    from paper_2307_05683_gb300 import whg
    assert sorted(whg.exported_symbols()) == declared_functions()
    for n in declared_functions():
        assert callable(getattr(whg, n))


def test_library_is_built_for_sm_103a(lib_path):
    from paper_2307_05683_gb300 import build
    assert "arch=compute_103a,code=sm_103a" in " ".join(build.NVCC_FLAGS)


def test_options_struct_layout(lib_path):
    from paper_2307_05683_gb300 import whg
    o = whg.whg_default_options()          # pure host function, no CUDA call
    assert o.gr_mode == 1 and o.newton_terms == 8
    assert o.c_light == pytest.approx(10065.32, rel=1e-5)
    assert o.close_encounter_hill == 0.0 and o.eject_factor == 0.0
    assert o.graph_launches == 0 and o.merge_jumps == 0 and o.halley_fp32 == 0
    assert ctypes.sizeof(whg.whg_options) == 80
    # the library writes the last field: the C struct reaches as far as the ctypes one
    s = whg.whg_options()
    s.halley_fp32 = 12345
    s.repack_frozen = 6789
    s.interaction_schedule = 4321
    s.queue_steps = 8765
    whg.load().whg_default_options(ctypes.byref(s))
    assert s.halley_fp32 == 0 and s.repack_frozen == -1 and s.interaction_schedule == 0
    assert s.queue_steps == 100


@pytest.mark.parametrize("field,value", [("gr_mode", 3), ("newton_terms", 7), ("lanes_per_system", 9),
                                         ("block_size", 48), ("steps_per_launch", -1),
                                         ("graph_launches", 5000), ("repack_frozen", 2),
                                         ("repack_frozen", -2),
                                         ("interaction_schedule", 2), ("queue_steps", -1),
                                         ("queue_steps", 10001), ("close_encounter_hill", -1.0),
                                         ("eject_factor", float("inf"))])
def test_create_rejects_bad_options(lib_path, field, value):
    """whg_create checks its options before any CUDA call: a bad value gives
    WHG_EINVAL, no context, and a message naming the option."""
    from paper_2307_05683_gb300 import whg
    lib = whg.load()
    o = whg.whg_default_options()
    setattr(o, field, value)
    h = ctypes.c_void_p(1)
    rc = lib.whg_create(ctypes.byref(h), 16, 8, ctypes.byref(o), None)
    assert rc == whg.WHG_EINVAL and not h.value
    msg = lib.whg_last_error(None).decode()
    key = {"close_encounter_hill": "stop rules", "eject_factor": "stop rules"}.get(field, field)
    assert key in msg, msg


def test_create_rejects_bad_sizes(lib_path):
    from paper_2307_05683_gb300 import whg
    lib = whg.load()
    h = ctypes.c_void_p()
    assert lib.whg_create(ctypes.byref(h), 0, 8, None, None) == whg.WHG_EINVAL
    assert lib.whg_create(ctypes.byref(h), 4, 9, None, None) == whg.WHG_EINVAL
    assert lib.whg_create(None, 4, 8, None, None) == whg.WHG_EINVAL


def _functions_importing(path, module):
    """Names of the top-level functions of a Python file that import `module`
    (None for an import at module level)."""
    import ast
    found = set()
    for top in ast.parse(open(path).read()).body:
        owner = top.name if isinstance(top, (ast.FunctionDef, ast.AsyncFunctionDef)) else None
        for node in ast.walk(top):
            if isinstance(node, ast.Import) and any(a.name.split(".")[0] == module for a in node.names):
                found.add(owner)
            if isinstance(node, ast.ImportFrom) and (node.module or "").split(".")[0] == module:
                found.add(owner)
    return found


def test_product_path_never_reaches_the_oracle():
    """The package and its CUDA sources neither import, include nor name the
    oracle; bench.py imports it only in its CPU-baseline and reference legs,
    __graft_entry__ only to build it and in smoke()."""
    pkg = os.path.join(ROOT, "paper_2307_05683_gb300")
    for dirpath, _, files in os.walk(pkg):
        if "_build" in dirpath:
            continue
        for f in files:
            if f.endswith(".py"):
                assert not _functions_importing(os.path.join(dirpath, f), "oracle"), f
            if f.endswith((".cu", ".cuh", ".h", ".py")):
                text = open(os.path.join(dirpath, f)).read()
                assert not re.search(r"\borc_[a-z]|liborc|#include\s+\"[^\"]*orc", text), f
    assert _functions_importing(os.path.join(ROOT, "bench.py"), "oracle") == {"oracle_rate", "run_reference"}
    assert _functions_importing(os.path.join(ROOT, "__graft_entry__.py"), "oracle") == {"build", "smoke"}
    # the one call of the oracle's timing in the GPU arm fills only cpu_baseline
    lines = open(os.path.join(ROOT, "bench.py")).read().splitlines()
    calls = [k for k, ln in enumerate(lines) if "oracle_rate(" in ln and not ln.startswith("def ")]
    assert len(calls) == 1 and lines[calls[0] + 1].strip().startswith('line["cpu_baseline"]')


def test_missing_library_fails_loudly(tmp_path):
    """With no libwhg.so at the configured path every call raises (there is
    no CPU fallback)."""
    code = ("from paper_2307_05683_gb300 import whg\n"
            "for call in (whg.whg_default_options, lambda: whg.Integrator(4, 2)):\n"
            "    try:\n"
            "        call()\n"
            "    except RuntimeError as e:\n"
            "        assert 'no CPU fallback' in str(e), e\n"
            "    else:\n"
            "        raise SystemExit('a call succeeded without the library')\n"
            "print('ok')\n")
    env = dict(os.environ, WHG_LIBRARY=str(tmp_path / "absent" / "libwhg.so"))
    r = subprocess.run([os.sys.executable, "-c", code], cwd=ROOT, env=env, capture_output=True, text=True,
                       timeout=300)
    assert r.returncode == 0 and r.stdout.strip() == "ok", r.stdout + r.stderr
