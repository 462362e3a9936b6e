"""Index checks of the debug build (the stand-in for a device memory checker,
which this pool does not offer): every kernel path runs on small inputs with
WHG_DEBUG_BOUNDS compiled in, and no check may fail."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_debug_build_index_checks_stay_clear():
    from paper_2307_05683_gb300 import build
    lib = build.build(debug=True)
    env = dict(os.environ, WHG_LIBRARY=lib, PYTHONPATH=ROOT)
    r = subprocess.run([sys.executable, os.path.join(ROOT, "tests", "_bounds_scenario.py")], cwd=ROOT, env=env,
                       capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-3000:]
    flags = json.loads(r.stdout.strip().splitlines()[-1])
    assert len(flags) == 5 and all(v == 0 for v in flags.values()), flags


def test_release_build_reports_no_index_checks():
    from paper_2307_05683_gb300 import build, inputs, whg
    build.build()
    it = whg.Integrator(8, 8)
    it.init(inputs.solar_ensemble(1, 8))
    with pytest.raises(whg.WhgError) as e:
        whg.whg_debug_bounds(it.ctx)
    assert e.value.code == whg.WHG_EINVAL
    it.close()
    with pytest.raises(whg.WhgError) as e:
        whg.whg_noalloc_debug_bounds()
    assert e.value.code == whg.WHG_EINVAL
