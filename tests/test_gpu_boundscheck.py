"""GPU: the bounds-checked build of the library (kernels compiled with
-DATLASGB_BOUNDSCHECK, every table index checked against the launch's
buffers) against the FP64 oracle on O2 and O4.

The build is made here (build.build(boundscheck=True)) and loaded in a child
process with ATLASGB_BOUNDSCHECK=1 (tests/boundscheck_child.py), which runs
every kind of launch -- per-node and node-group kernels for every operator,
the edge-based forms, a batch, band partitions, a remap -- and compares each
with the oracle.  No call may report a bounds violation (ATLAS_EBOUNDS) and
the results must meet the parity tolerances.  No out-of-range index is ever
planted on the GPU: a corrupted table is refused on the host before any
launch (test_geometry_cache.py).
"""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


def test_bounds_checked_build_matches_oracle_on_o2_o4():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1908_07038_gb300 import build
    lib = build.build(boundscheck=True)
    assert os.path.exists(lib)
    env = dict(os.environ, ATLASGB_BOUNDSCHECK="1",
               PYTHONPATH=os.pathsep.join([ROOT, HERE, os.environ.get("PYTHONPATH", "")]))
    r = subprocess.run([sys.executable, os.path.join(HERE, "boundscheck_child.py")], cwd=ROOT, env=env,
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    out = json.loads(r.stdout.strip().splitlines()[-1])
    assert "bounds-checked" in out["info"], out["info"]
    assert out["status"] == 0
    assert out["cases"] >= 100, out
    assert out["worst"]["f64"] <= 1e-13 and out["worst"]["f32"] <= 1e-5, out
