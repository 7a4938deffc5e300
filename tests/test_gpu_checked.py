"""The bounds-checked build (libxy_checked.so, -DXY_BOUNDS_CHECK): every
global index that comes from data is tested on the device.  Run in a child
process (the binding picks the library by XY_BOUNDS_CHECK=1 when it is first
loaded), it must give the oracle's results bit for bit and report no error:
a sweep chain with FP64 thresholds, labels of random and spiral masks, and an
engine of two lattices."""
import os
import subprocess
import sys
from pathlib import Path

import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

ROOT = Path(__file__).resolve().parent.parent

CHILD = r"""
import sys
import numpy as np
sys.path.insert(0, "tests")
import oracle as orc, synth
import paper_1210_6116_b300 as xy
assert xy.load_library()._name.endswith("libxy_checked.so")
L, beta, seed = 96, 1.12, 5
lat = xy.Lattice(L, beta, seed, tile_y=32)
th = orc.init_angles(L, seed, 0)
lat.sweep(30)
lat.measure()                      # sync = 1: raises on any device error
orc.sw_run(th, L, L, beta, seed, 0, 30, record=False)
assert np.array_equal(lat.get_angles(), th)
for Lm, (r, d) in ((100, synth.bond_masks(100, 100, 0.6, seed=3)), (129, synth.spiral_masks(129))):
    m = xy.Lattice(Lm, 1.0, 1, tile_y=32)
    assert np.array_equal(m.label_bonds(r, d), orc.label_bfs(r, d, Lm, Lm)[0])
eng = xy.Engine(2, exact=True, tile_y=32)
s0 = eng.admit(eng.config(64, 1.1, 7))
eng.admit(eng.config(128, 1.2, 8, update="wolff"))
eng.step(20)
assert len(eng.measure(s0)) == 20
th = orc.init_angles(64, 7, 0)
orc.sw_run(th, 64, 64, 1.1, 7, 0, 20, record=False)
assert np.array_equal(eng.get_angles(s0), th)
print("checked build ok")
"""


def test_bounds_checked_build_matches_oracle_without_errors():
    from paper_1210_6116_b300 import build as xybuild

    xybuild.build(checked=True)
    env = dict(os.environ, XY_BOUNDS_CHECK="1")
    res = subprocess.run([sys.executable, "-c", CHILD], cwd=ROOT, env=env,
                         capture_output=True, text=True, timeout=600)
    assert res.returncode == 0, res.stdout[-2000:] + res.stderr[-4000:]
    assert "checked build ok" in res.stdout
