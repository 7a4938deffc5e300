"""The L = 65536 workload at full size, in the launch configuration that
bench.py times: beta = 1.1199, ordered start, tile 32 x 64, FP32 bond
thresholds.  Its state is far too large for the oracle to recompute, so one
sweep is checked on sampled sites (xy_get_sites) and through properties that
hold at any size:

* bonds: each sampled right/down bond is the oracle's FP64 rule on the
  ordered start, up to the FP32 evaluation band;
* labels: a label is the minimum index of its cluster (label <= site, and
  the label of a label is itself), and an active bond joins equal labels;
* flip: every angle is 0 or C32, as the oracle's coin of the site's label says;
* observables: the angle field takes the two values 0 and C32, so with f the
  reflected fraction mx = 1 - f (1 - cos C32) and my = f sin C32.
"""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1210_6116_b300 as xy  # noqa: E402
from paper_1210_6116_b300 import build as xybuild  # noqa: E402

xybuild.build()


def test_l65536_one_sweep_sampled(orc):
    L, beta, seed = 65536, 1.1199, 2
    N = L * L
    cfg = xy.xy_config(L=L, tile_y=64, seed=seed, beta=beta, angle_dtype=xy.XY_F32,
                       threshold_mode=xy.XY_THR_F32, start=1, record_cap=0)
    free, _ = torch.cuda.mem_get_info()
    if xy.xy_workspace_size(cfg) > 0.9 * free:
        pytest.skip("not enough device memory for L = 65536")
    lat = xy.Lattice(L, beta, seed, start="ordered", tile_y=64, exact=False)
    try:
        lat.sweep(1)
        rec = lat.measure()
        rng = np.random.default_rng(65536)
        i = np.unique(rng.integers(0, N, size=20000, dtype=np.uint64))
        x, y = i % L, i // L
        th, lab, bd = lat.get_sites(i)
        _, lab_r, _ = lat.get_sites(y * L + (x + 1) % L)
        _, lab_d, _ = lat.get_sites(((y + 1) % L) * L + x)
        _, lab_root, _ = lat.get_sites(lab.astype(np.uint64))
    finally:
        lat.close()
    # labels
    assert np.all(lab <= i) and np.array_equal(lab_root, lab)
    right, down = (bd & 1) == 1, (bd & 2) == 2
    assert np.array_equal(lab_r[right], lab[right]) and np.array_equal(lab_d[down], lab[down])
    assert right.any() and down.any() and not right.all()
    # bonds against the FP64 rule on the ordered start (theta = 0 everywhere;
    # the zero array is allocated lazily, only the sampled pages are read)
    zeros = np.zeros(N, np.float32)
    eps = 4 * (2 * beta * 2e-6 + 3e-7) + 2.0 ** -24
    for k in range(3000):
        for direction, got in ((0, right[k]), (1, down[k])):
            u, p = orc.bond_up(zeros, L, L, beta, seed, 0, int(i[k]), direction)
            if got != (u < p):
                assert abs(u - p) <= eps, (int(i[k]), direction, u, p)
    # flips: each angle is 0 or C32 by the coin of its label
    c32 = orc.axis(seed, 0)[4]
    coins = np.array([orc.coin(seed, 0, int(v), L) for v in lab[:5000]])
    np.testing.assert_array_equal(th[:5000], np.where(coins == 1, c32, np.float32(0.0)))
    # observables of a two-valued field
    r = rec[0]
    f = r["my"] / math.sin(float(c32))
    assert -1e-6 <= f <= 1 + 1e-6
    assert abs(r["mx"] - (1 - f * (1 - math.cos(float(c32))))) < 1e-6
    assert abs(r["m2"] - (r["mx"] ** 2 + r["my"] ** 2)) < 1e-12
