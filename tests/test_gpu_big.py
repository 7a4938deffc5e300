"""The L = 65536 workload at full size (the paper's largest lattice, Table 1),
in the launch configuration that bench.py times: beta = 1.1199, ordered
start, tile 32 x 64, FP32 bond thresholds.

test_l65536_thermalised_sweep: after 200 sweeps (equilibrium clusters), one
more sweep is checked against the oracle:
* observables: the whole post-sweep configuration (16 GiB of angles) is
  copied to the host and the oracle's sums are taken over bands of rows
  (gpu_helpers.banded_measure); every field of the sweep's record must agree
  within the A19 tolerances of gpu_helpers;
* bonds: 64 full rows (32 pairs of rows) are recomputed by the oracle's FP64
  rule from the pre-sweep angles of those rows (orc.bonds_rows); a bit may
  differ only inside the FP32 evaluation band |u - p| <= eps;
* flip: those rows' new angles are the oracle's reflection of their old
  angles by the coin of each site's label;
* labels: on those rows, bonded neighbours share a label, a label is at most
  its site index, and the label of a label is itself.

test_l65536_one_sweep_sampled checks the first sweep from the ordered start
on sampled sites and through properties that hold at any size:

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

from gpu_helpers import banded_measure, obs_close, rec_dict

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


def _host_available_bytes() -> int:
    with open("/proc/meminfo") as f:
        for line in f:
            if line.startswith("MemAvailable:"):
                return int(line.split()[1]) * 1024
    return 0


def test_l65536_thermalised_sweep(orc):
    L, beta, seed, t_check = 65536, 1.1199, 2, 200
    N = L * L
    cfg = xy.xy_config(L=L, tile_y=64, seed=seed, beta=beta, angle_dtype=xy.XY_F32,
                       threshold_mode=xy.XY_THR_F32, start=1, record_cap=0)
    free, _ = torch.cuda.mem_get_info()
    if xy.xy_workspace_size(cfg) > 0.9 * free:
        pytest.skip("not enough device memory for L = 65536")
    if _host_available_bytes() < 40e9:
        pytest.skip("the host needs ~40 GB free for the full-lattice check")
    rng = np.random.default_rng(200)
    y_pairs = np.sort(rng.choice(L // 2, size=32, replace=False)) * 2  # rows y, y + 1
    x = np.arange(L, dtype=np.uint64)
    rows3 = [np.concatenate([((y + k) % L) * L + x for k in range(3)]).astype(np.uint64)
             for y in y_pairs]
    lat = xy.Lattice(L, beta, seed, start="ordered", tile_y=64, exact=False)
    try:
        lat.sweep(t_check)
        lat.measure(max_records=0)
        before = [lat.get_sites(i)[0] for i in rows3]  # angles of rows y, y+1, y+2
        lat.sweep(1)  # sweep t_check
        rec = lat.measure()
        assert len(rec) == 1 and int(rec[0]["sweep"]) == t_check
        after = [lat.get_sites(i[: 2 * L]) for i in rows3]
        roots = np.unique(np.concatenate([a[1] for a in after])).astype(np.uint64)
        _, root_of_root, _ = lat.get_sites(roots)
        theta = lat.get_angles()
    finally:
        lat.close()
    # observables of the whole configuration
    o = banded_measure(orc, theta, L, beta)
    del theta
    bad = obs_close(rec_dict(rec[0]), o, N, beta)
    assert not bad, bad
    assert abs(rec[0]["energy_per_site"] + 1.45) < 0.05  # equilibrium near T_KT
    # bonds, flip and labels of the sampled rows
    eps = 4 * (2 * beta * 2e-6 + 3e-7) + 2.0 ** -24
    c32 = orc.axis(seed, t_check)[4]
    np.testing.assert_array_equal(root_of_root, roots)
    n_diff = 0
    col = np.arange(2 * L)
    for y, th3, (th_new, lab, bd) in zip(y_pairs, before, after):
        r_o, d_o, gap_r, gap_d = orc.bonds_rows(th3, L, int(y), 2, beta, seed, t_check)
        r_g, d_g = (bd & 1).astype(np.uint8), ((bd >> 1) & 1).astype(np.uint8)
        for g, o_, gap in ((r_g, r_o, gap_r), (d_g, d_o, gap_d)):
            diff = np.nonzero(g != o_)[0]
            assert np.all(np.abs(gap[diff]) <= eps), (int(y), diff[:5], gap[diff][:5])
            n_diff += diff.size
        flip = th3[: 2 * L].copy()
        orc.flip(flip, lab, L, 2, seed, t_check, c32)
        np.testing.assert_array_equal(th_new, flip)
        sites = int(y) * L + col.astype(np.uint64)
        assert np.all(lab <= sites)
        right = r_g == 1
        nxt = (col // L) * L + (col + 1) % L
        np.testing.assert_array_equal(lab[nxt[right]], lab[right])
        down = d_g[:L] == 1
        np.testing.assert_array_equal(lab[L:][down], lab[:L][down])
    assert n_diff <= 64, n_diff  # FP32 thresholds differ on ~1e-7 of the bonds
