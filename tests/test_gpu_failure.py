"""Failure detection on the GPU without a fault: the device-side loop bound.

Every global find, union and pointer-jumping loop of the labeling kernels
stops after a bounded number of iterations, records an error bit in the
lattice's device state and lets its launch finish; the next synchronising
call returns XY_ETIMEOUT and clears the bit.  A valid lattice never comes
near the default bound (2^22), so the tests lower it to one iteration
(xy_set_loop_bound), which makes it run out on any cluster that crosses
tiles more than once, and then check that the same handle labels and sweeps
exactly like the oracle once the default is restored.  Nothing here faults,
traps or hangs a GPU: the bound is what ends every loop.
"""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1210_6116_b300 as xy  # noqa: E402
from paper_1210_6116_b300 import build as xybuild  # noqa: E402

xybuild.build()


def test_loaded_device_code_is_sm_103():
    assert xy.xy_build_arch() == 103


@pytest.mark.parametrize("masks", ["spiral", "dense"])
def test_label_loop_bound_runs_out_then_recovers(orc, masks):
    L = 129
    if masks == "spiral":
        r, d = synth.spiral_masks(L)
    else:
        r, d = synth.bond_masks(L, L, 0.7, seed=4711)
    want = orc.label_bfs(r, d, L, L)[0]
    lat = xy.Lattice(L, 1.0, 1, tile_y=32)
    try:
        lat.set_loop_bound(1)
        with pytest.raises(xy.XyError) as e:
            lat.label_bonds(r, d)
        assert e.value.status == xy.XY_ETIMEOUT
        assert "bound" in xy.xy_last_error()
        lat.set_loop_bound(0)
        np.testing.assert_array_equal(lat.label_bonds(r, d), want)
    finally:
        lat.close()


def test_sweep_loop_bound_runs_out_then_recovers(orc):
    """A sweep whose labeling hit the bound is reported by xy_measure(sync=1);
    with the default bound restored, the next sweep from known angles is the
    oracle's sweep bit for bit."""
    # an ordered field at beta = 2 whose sweep-0 axis is nearly parallel to
    # it (seed 33: |cos phi| = 0.96) bonds ~97 % of the links into one
    # cluster that crosses every tile edge
    L, beta, seed = 96, 2.0, 33
    th0 = synth.ordered_angles(L * L)
    r, d, _ = orc.bonds(th0, L, L, beta, seed, 0)
    assert len(np.unique(orc.label_bfs(r, d, L, L)[0])) == 1
    lat = xy.Lattice(L, beta, seed, tile_y=32)
    try:
        lat.set_angles(th0)
        lat.set_loop_bound(1)
        lat.sweep(1)
        with pytest.raises(xy.XyError) as e:
            lat.measure()
        assert e.value.status == xy.XY_ETIMEOUT
        lat.set_loop_bound(0)
        lat.measure()  # the error was reported once: this call succeeds
        lat.set_angles(th0)
        lat.sweep(1)
        rec = lat.measure()
        th = th0.copy()
        orc.sw_run(th, L, L, beta, seed, 1, 1)  # the lattice is at sweep 1
        np.testing.assert_array_equal(lat.get_angles(), th)
        assert len(rec) == 1 and int(rec[0]["sweep"]) == 1
    finally:
        lat.close()


def test_link_capacity_overflow_is_internal_error_then_recovers(orc):
    """With one link slot per tile, a dense mask's merge overflows the link
    list: the consistency error reaches the host as XY_EINTERNAL, and with
    the default capacity restored the same handle labels exactly."""
    L = 129
    r, d = synth.bond_masks(L, L, 0.7, seed=4712)
    want = orc.label_bfs(r, d, L, L)[0]
    lat = xy.Lattice(L, 1.0, 1, tile_y=32)
    try:
        lat.set_link_cap(1)
        with pytest.raises(xy.XyError) as e:
            lat.label_bonds(r, d)
        assert e.value.status == xy.XY_EINTERNAL
        lat.set_link_cap(0)
        np.testing.assert_array_equal(lat.label_bonds(r, d), want)
    finally:
        lat.close()
