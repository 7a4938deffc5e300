"""Restricted oracle computations used by the full-size (L = 65536) checks,
against the whole-lattice oracle on small lattices: bonds of selected rows
from those rows' angles only, and observables summed over bands of rows."""
import numpy as np
import pytest

import synth
from gpu_helpers import banded_measure


@pytest.mark.parametrize("y0,nrows", [(0, 2), (10, 5), (62, 2), (63, 1)])
def test_row_bonds_equal_whole_lattice_bonds(orc, y0, nrows):
    L, beta, seed, t = 64, 1.12, 9, 3
    th = synth.angles(L * L, seed=5)
    right, down, _ = orc.bonds(th, L, L, beta, seed, t)
    rows = np.concatenate([th.reshape(L, L)[(y0 + k) % L] for k in range(nrows + 1)])
    r, d, gr, gd = orc.bonds_rows(rows, L, y0, nrows, beta, seed, t)
    idx = np.concatenate([((y0 + k) % L) * L + np.arange(L) for k in range(nrows)])
    np.testing.assert_array_equal(r, right[idx])
    np.testing.assert_array_equal(d, down[idx])
    # u - p agrees with the single-bond oracle call
    for k in (0, 5, L + 3):
        if k < nrows * L:
            i = int(idx[k])
            for direction, gap in ((0, gr), (1, gd)):
                u, p = orc.bond_up(th, L, L, beta, seed, t, i, direction)
                assert gap[k] == u - p


@pytest.mark.parametrize("band", [7, 16, 64])
def test_banded_observables_equal_whole_lattice(orc, band):
    L, beta = 64, 1.1
    th = synth.angles(L * L, seed=77)
    want = orc.measure(th, L, L, beta)
    got = banded_measure(orc, th, L, beta, band=band)
    for f in ("energy_per_site", "mx", "my", "m2", "ex", "sx", "ey", "sy", "upsilon",
              "l1_mx", "l1_sx", "l1_ex"):
        assert got[f] == pytest.approx(want[f], rel=1e-12, abs=1e-15), f
