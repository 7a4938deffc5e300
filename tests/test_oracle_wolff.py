"""Pins of the oracle's Wolff single-cluster update.

* the cluster grown by breadth-first search from the seed site, testing
  each boundary bond when it is met, is exactly the seed's component of the
  full SW bond configuration of the same sweep (a second route through the
  bond randomness: per-bond tests against whole-lattice bonds + labels),
  including 2 x 2 and 3 x 3 lattices with doubled links and open chains;
* the seed site is uniform;
* beta = 0: the cluster is the seed alone; beta -> infinity on an ordered
  lattice: the whole lattice;
* statistics: the Wolff chain samples the same distribution as the SW chain
  (L = 16), and the open chain has <cos dtheta> = I1(beta)/I0(beta).
"""
import math

import numpy as np
import pytest
from scipy.special import iv

import synth
from stats import mean_err


@pytest.mark.parametrize("Lx,Ly,per", [(2, 2, 1), (3, 3, 1), (5, 4, 1), (16, 16, 1), (33, 17, 1),
                                        (24, 1, 0)])
@pytest.mark.parametrize("dtype", [np.float32, np.uint16])
def test_cluster_is_the_seed_component(orc, Lx, Ly, per, dtype):
    n = Lx * Ly
    th = synth.angles(n, seed=Lx * 31 + Ly, dtype=dtype)
    for t in range(12):
        beta = 0.4 + 0.15 * t
        inc, size = orc.wolff_cluster(th, Lx, Ly, beta, 77, t, per_x=per, per_y=per)
        r, d, _ = orc.bonds(th, Lx, Ly, beta, 77, t, per_x=per, per_y=per)
        lab, _ = orc.label_bfs(r, d, Lx, Ly, per_x=per, per_y=per)
        i0 = orc.seed_site(77, t, n)
        np.testing.assert_array_equal(inc, (lab == lab[i0]).astype(np.uint8))
        assert size == int(inc.sum()) and inc[i0] == 1


def test_seed_site_uniform(orc):
    n = 37
    sites = [orc.seed_site(5, t, n) for t in range(7400)]
    assert min(sites) >= 0 and max(sites) < n
    h = np.bincount(sites, minlength=n)
    e = len(sites) / n
    assert ((h - e) ** 2 / e).sum() < (n - 1) + 5 * math.sqrt(2 * (n - 1))


@pytest.mark.parametrize("dtype", [np.float32, np.uint16])
def test_beta_zero_flips_the_seed_only(orc, dtype):
    L = 12
    th0 = synth.angles(L * L, seed=3, dtype=dtype)
    th = th0.copy()
    obs = orc.wolff_run(th, L, L, 0.0, 9, 0, 50)
    assert np.all(obs["flipped"] == 1)
    one = th0.copy()
    orc.wolff_run(one, L, L, 0.0, 9, 0, 1)
    i0 = orc.seed_site(9, 0, L * L)
    changed = np.nonzero(one != th0)[0]
    assert set(changed) <= {i0}


def test_infinite_beta_ordered_flips_everything(orc):
    L = 10
    th = orc.init_angles(L, 4, start=1)
    obs = orc.wolff_run(th, L, L, 1e12, 4, 0, 20)
    assert np.all(obs["flipped"] == L * L)
    assert np.all(obs["energy_per_site"] == -2.0)


def test_wolff_samples_the_sw_distribution(orc):
    L, beta = 16, 1.0
    sw = orc.sw_run(orc.init_angles(L, 51, 0), L, L, beta, 51, 0, 12000)
    wo = orc.wolff_run(orc.init_angles(L, 52, 0), L, L, beta, 52, 0, 40000)
    for f in ("energy_per_site", "m2"):
        ma, ea = mean_err(sw[f][500:])
        mb, eb = mean_err(wo[f][2000:], n_bins=40)
        assert abs(ma - mb) < 4 * math.hypot(ea, eb), (f, ma, ea, mb, eb)


@pytest.mark.parametrize("beta", [1.0, 3.0])
def test_open_chain_closed_form(orc, beta):
    N, n = 48, 60000
    th = orc.init_angles(N, 600 + int(beta), start=0, Ly=1)
    obs = orc.wolff_run(th, N, 1, beta, 600 + int(beta), 0, n, per_x=0, per_y=0)
    t = iv(1, beta) / iv(0, beta)
    m, e = mean_err((obs["ex"] * N / (N - 1))[1000:], n_bins=40)
    assert abs(m - t) < 4 * e + 1e-4, (m, e, t)
