"""Wolff single-cluster updates on the GPU against the oracle, which grows
each cluster by a breadth-first search from the seed site: bonds, labels,
the reflected cluster and its size, angles bit for bit, observables within
the tolerance of gpu_helpers; engine batches that mix SW and Wolff
lattices; <m^2> at beta_KT(64) against Table 1."""
import math

import numpy as np
import pytest

import synth
from gpu_helpers import band_mismatches, obs_close, rec_dict

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1210_6116_b300 as xy  # noqa: E402
from paper_1210_6116_b300 import build as xybuild  # noqa: E402

xybuild.build()
NP = {"f32": np.float32, "f16": np.float16, "u16": np.uint16}


def _lat(L, beta, seed, **kw):
    return xy.Lattice(L, beta, seed, update="wolff", **kw)


@pytest.mark.parametrize("L,ty", [(2, 16), (3, 16), (33, 16), (64, 32), (130, 64)])
@pytest.mark.parametrize("beta", [0.0, 1.1, 3.0])
@pytest.mark.parametrize("dtype", ["f32", "u16"])
def test_single_update_steps(orc, L, ty, beta, dtype):
    seed = 500 + L
    th0 = synth.angles(L * L, seed=L * 3 + 1, dtype=NP[dtype])
    lat = _lat(L, beta, seed, tile_y=ty, dtype=dtype)
    lat.set_angles(th0)
    lat.sweep(1)
    rec = lat.measure()
    g_r, g_d = lat.get_bonds()
    o_r, o_d, _ = orc.bonds(th0, L, L, beta, seed, 0)
    inside, outside = band_mismatches(orc, th0, L, beta, seed, 0, g_r, g_d, o_r, o_d)
    assert not outside and not inside
    inc, size = orc.wolff_cluster(th0, L, L, beta, seed, 0)
    g_lab = lat.get_labels()
    i0 = orc.seed_site(seed, 0, L * L)
    np.testing.assert_array_equal((g_lab == g_lab[i0]).astype(np.uint8), inc)
    th = th0.copy()
    o = orc.wolff_run(th, L, L, beta, seed, 0, 1)
    np.testing.assert_array_equal(lat.get_angles().view(np.uint8), th.view(np.uint8))
    assert int(rec[0]["flipped"]) == size
    od = {n: float(o[0][n]) for n in o.dtype.names}
    bad = obs_close(rec_dict(rec[0]), od, L * L, beta, flips=True)
    assert not bad, bad


@pytest.mark.parametrize("L,ty,dtype", [(64, 32, "f32"), (100, 32, "f32"), (64, 64, "u16"),
                                        (48, 16, "f16")])
def test_chain_bit_exact(orc, L, ty, dtype):
    """400 updates from the random start (exact mode)."""
    beta, seed, n = 1.1, 71 + L, 400
    lat = _lat(L, beta, seed, tile_y=ty, dtype=dtype)
    th = orc.init_angles(L, seed, 0, dtype=NP[dtype])
    lat.sweep(n)
    recs = lat.measure()
    o = orc.wolff_run(th, L, L, beta, seed, 0, n)
    np.testing.assert_array_equal(lat.get_angles().view(np.uint8), th.view(np.uint8))
    for k in range(n):
        od = {f: float(o[k][f]) for f in o.dtype.names}
        bad = obs_close(rec_dict(recs[k]), od, L * L, beta, flips=True)
        assert not bad, (k, bad)


def test_beta_zero_reflects_one_site():
    lat = _lat(64, 0.0, 5)
    lat.sweep(40)
    assert np.all(lat.measure()["flipped"] == 1)


def test_engine_mixes_sw_and_wolff():
    table = synth.replica_table(8, seed=13, sizes=(64, 128, 256), beta_range=(1.0, 1.2))
    eng = xy.Engine(len(table), tile_y=32, exact=True)
    upd = ["wolff" if k % 2 else "sw" for k in range(len(table))]
    pcc = xy.xy_pcc_params(target=0.636508, dbeta0=0.001, halve_every=0, block=5)
    slots = [eng.admit(eng.config(r["L"], r["beta"], r["seed"], update=u), pcc if k < 4 else None)
             for k, (r, u) in enumerate(zip(table, upd))]
    eng.step(30)
    for k, (r, s, u) in enumerate(zip(table, slots, upd)):
        lat = xy.Lattice(r["L"], r["beta"], r["seed"], tile_y=32, exact=True, update=u)
        if k < 4:
            lat.pcc_step(30, target=0.636508, dbeta0=0.001, halve_every=0, block=5)
        else:
            lat.sweep(30)
        np.testing.assert_array_equal(eng.measure(s), lat.measure())
        np.testing.assert_array_equal(eng.get_angles(s), lat.get_angles())


def test_table1_m2_at_beta_kt_64():
    """Wolff updates at beta_KT(64) = 1.09167 reproduce <m^2>_64 = 0.34924(29)
    (16 replicas; the error is the replica spread)."""
    L, reps, beta = 64, 16, 1.09167
    eng = xy.Engine(reps, tile_y=32)
    slots = [eng.admit(eng.config(L, beta, 9100 + k, update="wolff", record_cap=20000))
             for k in range(reps)]
    eng.step(2000)
    for s in slots:
        eng.measure(s)
    eng.step(20000)
    m2 = np.array([eng.measure(s)["m2"].mean() for s in slots])
    err = m2.std(ddof=1) / math.sqrt(reps)
    assert abs(m2.mean() - 0.34924) < 4 * math.hypot(err, 0.00029), (m2.mean(), err)
