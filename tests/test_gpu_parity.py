"""GPU parity: the CUDA sweep (through the C ABI) against the CPU oracle.

Exact mode (FP64 thresholds) must reproduce the oracle bit for bit in bond
masks (except bonds with |u - p| < 1e-12, counted and reported), labels,
flip sets and angles; observables agree within the tolerances derived in
gpu_helpers.  Sizes span several tiles with ragged right and bottom tiles.
"""
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


def _lat(L, beta, seed, **kw):
    return xy.Lattice(L, beta, seed, **kw)


# ------------------------------------------------------------- initial angles
@pytest.mark.parametrize("L", [64, 100, 4096])
def test_random_start_bit_exact(orc, L):
    lat = _lat(L, 1.0, 12345, start="random")
    np.testing.assert_array_equal(lat.get_angles(), orc.init_angles(L, 12345, 0))
    lat16 = _lat(L, 1.0, 12345, start="random", dtype="f16")
    np.testing.assert_array_equal(lat16.get_angles().view(np.uint16),
                                  orc.init_angles(L, 12345, 0, dtype=np.float16).view(np.uint16))
    lat0 = _lat(L, 1.0, 7, start="ordered")
    assert not lat0.get_angles().any()
    lat_q = _lat(L, 1.0, 12345, start="random", dtype="u16")
    np.testing.assert_array_equal(lat_q.get_angles(), orc.init_angles(L, 12345, 0, dtype=np.uint16))


# ---------------------------------------------------- one sweep, step by step
GEOMS = [(2, 16), (3, 16), (5, 16), (17, 16), (32, 32), (33, 16), (64, 0), (64, 16),
         (100, 32), (130, 64), (256, 128), (257, 64)]


@pytest.mark.parametrize("L,ty", GEOMS)
@pytest.mark.parametrize("beta", [0.0, 0.6, 1.12, 3.0])
def test_single_sweep_steps(orc, L, ty, beta):
    seed = 1000 + L
    th0 = synth.angles(L * L, seed=L * 7 + 1)
    lat = _lat(L, beta, seed, tile_y=ty)
    lat.set_angles(th0)
    lat.sweep(1)
    rec = lat.measure()
    assert len(rec) == 1 and int(rec[0]["sweep"]) == 0
    g_r, g_d = lat.get_bonds()
    o_r, o_d, _ = orc.bonds(th0, L, L, beta, seed, 0)
    inside, outside = band_mismatches(orc, th0, L, beta, seed, 0, g_r, g_d, o_r, o_d)
    assert not outside, outside[:5]
    assert len(inside) == 0  # none expected at these sizes; reported if ever nonzero
    # labels of the GPU's own bonds
    g_lab = lat.get_labels()
    o_lab, _ = orc.label_bfs(g_r, g_d, L, L)
    np.testing.assert_array_equal(g_lab, o_lab)
    # flip of the oracle on the same labels
    th = th0.copy()
    phi, c, s, C64, C32 = orc.axis(seed, 0)
    orc.flip(th, g_lab, L, L, seed, 0, C32)
    np.testing.assert_array_equal(lat.get_angles(), th)
    # observables of the new configuration
    o = orc.measure(th, L, L, beta)
    bad = obs_close(rec_dict(rec[0]), o, L * L, beta)
    assert not bad, bad


# ------------------------------------------------- u16 fixed-point angles
@pytest.mark.parametrize("L,ty", [(3, 16), (33, 16), (64, 32), (130, 64), (257, 128)])
@pytest.mark.parametrize("beta", [0.0, 1.12, 3.0])
def test_u16_single_sweep_steps(orc, L, ty, beta):
    """u16 angles: bonds on the grid axis (exact mode), labels, the integer
    flip bit for bit, observables within tolerance."""
    seed = 2000 + L
    q0 = synth.angles(L * L, seed=L * 5 + 3, dtype=np.uint16)
    lat = _lat(L, beta, seed, tile_y=ty, dtype="u16")
    lat.set_angles(q0)
    lat.sweep(1)
    rec = lat.measure()
    g_r, g_d = lat.get_bonds()
    o_r, o_d, _ = orc.bonds(q0, L, L, beta, seed, 0)
    inside, outside = band_mismatches(orc, q0, L, beta, seed, 0, g_r, g_d, o_r, o_d)
    assert not outside, outside[:5]
    assert len(inside) == 0
    g_lab = lat.get_labels()
    np.testing.assert_array_equal(g_lab, orc.label_bfs(g_r, g_d, L, L)[0])
    q = q0.copy()
    orc.flip(q, g_lab, L, L, seed, 0, orc.axis_u16(seed, 0)[4])
    np.testing.assert_array_equal(lat.get_angles(), q)
    bad = obs_close(rec_dict(rec[0]), orc.measure(q, L, L, beta), L * L, beta)
    assert not bad, bad


@pytest.mark.parametrize("exact,geoms,n", [(True, ((64, 32), (96, 64)), 300),
                                           (False, ((64, 32),), 30)])
def test_u16_chain_bit_exact(orc, exact, geoms, n):
    """Chains from the random start: angles bit-exact and every record within
    tolerance.  Exact mode: 300 sweeps at L = 64 and L = 96 (ragged tile
    rows).  FP32 thresholds: 30 sweeps at L = 64, where the expected number
    of bonds that FP32 decides differently from FP64 (~8e-8 per bond) is
    0.02."""
    for L, ty in geoms:
        beta, seed = 1.12, 31 + L
        lat = _lat(L, beta, seed, tile_y=ty, dtype="u16", exact=exact)
        q = orc.init_angles(L, seed, 0, dtype=np.uint16)
        lat.sweep(n)
        recs = lat.measure()
        o = orc.sw_run(q, L, L, beta, seed, 0, n)
        np.testing.assert_array_equal(lat.get_angles(), q)
        for k in range(n):
            od = {n: float(o[k][n]) for n in o.dtype.names}
            assert not obs_close(rec_dict(recs[k]), od, L * L, beta), (L, k)


def test_u16_bench_size_one_sweep(orc):
    """L = 4096, tile 64, one u16 sweep from the random start."""
    L, beta, seed = 4096, 1.12, 1003
    lat = _lat(L, beta, seed, tile_y=64, dtype="u16", measure_xi=True)
    q0 = orc.init_angles(L, seed, 0, dtype=np.uint16)
    lat.sweep(1)
    rec = lat.measure()
    g_r, g_d = lat.get_bonds()
    o_r, o_d, band = orc.bonds(q0, L, L, beta, seed, 0)
    assert int((g_r != o_r).sum() + (g_d != o_d).sum()) <= band
    g_lab = lat.get_labels()
    np.testing.assert_array_equal(g_lab, orc.label_bfs(g_r, g_d, L, L)[0])
    q = q0.copy()
    orc.flip(q, g_lab, L, L, seed, 0, orc.axis_u16(seed, 0)[4])
    np.testing.assert_array_equal(lat.get_angles(), q)
    assert not obs_close(rec_dict(rec[0]), orc.measure(q, L, L, beta), L * L, beta, xi=True)


# ------------------------------------------------------------ whole chains
def test_config0_chain_1000_sweeps(orc):
    """L = 64, FP32 angles from seed 1 (Philox INIT), beta = 1.12, 1000 sweeps:
    angles bit-exact after every 100 sweeps, every observable record within
    tolerance."""
    L, beta, seed = 64, 1.12, 1
    lat = _lat(L, beta, seed)
    th = orc.init_angles(L, seed, 0)
    for block in range(10):
        lat.sweep(100)
        recs = lat.measure()
        o = orc.sw_run(th, L, L, beta, seed, block * 100, 100)
        np.testing.assert_array_equal(lat.get_angles(), th)
        assert np.array_equal(recs["sweep"], np.arange(block * 100, block * 100 + 100))
        for k in range(100):
            od = {n: float(o[k][n]) for n in o.dtype.names}
            bad = obs_close(rec_dict(recs[k]), od, L * L, beta)
            assert not bad, (block * 100 + k, bad)


@pytest.mark.parametrize("L,ty", [(48, 16), (96, 32), (200, 64)])
def test_chain_ragged_exact(orc, L, ty):
    beta, seed = 1.05, 77 + L
    lat = _lat(L, beta, seed, tile_y=ty, start="ordered")
    th = orc.init_angles(L, seed, 1)
    lat.sweep(40)
    orc.sw_run(th, L, L, beta, seed, 0, 40, record=False)
    np.testing.assert_array_equal(lat.get_angles(), th)


def test_fp16_bench_size_one_sweep(orc):
    """L = 4096, tile 64, one FP16 sweep from the random start (the
    benchmark's path with FP16 storage): bonds, labels, the stored halves of
    the flipped configuration and its observables."""
    L, beta, seed = 4096, 1.12, 1005
    lat = _lat(L, beta, seed, tile_y=64, dtype="f16")
    h0 = orc.init_angles(L, seed, 0, dtype=np.float16)
    lat.sweep(1)
    rec = lat.measure()
    g_r, g_d = lat.get_bonds()
    o_r, o_d, band = orc.bonds(h0, L, L, beta, seed, 0)
    assert int((g_r != o_r).sum() + (g_d != o_d).sum()) <= band
    g_lab = lat.get_labels()
    np.testing.assert_array_equal(g_lab, orc.label_bfs(g_r, g_d, L, L)[0])
    h = h0.copy()
    orc.flip(h, g_lab, L, L, seed, 0, orc.axis(seed, 0)[4])
    np.testing.assert_array_equal(lat.get_angles().view(np.uint16), h.view(np.uint16))
    assert not obs_close(rec_dict(rec[0]), orc.measure(h, L, L, beta), L * L, beta)


def test_fp16_chain_bit_exact(orc):
    L, beta, seed = 80, 1.1, 5
    lat = _lat(L, beta, seed, dtype="f16", tile_y=32)
    th = orc.init_angles(L, seed, 0, dtype=np.float16)
    lat.sweep(30)
    recs = lat.measure()
    o = orc.sw_run(th, L, L, beta, seed, 0, 30)
    np.testing.assert_array_equal(lat.get_angles().view(np.uint16), th.view(np.uint16))
    for k in range(30):
        od = {n: float(o[k][n]) for n in o.dtype.names}
        assert not obs_close(rec_dict(recs[k]), od, L * L, beta)


@pytest.mark.parametrize("L,ty,dtype", [(3, 16, "f32"), (64, 32, "f32"), (100, 32, "f32"),
                                        (257, 64, "f32"), (80, 32, "f16"), (512, 128, "f32")])
def test_chik_chain_matches_oracle(orc, L, ty, dtype):
    """chik (Eq. (9) at the smallest wave vector) recorded every sweep of a
    chain: angles bit-exact, chik within the bound of gpu_helpers."""
    beta, seed = 1.1, 900 + L
    lat = _lat(L, beta, seed, tile_y=ty, dtype=dtype, measure_xi=True)
    th = orc.init_angles(L, seed, 0, dtype=np.float16 if dtype == "f16" else np.float32)
    lat.sweep(25)
    recs = lat.measure()
    o = orc.sw_run(th, L, L, beta, seed, 0, 25)
    np.testing.assert_array_equal(lat.get_angles().view(np.uint8), th.view(np.uint8))
    for k in range(25):
        od = {n: float(o[k][n]) for n in o.dtype.names}
        bad = obs_close(rec_dict(recs[k]), od, L * L, beta, xi=True)
        assert not bad, (k, bad)


# ------------------------------------------------------------ limits on GPU
def test_beta_zero_has_no_bonds():
    lat = _lat(64, 0.0, 3)
    lat.sweep(3)
    r, d = lat.get_bonds()
    assert r.sum() == 0 and d.sum() == 0
    assert np.array_equal(lat.get_labels(), np.arange(64 * 64, dtype=np.uint32))


def test_infinite_beta_ordered_stays_ordered():
    lat = _lat(128, 1e9, 3, start="ordered")
    lat.sweep(20)
    recs = lat.measure()
    assert np.all(recs["energy_per_site"] == -2.0)
    a = lat.get_angles()
    assert np.all(a == a[0])


# ------------------------------------------------------- labeling kernels only
@pytest.mark.parametrize("L,ty", [(4, 16), (5, 16), (8, 16), (16, 16), (17, 16), (64, 16),
                                  (64, 64), (100, 32), (257, 128)])
@pytest.mark.parametrize("density", [0.0, 0.3, 0.5, 0.7, 1.0])
def test_label_random_masks(orc, L, ty, density):
    lat = _lat(L, 1.0, 1, tile_y=ty)
    r, d = synth.bond_masks(L, L, density, seed=L * 100 + int(density * 10))
    np.testing.assert_array_equal(lat.label_bonds(r, d), orc.label_bfs(r, d, L, L)[0])


@pytest.mark.parametrize("L,ty", [(33, 16), (64, 16), (129, 32)])
def test_label_structured_masks(orc, L, ty):
    lat = _lat(L, 1.0, 1, tile_y=ty)
    for r, d in (synth.spiral_masks(L), synth.wrap_masks(L)):
        np.testing.assert_array_equal(lat.label_bonds(r, d), orc.label_bfs(r, d, L, L)[0])


def test_label_exhaustive_2x2(orc):
    lat = _lat(2, 1.0, 1)
    for bits in range(256):
        m = ((bits >> np.arange(8)) & 1).astype(np.uint8)
        r, d = m[:4].copy(), m[4:].copy()
        np.testing.assert_array_equal(lat.label_bonds(r, d), orc.label_bfs(r, d, 2, 2)[0])


def test_label_3x3_sample(orc):
    lat = _lat(3, 1.0, 1)
    rng = np.random.default_rng(5)
    for bits in rng.integers(0, 1 << 18, size=1500):
        m = ((int(bits) >> np.arange(18)) & 1).astype(np.uint8)
        r, d = m[:9].copy(), m[9:].copy()
        np.testing.assert_array_equal(lat.label_bonds(r, d), orc.label_bfs(r, d, 3, 3)[0])


def test_label_repeatable_race_smell(orc):
    """Labeling the same dense mask many times gives identical labels."""
    L = 512
    lat = _lat(L, 1.0, 1, tile_y=64)
    r, d = synth.bond_masks(L, L, 0.52, seed=9)
    ref = orc.label_bfs(r, d, L, L)[0]
    for _ in range(5):
        np.testing.assert_array_equal(lat.label_bonds(r, d), ref)


# ------------------------------------------------------------ FP32 mode
def test_fp32_threshold_mode_mismatch_rate(orc):
    """FP32 thresholds: differences against the FP64 rule are rare."""
    L, beta, seed = 256, 1.12, 11
    th0 = synth.angles(L * L, seed=3)
    lat = _lat(L, beta, seed, exact=False)
    lat.set_angles(th0)
    lat.sweep(1)
    g_r, g_d = lat.get_bonds()
    o_r, o_d, _ = orc.bonds(th0, L, L, beta, seed, 0)
    diff = int((g_r != o_r).sum() + (g_d != o_d).sum())
    assert diff <= 5, diff


def test_band_statistics_exact_mode():
    lat = _lat(1024, 1.12, 4)
    lat.sweep(10)
    n64, wrong = lat.band_stats()
    bonds = 2 * 1024 * 1024 * 10
    assert 0 < n64 < 1e-3 * bonds
    assert wrong <= n64


# ------------------------------------------------------------ checkpoint
def test_checkpoint_resume_bit_identical():
    L = 96
    a = _lat(L, 1.1, 42, tile_y=32)
    a.sweep(50)
    ra = a.measure()
    blob = a.save()
    a.sweep(50)
    ra2 = a.measure()
    b = _lat(L, 1.1, 42, tile_y=32)
    b.load(blob)
    b.sweep(50)
    rb2 = b.measure()
    np.testing.assert_array_equal(a.get_angles(), b.get_angles())
    np.testing.assert_array_equal(ra2, rb2)
    c = _lat(L, 1.1, 42, tile_y=32)
    c.sweep(100)
    rc = c.measure()
    np.testing.assert_array_equal(np.concatenate([ra, ra2]), rc)


# ------------------------------------------------------------ PCC
@pytest.mark.parametrize("block,halve", [(1, 500), (10, 0)])
def test_pcc_trajectory_matches_oracle(orc, block, halve):
    L, seed = 48, 8
    lat = _lat(L, 1.0, seed, tile_y=16)
    th = orc.init_angles(L, seed, 0)
    st = orc.PCCState(1.0)
    n = 300
    lat.pcc_step(n, target=2 / math.pi, dbeta0=0.01, halve_every=halve, block=block)
    g = lat.measure()
    o = orc.pcc_run(th, L, st, 2 / math.pi, 0.01, halve, block, seed, 0, 0, n)
    np.testing.assert_array_equal(g["beta"], o["beta"])
    np.testing.assert_array_equal(lat.get_angles(), th)
    b, t = lat.state()
    assert t == n and b == float(st.beta[0])


# ------------------------------------------------------------ bench size
def test_bench_size_one_sweep_full_parity(orc):
    """L = 4096 (the benchmark lattice), the benchmark's tile, one sweep from
    the Philox random start: bonds, labels, angles and observables."""
    L, beta, seed = 4096, 1.12, 1001
    lat = _lat(L, beta, seed, tile_y=64)
    th0 = orc.init_angles(L, seed, 0)
    lat.sweep(1)
    rec = lat.measure()
    g_r, g_d = lat.get_bonds()
    o_r, o_d, band = orc.bonds(th0, L, L, beta, seed, 0)
    n_diff = int((g_r != o_r).sum() + (g_d != o_d).sum())
    assert n_diff <= band, (n_diff, band)
    g_lab = lat.get_labels()
    np.testing.assert_array_equal(g_lab, orc.label_bfs(g_r, g_d, L, L)[0])
    th = th0.copy()
    orc.flip(th, g_lab, L, L, seed, 0, orc.axis(seed, 0)[4])
    np.testing.assert_array_equal(lat.get_angles(), th)
    assert not obs_close(rec_dict(rec[0]), orc.measure(th, L, L, beta), L * L, beta)
    # the same sweep with chik recorded: same angles, chik within its bound
    lat_xi = _lat(L, beta, seed, tile_y=64, measure_xi=True)
    lat_xi.sweep(1)
    rec_xi = lat_xi.measure()
    np.testing.assert_array_equal(lat_xi.get_angles(), th)
    assert not obs_close(rec_dict(rec_xi[0]), orc.measure(th, L, L, beta), L * L, beta, xi=True)


def test_run_host_async_equals_run_host():
    """xy_run_host_async + xy_sync on a lattice with its own stream gives the
    records and angles of xy_run_host, step for step."""
    import torch
    L = 256
    a = _lat(L, 1.1, 31)
    b = _lat(L, 1.1, 31, stream=torch.cuda.Stream())
    th = synth.angles(L * L, seed=5)
    for step in range(4):
        ra, rb = np.zeros(2, xy.OBS_DTYPE), np.zeros(2, xy.OBS_DTYPE)
        oa, ob = np.zeros(L * L, np.float32), np.zeros(L * L, np.float32)
        a.run_host(th, 2, ra, oa)
        b.run_host_async(th, 2, rb, ob)
        b.sync()
        np.testing.assert_array_equal(ra, rb)
        np.testing.assert_array_equal(oa, ob)
        th = oa
