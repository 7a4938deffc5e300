"""Engine (many lattices, shared launches): every lattice's results are the
same bit for bit as when it runs alone through the single-lattice API, for
fixed beta and PCC, FP32 and FP16, with lattices joining and leaving between
steps.  One engine lattice is also checked against the CPU oracle."""
import math

import numpy as np
import pytest

import synth
from gpu_helpers import obs_close, rec_dict

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1210_6116_b300 as xy  # noqa: E402
from paper_1210_6116_b300 import build as xybuild  # noqa: E402

xybuild.build()


def _alone(L, beta, seed, n, *, dtype="f32", exact=False, tile_y=32, pcc=None, start="random",
           measure_xi=False):
    lat = xy.Lattice(L, beta, seed, dtype=dtype, exact=exact, tile_y=tile_y, start=start,
                     measure_xi=measure_xi)
    if pcc is None:
        lat.sweep(n)
    else:
        lat.pcc_step(n, target=pcc.target, dbeta0=pcc.dbeta0, halve_every=pcc.halve_every,
                     block=pcc.block)
    return lat.measure(), lat.get_angles()


@pytest.mark.parametrize("dtype,exact", [("f32", False), ("f32", True), ("f16", False),
                                         ("u16", False), ("u16", True)])
def test_mixed_batch_equals_alone(dtype, exact):
    table = synth.replica_table(12, seed=5, sizes=(64, 128, 256, 512), beta_range=(1.0, 1.3))
    eng = xy.Engine(len(table), dtype=dtype, exact=exact, tile_y=32)
    slots = [eng.admit(eng.config(r["L"], r["beta"], r["seed"])) for r in table]
    eng.step(25)
    for r, s in zip(table, slots):
        recs, ang = _alone(r["L"], r["beta"], r["seed"], 25, dtype=dtype, exact=exact)
        np.testing.assert_array_equal(eng.measure(s), recs)
        np.testing.assert_array_equal(eng.get_angles(s).view(np.uint8), ang.view(np.uint8))


def test_xi_and_plain_lattices_share_launches():
    """Lattices that record chik and lattices that do not run in one engine
    (the engine then launches the chik-summing observable kernel for all of
    them): each equals its alone run, and chik stays 0 where it is off."""
    table = synth.replica_table(8, seed=9, sizes=(64, 128, 256), beta_range=(1.0, 1.2))
    eng = xy.Engine(len(table), tile_y=32)
    xi = [k % 2 == 0 for k in range(len(table))]
    slots = [eng.admit(eng.config(r["L"], r["beta"], r["seed"], measure_xi=x))
             for r, x in zip(table, xi)]
    eng.step(20)
    for r, s, x in zip(table, slots, xi):
        recs, ang = _alone(r["L"], r["beta"], r["seed"], 20, measure_xi=x)
        got = eng.measure(s)
        np.testing.assert_array_equal(got, recs)
        np.testing.assert_array_equal(eng.get_angles(s), ang)
        assert (got["chik"] > 0).all() if x else not got["chik"].any()


def test_admission_and_retirement_between_steps():
    eng = xy.Engine(4, tile_y=32)
    a = eng.admit(eng.config(128, 1.1, 11))
    eng.step(10)
    b = eng.admit(eng.config(64, 1.2, 12))   # joins late
    eng.step(10)
    eng.retire(a)                              # leaves early (20 sweeps)
    c = eng.admit(eng.config(256, 1.05, 13))  # reuses a's slot
    eng.step(15)
    rb = eng.measure(b)
    rc = eng.measure(c)
    assert len(rb) == 25 and len(rc) == 15
    np.testing.assert_array_equal(rb, _alone(64, 1.2, 12, 25)[0])
    np.testing.assert_array_equal(rc, _alone(256, 1.05, 13, 15)[0])
    assert eng.state(b)[1] == 25


def test_pcc_in_engine_equals_alone():
    pcc = xy.xy_pcc_params(target=2 / math.pi, dbeta0=0.01, halve_every=500, block=1)
    eng = xy.Engine(3, tile_y=32)
    slots = [eng.admit(eng.config(L, 1.0, 40 + L), pcc) for L in (64, 128, 256)]
    eng.step(60)
    for L, s in zip((64, 128, 256), slots):
        recs, ang = _alone(L, 1.0, 40 + L, 60, pcc=pcc)
        np.testing.assert_array_equal(eng.measure(s), recs)
        np.testing.assert_array_equal(eng.get_angles(s), ang)


def test_engine_lattice_matches_oracle(orc):
    eng = xy.Engine(2, exact=True, tile_y=32)
    s0 = eng.admit(eng.config(96, 1.12, 77))
    eng.admit(eng.config(64, 1.3, 78))
    eng.step(20)
    th = orc.init_angles(96, 77, 0)
    orecs = orc.sw_run(th, 96, 96, 1.12, 77, 0, 20)
    np.testing.assert_array_equal(eng.get_angles(s0), th)
    recs = eng.measure(s0)
    assert len(recs) == 20
    for k in range(20):  # observables of every sweep (Eqs. (3)-(6))
        assert not obs_close(rec_dict(recs[k]), rec_dict(orecs[k]), 96 * 96, 1.12), k


def test_engine_rejects_bad_lattices():
    eng = xy.Engine(1, tile_y=32)
    with pytest.raises(xy.XyError) as e:
        eng.admit(eng.config(100, 1.0, 1))  # L not divisible by 32
    assert e.value.status == xy.XY_EUNSUPPORTED
    eng.admit(eng.config(64, 1.0, 1))
    with pytest.raises(xy.XyError) as e:
        eng.admit(eng.config(64, 1.0, 2))   # no free slot
    assert e.value.status == xy.XY_ENOMEM


@pytest.mark.parametrize("dtype", ["f32", "f16"])
def test_full_batch_sampled_replicas_equal_alone(dtype):
    """The batched workload at full size (256 replicas, L from {64 .. 2048},
    beta in [1.0, 1.3], FP32 thresholds, tile 32 x 64): after 3 sweeps,
    sampled replicas of every size equal their alone runs bit for bit."""
    table = synth.replica_table(256, seed=3, sizes=(64, 128, 256, 512, 1024, 2048),
                                beta_range=(1.0, 1.3))
    eng = xy.Engine(len(table), dtype=dtype, exact=False, tile_y=64)
    slots = [eng.admit(eng.config(r["L"], r["beta"], r["seed"])) for r in table]
    eng.step(3)
    picked = {}
    for k, r in enumerate(table):
        picked.setdefault(r["L"], k)
    for L, k in sorted(picked.items()):
        r = table[k]
        recs, ang = _alone(r["L"], r["beta"], r["seed"], 3, dtype=dtype, tile_y=64)
        np.testing.assert_array_equal(eng.measure(slots[k]), recs)
        np.testing.assert_array_equal(eng.get_angles(slots[k]).view(np.uint8), ang.view(np.uint8))
    eng.close()


def test_step64_sizes_batch_equals_alone_and_oracle(orc):
    """The batched workload's second size reading (multiples of 64, most not
    powers of two), tile 32 x 64: replicas of L = 192, 320, 960 and 1984 in
    one engine equal their alone runs bit for bit, and one of them equals
    the oracle's chain (FP64 thresholds)."""
    sizes = (192, 320, 960, 1984)
    eng = xy.Engine(len(sizes), exact=True, tile_y=64)
    slots = [eng.admit(eng.config(L, 1.05 + 0.05 * k, 900 + k)) for k, L in enumerate(sizes)]
    eng.step(4)
    for k, (L, s) in enumerate(zip(sizes, slots)):
        recs, ang = _alone(L, 1.05 + 0.05 * k, 900 + k, 4, exact=True, tile_y=64)
        np.testing.assert_array_equal(eng.measure(s), recs)
        np.testing.assert_array_equal(eng.get_angles(s), ang)
    th = orc.init_angles(320, 901, 0)
    orc.sw_run(th, 320, 320, 1.1, 901, 0, 4, record=False)
    np.testing.assert_array_equal(eng.get_angles(slots[1]), th)
    eng.close()


def test_chunk_graph_steps_equal_single_steps():
    # xy_engine_step replays a 4-sweep graph while at least 4 sweeps remain:
    # step(7) (one chunk, three single sweeps) equals seven step(1) calls
    pcc = xy.xy_pcc_params(target=2 / math.pi, dbeta0=0.01, halve_every=5, block=2)
    engines = [xy.Engine(4, tile_y=32) for _ in range(2)]
    slots = []
    for eng in engines:
        slots.append([eng.admit(eng.config(L, 1.05, 70 + L), pcc) for L in (32, 64, 96)])
    engines[0].step(7)
    for _ in range(7):
        engines[1].step(1)
    for sa, sb in zip(*slots):
        ra, rb = engines[0].measure(sa), engines[1].measure(sb)
        assert len(ra) == 7 and ra.tobytes() == rb.tobytes()
        assert engines[0].get_angles(sa).tobytes() == engines[1].get_angles(sb).tobytes()
