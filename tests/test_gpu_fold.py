"""Fixed-beta sweeps fold the finalize step into the next sweep's first kernel.

Block 0 of k_bond_label appends the previous sweep's record (Eqs. (3)-(6))
and draws the next sweep's random axis (Sec. 2). k_finalize then runs only at
the end of each xy_sweep call. xy_pcc_step with dbeta0 = 0 keeps beta fixed
but runs the unfolded path, with k_finalize after every sweep. The two must
give bit-identical angles, labels, records and state. The calls are of 1, 2,
3 and 4 sweeps, so that a call ends in either parameter slot. The tests also
mix the two kinds of call on one lattice and cross a save / load. The
unfolded path is itself checked against the oracle in test_gpu_parity.py.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1210_6116_b300 as xy  # noqa: E402
from paper_1210_6116_b300 import build as xybuild  # noqa: E402

xybuild.build()

BETA = 1.12
CALLS = (1, 3, 2, 1, 4)
CASES = {
    "f32": dict(L=64),
    "f32_ragged": dict(L=100, tile_y=32),
    "f16": dict(L=64, dtype="f16"),
    "u16": dict(L=64, dtype="u16"),
    "fp32_thresholds": dict(L=64, exact=False),
    "xi": dict(L=96, measure_xi=True),
    "wolff": dict(L=64, update="wolff"),
}


def _pair(kw, seed=77):
    kw = dict(kw)
    L = kw.pop("L")
    return (xy.Lattice(L, BETA, seed, **kw), xy.Lattice(L, BETA, seed, **kw))


def _unfolded(lat, n):
    lat.pcc_step(n, target=0.5, dbeta0=0.0, block=1)


def _same(a, b):
    ra, rb = a.measure(), b.measure()
    assert len(ra) == len(rb)
    assert ra.tobytes() == rb.tobytes(), "records differ"
    assert a.get_angles().tobytes() == b.get_angles().tobytes(), "angles differ"
    np.testing.assert_array_equal(a.get_labels(), b.get_labels())
    assert a.state() == b.state()
    return ra


@pytest.mark.parametrize("name", list(CASES))
def test_fold_matches_finalize(name):
    a, b = _pair(CASES[name])
    for n in CALLS:
        a.sweep(n)
        _unfolded(b, n)
    recs = _same(a, b)
    total = sum(CALLS)
    assert [int(r["sweep"]) for r in recs] == list(range(total))
    assert np.all(recs["beta"] == BETA)
    assert a.state() == (BETA, total)


def test_fold_mixed_calls_and_checkpoint():
    a, b = _pair(CASES["f32_ragged"], seed=5)
    # fold and unfold alternate on `a`; `b` never folds
    for n, fold in ((2, True), (1, False), (3, True), (2, False), (1, True)):
        if fold:
            a.sweep(n)
        else:
            _unfolded(a, n)
        _unfolded(b, n)
    _same(a, b)
    # a checkpoint taken between calls restores both parameter slots
    blob = a.save()
    c = xy.Lattice(100, BETA, 5, tile_y=32)
    c.load(blob)
    a.sweep(3)
    c.sweep(3)
    _same(a, c)


def test_fold_profile_counts():
    lat = xy.Lattice(64, BETA, 9)
    lat.profile(True, every=1)
    lat.sweep(3)
    lat.sweep(1)
    kt = lat.profile_read()
    lat.profile(False)
    assert kt["bond_label"][1] == 4 and kt["flip_measure"][1] == 4
    assert kt["finalize"][1] == 2  # one record-only finalize per call
    _unfolded(lat, 2)
    assert len(lat.measure()) == 6


# ------------------------------------------------------------ chunk graphs
# xy_sweep replays a recorded CUDA graph of 16 middle sweeps (from an odd
# sweep index of the call), so calls of >= 18 sweeps go partly through it.
@pytest.mark.parametrize("name", ["f32", "f32_ragged", "u16", "xi", "wolff"])
def test_graph_chunks_match_finalize(name):
    a, b = _pair(CASES[name], seed=11)
    for n in (40, 18, 35):  # 2, 1 and 2 replays, with direct launches around them
        a.sweep(n)
        _unfolded(b, n)
    assert len(_same(a, b)) == 93
    # a new descriptor drops the recorded graph; the next call records it again
    a.set_loop_bound(0)
    b.set_loop_bound(0)
    a.sweep(20)
    _unfolded(b, 20)
    _same(a, b)


def test_graph_chunks_with_profiling():
    a, b = _pair(CASES["f32"], seed=12)
    # every 4th sweep timed: every run of 16 holds a timed sweep, no replays
    a.profile(True, every=4)
    a.sweep(40)
    assert a.profile_read()["bond_label"][1] == 10
    # every 64th: sweep 0 timed, sweeps 1-32 replayed, 33-39 launched directly
    a.profile(True, every=64)
    a.sweep(40)
    kt = a.profile_read()
    a.profile(False)
    assert kt["bond_label"][1] == 1 and kt["finalize"][1] == 0
    _unfolded(b, 80)
    _same(a, b)


def test_pcc_graph_chunks_match_direct_launches():
    # xy_pcc_step replays its own 16-sweep graph; with every sweep timed by
    # xy_profile all sweeps are launched directly instead
    a, b = _pair(CASES["f32_ragged"], seed=13)
    b.profile(True, every=1)
    for n in (40, 19):
        for lat in (a, b):
            lat.pcc_step(n, target=0.6, dbeta0=0.01, halve_every=10, block=3)
    b.profile(False)
    recs = _same(a, b)
    assert len(np.unique(recs["beta"])) > 1  # beta moved


def test_sweep_captured_by_the_caller():
    # while the caller captures the lattice's stream, xy_sweep launches every
    # kernel directly (no nested graph); replaying the caller's graph once
    # advances the lattice like the same call made directly
    s = torch.cuda.Stream()
    a = xy.Lattice(64, BETA, 21, stream=s)
    b = xy.Lattice(64, BETA, 21)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        a.sweep(20)
    g.replay()
    torch.cuda.synchronize()
    b.sweep(20)
    assert a.get_angles().tobytes() == b.get_angles().tobytes()
    assert a.state() == b.state() == (BETA, 20)
    rb = b.measure()
    ra = a.measure()  # the ring holds the replayed sweeps' records
    assert ra.tobytes() == rb.tobytes()


def test_pcc_captured_by_the_caller():
    # the same for xy_pcc_step: no nested graph while the caller captures
    s = torch.cuda.Stream()
    a = xy.Lattice(64, 1.0, 22, stream=s)
    b = xy.Lattice(64, 1.0, 22)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        a.pcc_step(20, target=0.6, dbeta0=0.01, block=1)
    g.replay()
    torch.cuda.synchronize()
    b.pcc_step(20, target=0.6, dbeta0=0.01, block=1)
    assert a.get_angles().tobytes() == b.get_angles().tobytes()
    assert a.state() == b.state()
    assert a.measure().tobytes() == b.measure().tobytes()
