"""Accuracy of the device cos/sin routine behind the observable sums.

The observable kernel evaluates cos and sin of every new angle with its own
routine (a Cody-Waite reduction by pi/2 and the Taylor polynomials of sin and
cos on [-pi/4, pi/4]); the tolerances of the observable parity tests assume
an absolute error of at most 1.2e-7 per value.  xy_get_spins runs the same
routine on the stored angles, so these tests set angles on purpose (random
ones, every float near the quadrant edges k pi/4, the ends of [0, 2 pi)) and
compare with cos and sin in FP64.
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

BOUND = 1e-7  # what the routine guarantees; the parity tolerances assume 1.2e-7
TWO_PI_F = np.float32(2 * np.pi)  # rounds up: every float below it is < 2 pi


def _edge_floats(per_side=2000):
    """Every float within per_side ulps of k pi/4 (k = 0..8) that lies in
    [0, 2 pi), and the smallest positive floats."""
    out = [np.arange(1, 64, dtype=np.uint32).view(np.float32)]  # denormals
    for k in range(9):
        b = np.float32(k * np.pi / 4)
        bits = int(b.view(np.uint32))
        lo, hi = max(bits - per_side, 0), bits + per_side
        out.append(np.arange(lo, hi, dtype=np.uint32).view(np.float32))
    a = np.concatenate(out)
    return a[(a >= 0) & (a < TWO_PI_F)]


def _fill(L, special, rng):
    n = L * L
    a = rng.uniform(0, 2 * np.pi, n).astype(np.float32)
    a[a >= TWO_PI_F] = 0.0
    a[: special.size] = special
    return a


def _errors(c, s, theta64):
    return (np.abs(c.astype(np.float64) - np.cos(theta64)).max(),
            np.abs(s.astype(np.float64) - np.sin(theta64)).max())


@pytest.mark.parametrize("seed", [1, 2])
def test_spins_f32_accuracy(seed):
    L = 1024
    rng = np.random.default_rng(seed)
    special = _edge_floats()
    assert special.size < L * L
    a = _fill(L, special, rng)
    lat = xy.Lattice(L, 1.0, 7, dtype="f32")
    lat.set_angles(a)
    c, s = lat.get_spins()
    ec, es = _errors(c, s, a.astype(np.float64))
    assert ec <= BOUND and es <= BOUND, (ec, es)
    # exact at the points where both values are exact floats
    assert c[a == 0.0].min() == 1.0 and np.all(s[a == 0.0] == 0.0)


def test_spins_f16_accuracy():
    L = 512
    rng = np.random.default_rng(3)
    # every half value in [0, 2 pi) at the start, random ones after
    allh = np.arange(0, 0x7C00, dtype=np.uint16).view(np.float16)
    allh = allh[(allh.astype(np.float32) >= 0) & (allh.astype(np.float32) < TWO_PI_F)]
    a = rng.uniform(0, 2 * np.pi, L * L).astype(np.float16)
    a[a.astype(np.float32) >= TWO_PI_F] = 0
    a[: allh.size] = allh
    lat = xy.Lattice(L, 1.0, 7, dtype="f16")
    lat.set_angles(a)
    c, s = lat.get_spins()
    ec, es = _errors(c, s, a.astype(np.float64))
    assert ec <= BOUND and es <= BOUND, (ec, es)


def test_spins_u16_accuracy():
    L = 256  # 65536 sites: every grid angle q once
    q = np.random.default_rng(4).permutation(65536).astype(np.uint16)
    lat = xy.Lattice(L, 1.0, 7, dtype="u16")
    lat.set_angles(q)
    c, s = lat.get_spins()
    ec, es = _errors(c, s, q.astype(np.float64) * (2 * np.pi / 65536))
    assert ec <= BOUND and es <= BOUND, (ec, es)


def test_spins_ragged_and_null_outputs():
    L = 37
    a = _fill(L, np.zeros(0, np.float32), np.random.default_rng(5))
    lat = xy.Lattice(L, 1.0, 7, dtype="f32")
    lat.set_angles(a)
    c, s = lat.get_spins()
    ec, es = _errors(c, s, a.astype(np.float64))
    assert ec <= BOUND and es <= BOUND
    # one output only: the C ABI takes NULL for the other
    only_c = np.zeros(L * L, np.float32)
    xy._check(xy.load_library().xy_get_spins(lat.handle, xy._ptr(only_c), None))
    np.testing.assert_array_equal(only_c, c)
