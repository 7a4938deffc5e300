"""Pins of the oracle's sweep against closed forms, limits, an independent
sampler and the paper's own numbers.

* observables: twisted configurations with known sums (Eqs. (3)-(6));
* flip: the angle rule equals the vector reflection s' = s - 2 (s.r) r;
* bonds: beta = 0 gives none, beta -> infinity on an ordered lattice all;
* whole chain: the open 1D chain, where bonds are independent, has
  <cos dtheta> = I1(beta)/I0(beta) and a closed form for <|sum s|^2>;
* limits: E/site = -beta + O(beta^3) at small beta, -2 + 1/(2 beta) in the
  spin-wave regime, -2 exactly for an ordered start at beta -> infinity;
* independent sampler: Metropolis (own code) agrees at L = 8;
* the paper's Table 1 row L = 64 at beta_KT(64): <m^2> and beta*Upsilon.
Statistical checks use binned errors and accept |delta| < 4 sigma.
"""
import json
import math
from pathlib import Path

import numpy as np
import pytest
from scipy.special import iv

import synth
from stats import mean_err

GOLDEN = Path(__file__).resolve().parent / "golden"


# ---------------------------------------------------------------- observables
@pytest.mark.parametrize("L,k", [(8, 1), (16, 3), (33, 5)])
def test_observables_twisted_x(orc, L, k):
    th = synth.twisted_angles(L, k, axis=0)
    beta = 0.7
    o = orc.measure(th, L, L, beta)
    q = 2 * math.pi * k / L
    assert o["ex"] == pytest.approx(math.cos(q), abs=2e-6)
    assert o["sx"] == pytest.approx(-math.sin(q), abs=2e-6)
    assert o["ey"] == pytest.approx(1.0, abs=1e-12)
    assert o["sy"] == pytest.approx(0.0, abs=1e-12)
    assert o["energy_per_site"] == pytest.approx(-(math.cos(q) + 1.0), abs=2e-6)
    assert o["m2"] == pytest.approx(0.0, abs=1e-10)
    ups = math.cos(q) - beta * L * L * math.sin(q) ** 2
    assert o["upsilon"] == pytest.approx(ups, rel=1e-5)


@pytest.mark.parametrize("L,k", [(8, 1), (17, 2)])
def test_observables_twisted_y(orc, L, k):
    th = synth.twisted_angles(L, k, axis=1)
    o = orc.measure(th, L, L, 1.1)
    q = 2 * math.pi * k / L
    assert o["ex"] == pytest.approx(1.0, abs=1e-12)
    assert o["sx"] == pytest.approx(0.0, abs=1e-12)
    assert o["ey"] == pytest.approx(math.cos(q), abs=2e-6)
    assert o["sy"] == pytest.approx(-math.sin(q), abs=2e-6)
    assert o["upsilon"] == pytest.approx(1.0, abs=1e-12)


@pytest.mark.parametrize("L,k", [(8, 1), (33, 5)])
def test_observable_l1_norms_twisted_x(orc, L, k):
    """The L1 norms per site of the sums behind m, e and s on a twisted
    field: every x-link has |cos| = |cos q| and |sin| = |sin q|, every y-link
    cos = 1 and sin = 0, and the site sums average |cos|, |sin| of 2 pi k x / L
    over the columns."""
    th = synth.twisted_angles(L, k, axis=0)
    o = orc.measure(th, L, L, 0.9)
    q = 2 * math.pi * k / L
    assert o["l1_ex"] == pytest.approx(abs(math.cos(q)), abs=2e-6)
    assert o["l1_sx"] == pytest.approx(abs(math.sin(q)), abs=2e-6)
    assert o["l1_ey"] == pytest.approx(1.0, abs=1e-12)
    assert o["l1_sy"] == pytest.approx(0.0, abs=1e-12)
    col = 2 * math.pi * k * np.arange(L) / L
    assert o["l1_mx"] == pytest.approx(np.abs(np.cos(col)).mean(), abs=1e-6)
    assert o["l1_my"] == pytest.approx(np.abs(np.sin(col)).mean(), abs=1e-6)
    # a sum never exceeds its L1 norm
    for f in ("mx", "my", "ex", "sx", "ey", "sy"):
        assert abs(o[f]) <= o["l1_" + f] + 1e-15


def test_observables_uniform_field(orc):
    L = 10
    th = np.full(L * L, np.float32(1.25))
    o = orc.measure(th, L, L, 1.0)
    assert o["energy_per_site"] == -2.0
    assert o["m2"] == pytest.approx(1.0, abs=1e-14)
    assert o["mx"] == pytest.approx(math.cos(np.float32(1.25)), abs=1e-14)


# ----------------------------------------------------------------------- axis
def test_axis_properties(orc):
    phis = []
    for t in range(2000):
        phi, c, s, C64, C32 = orc.axis(9, t)
        assert 0.0 <= phi < 2 * math.pi
        assert c == pytest.approx(math.cos(phi), abs=0)
        assert c * c + s * s == pytest.approx(1.0, abs=1e-15)
        assert 0.0 <= C64 < 2 * math.pi
        assert math.cos(C64) == pytest.approx(math.cos(math.pi + 2 * phi), abs=1e-12)
        assert 0.0 <= float(C32) < float(np.float32(2 * math.pi))
        phis.append(phi)
    h = np.histogram(phis, bins=20, range=(0, 2 * math.pi))[0]
    e = len(phis) / 20
    assert ((h - e) ** 2 / e).sum() < 19 + 5 * math.sqrt(38)


# ----------------------------------------------------------------------- flip
def test_flip_is_vector_reflection(orc):
    """For every flipped site theta' equals the angle of s - 2 (s.r) r, and the
    projection on r changes sign; unflipped sites are unchanged."""
    L, seed = 24, 5
    th0 = synth.angles(L * L, seed=11)
    for t in range(5):
        phi, c, s, C64, C32 = orc.axis(seed, t)
        right, down, _ = orc.bonds(th0, L, L, 1.0, seed, t)
        lab, _ = orc.label_bfs(right, down, L, L)
        th = th0.copy()
        fl = orc.flip(th, lab, L, L, seed, t, C32)
        sx, sy = np.cos(th0.astype(np.float64)), np.sin(th0.astype(np.float64))
        proj = sx * c + sy * s
        rx, ry = sx - 2 * proj * c, sy - 2 * proj * s
        want = np.mod(np.arctan2(ry, rx), 2 * math.pi)
        got = th.astype(np.float64)
        d = np.abs(np.angle(np.exp(1j * (got - want))))
        assert np.all(d[fl == 1] < 2e-6)
        np.testing.assert_array_equal(th[fl == 0], th0[fl == 0])
        newproj = np.cos(got) * c + np.sin(got) * s
        assert np.all(np.abs(newproj[fl == 1] + proj[fl == 1]) < 2e-6)
        # the flip set is a union of whole clusters
        for r in np.unique(lab):
            assert len(np.unique(fl[lab == r])) == 1


def test_coin_is_fair(orc):
    n = 40000
    flips = sum(orc.coin(77, t, r, 64) for t in range(40) for r in range(n // 40))
    assert abs(flips - n / 2) < 4 * math.sqrt(n / 4)


# ---------------------------------------------------------------------- bonds
def test_bonds_beta_zero_none(orc):
    L = 32
    th = synth.angles(L * L, seed=3)
    for t in range(5):
        right, down, _ = orc.bonds(th, L, L, 0.0, 21, t)
        assert right.sum() == 0 and down.sum() == 0


def test_bonds_beta_infinite_ordered_all(orc):
    L = 16
    th = np.zeros(L * L, np.float32)
    for t in range(10):
        _, c, _, _, _ = orc.axis(21, t)
        if abs(c) < 1e-3:
            continue
        right, down, _ = orc.bonds(th, L, L, 1e9, 21, t)
        assert right.all() and down.all()


def test_ordered_start_stays_ordered_at_infinite_beta(orc):
    L = 16
    th = orc.init_angles(L, 5, start=1)
    obs = orc.sw_run(th, L, L, 1e9, 5, 0, 20)
    assert np.all(obs["energy_per_site"] == -2.0)
    assert np.all(th == th[0])


def test_init_angles(orc):
    th = orc.init_angles(64, 1, start=0)
    assert th.dtype == np.float32
    assert th.min() >= 0 and th.max() < np.float32(2 * math.pi)
    # uniform: mean angle ~ pi, resultant small
    assert abs(np.mean(np.cos(th))) < 5 / 64 and abs(np.mean(np.sin(th))) < 5 / 64
    h = orc.init_angles(64, 1, start=0, dtype=np.float16)
    assert h.dtype == np.float16
    assert h.astype(np.float32).max() < np.float32(2 * math.pi)
    # FP16 start is the FP32 start rounded to nearest half (then wrapped)
    assert np.max(np.abs(h.astype(np.float32) - th)) <= 2 ** -8 + 1e-7


# ----------------------------------------------------------- 1D chain closed forms
@pytest.mark.parametrize("beta", [0.5, 1.0, 2.0, 5.0])
def test_open_chain_closed_form(orc, beta):
    N, n = 64, 20000
    th = orc.init_angles(N, 100 + int(beta * 10), start=0, Ly=1)
    obs = orc.sw_run(th, N, 1, beta, 100 + int(beta * 10), 0, n, per_x=0, per_y=0)
    t = iv(1, beta) / iv(0, beta)
    cos_bond = obs["ex"] * N / (N - 1)  # sum over the N - 1 links / (N - 1)
    m, e = mean_err(cos_bond[200:])
    assert abs(m - t) < 4 * e + 1e-4, (m, e, t)
    m2_theory = (N * (1 + t) / (1 - t) - 2 * t * (1 - t ** N) / (1 - t) ** 2) / N ** 2
    m, e = mean_err(obs["m2"][200:])
    assert abs(m - m2_theory) < 4 * e, (m, e, m2_theory)
    # no links along y in the open chain
    assert np.all(obs["ey"] == 0.0)


# ------------------------------------------------------------------- limits
def test_small_beta_energy(orc):
    L, beta, n = 16, 0.05, 20000
    th = synth.angles(L * L, seed=4)
    obs = orc.sw_run(th, L, L, beta, 17, 0, n)
    m, e = mean_err(obs["energy_per_site"])
    # high-temperature expansion: E/site = -2 I1/I0 + O(beta^3) = -beta + O(beta^3)
    assert abs(m - (-beta)) < 4 * e + beta ** 3, (m, e)


def test_beta_zero_energy_vanishes(orc):
    L = 16
    th = synth.angles(L * L, seed=5)
    obs = orc.sw_run(th, L, L, 0.0, 19, 0, 4000)
    m, e = mean_err(obs["energy_per_site"])
    assert abs(m) < 4 * e


@pytest.mark.parametrize("beta", [20.0, 50.0])
def test_spin_wave_energy(orc, beta):
    L, n = 16, 6000
    th = orc.init_angles(L, 23, start=1)
    obs = orc.sw_run(th, L, L, beta, 23, 0, n)
    m, e = mean_err(obs["energy_per_site"][500:])
    # equipartition of the N quadratic modes: E/site = -2 + T/2 + O(T^2)
    assert abs((m + 2.0) - 0.5 / beta) < 4 * e + 1.0 / beta ** 2, (m, e)


# ------------------------------------------------------ independent sampler
@pytest.mark.parametrize("beta", [0.5, 1.12, 2.0])
def test_metropolis_agrees(orc, beta):
    L = 8
    n_sw, n_mc = 20000, 60000
    th = synth.angles(L * L, seed=8)
    sw = orc.sw_run(th, L, L, beta, 31, 0, n_sw)[500:]
    th64 = synth.angles(L * L, seed=9).astype(np.float64)
    mc, acc = orc.metropolis_run(th64, L, beta, 2.0, 37, 0, n_mc)
    mc = mc[2000:]
    for key in ("energy_per_site", "m2", "upsilon"):
        a, ea = mean_err(sw[key])
        b, eb = mean_err(mc[key])
        assert abs(a - b) < 4 * math.hypot(ea, eb), (key, a, ea, b, eb)


# ------------------------------------------------------------- paper Table 1
def test_table1_L64(orc):
    """At beta = beta_KT(64) = 1.09167 the fixed-beta chain must reproduce
    Table 1's <m^2>_64 = 0.34924(29) and beta*Upsilon at the PCC target."""
    golden = json.loads((GOLDEN / "table1.json").read_text())
    row = next(r for r in golden["rows"] if r["L"] == 64)
    target = golden["critical_beta_upsilon"]["value"]
    L, beta = 64, row["beta_kt"]
    th = orc.init_angles(L, 64, start=0)
    orc.sw_run(th, L, L, beta, 64, 0, 300, record=False)
    obs = orc.sw_run(th, L, L, beta, 64, 300, 6000)
    m, e = mean_err(obs["m2"])
    assert abs(m - row["m2"]) < 4 * math.hypot(e, row["m2_err"]), (m, e)
    b, eb = mean_err(obs["beta"] * obs["upsilon"])
    # the PCC fixes beta by the mean of beta*Upsilon; beta itself is known to
    # +-0.00025, which moves beta*Upsilon by about 1.5 x that.
    assert abs(b - target) < 4 * math.hypot(eb, 1.5 * row["beta_err"]), (b, eb)


# ----------------------------------------------------------------------- PCC
def test_pcc_rule(orc):
    assert orc.pcc_next_beta(1.0, 0.5, 0.636508, 0.01) == 1.01
    assert orc.pcc_next_beta(1.0, 0.7, 0.636508, 0.01) == 0.99
    assert orc.pcc_next_beta(1.0, 0.636508, 0.636508, 0.01) == 0.99  # tie: decrease
    assert orc.pcc_dbeta(0.01, 500, 499) == 0.01
    assert orc.pcc_dbeta(0.01, 500, 500) == 0.005
    assert orc.pcc_dbeta(0.01, 500, 1500) == 0.00125
    assert orc.pcc_dbeta(0.0005, 0, 10 ** 6) == 0.0005


def test_pcc_drives_beta_to_the_crossing(orc):
    """A block-averaged PCC run at L = 16 ends at a beta where fixed-beta runs
    bracket the target: beta*Upsilon below it 0.08 lower, above it 0.08 higher."""
    L, seed = 16, 99
    target = 0.636508
    th = orc.init_angles(L, seed, start=0)
    st = orc.PCCState(0.8)
    orc.pcc_run(th, L, st, target, 0.02, 400, 50, seed, 0, 0, 4000)
    bf = float(st.beta[0])
    assert 0.85 < bf < 1.3
    lo = orc.sw_run(th.copy(), L, L, bf - 0.08, 5, 10000, 4000)
    hi = orc.sw_run(th.copy(), L, L, bf + 0.08, 6, 20000, 4000)
    ml, el = mean_err((lo["beta"] * lo["upsilon"])[200:])
    mh, eh = mean_err((hi["beta"] * hi["upsilon"])[200:])
    assert ml < target + 2 * el and mh > target - 2 * eh, (bf, ml, el, mh, eh)


def test_fp16_flip_is_vector_reflection(orc):
    """FP16 storage: a flipped angle is the reflection of the stored half
    angle, rounded to FP16 (within half an FP16 ulp at [4, 8): 2^-9, plus the
    FP32 step), and unflipped angles keep their bits."""
    L, seed = 24, 6
    th0 = synth.angles(L * L, seed=12, dtype=np.float16)
    for t in range(4):
        phi, c, s, C64, C32 = orc.axis(seed, t)
        right, down, _ = orc.bonds(th0, L, L, 1.0, seed, t)
        lab, _ = orc.label_bfs(right, down, L, L)
        th = th0.copy()
        fl = orc.flip(th, lab, L, L, seed, t, C32)
        old = th0.astype(np.float64)
        proj = np.cos(old) * c + np.sin(old) * s
        rx, ry = np.cos(old) - 2 * proj * c, np.sin(old) - 2 * proj * s
        want = np.mod(np.arctan2(ry, rx), 2 * math.pi)
        d = np.abs(np.angle(np.exp(1j * (th.astype(np.float64) - want))))
        assert np.all(d[fl == 1] <= 2.0 ** -9 + 1e-6)
        np.testing.assert_array_equal(th.view(np.uint16)[fl == 0], th0.view(np.uint16)[fl == 0])
        assert np.all(th.astype(np.float32) < np.float32(2 * math.pi))


# ------------------------------------------------------------ xi_2nd (Eq. (9))
@pytest.mark.parametrize("L,k", [(16, 1), (24, 1), (32, 2)])
def test_chik_plane_waves(orc, L, k):
    """theta = 2 pi k x / L: s(r) = (cos q x, sin q x).  At the smallest wave
    vector along x, |F|^2 = N^2/2 when k = 1 (and 0 when k > 1, orthogonal
    harmonics); along y every column sums to zero.  chik = (|Fx|^2+|Fy|^2)/2N."""
    N = L * L
    o = orc.measure(synth.twisted_angles(L, k, axis=0), L, L, 1.0)
    want = (N * N / 2.0 if k == 1 else 0.0) / (2 * N)
    assert o["chik"] == pytest.approx(want, abs=1e-6 * N)
    o = orc.measure(synth.twisted_angles(L, k, axis=1), L, L, 1.0)
    assert o["chik"] == pytest.approx(want, abs=1e-6 * N)


def test_chik_uniform_and_staggered(orc):
    L = 20
    assert orc.measure(np.full(L * L, np.float32(0.7)), L, L, 1.0)["chik"] == pytest.approx(0.0, abs=1e-9)
    # a single flipped site (theta = pi) on an ordered field: F(k) = -2 e^{ik r0}
    th = np.zeros(L * L, np.float32)
    th[3 * L + 5] = np.float32(math.pi)
    assert orc.measure(th, L, L, 1.0)["chik"] == pytest.approx((4 + 4) / (2 * L * L), rel=1e-6)


# ------------------------------------------------- u16 fixed-point angles
# theta = q 2pi / 65536.  The axis sits on the reflection grid, so the flip is
# the integer map q -> (Cq - q) mod 65536 and the update is an exact cluster
# move of the 65536-state clock model.
U16_STEP = 2 * math.pi / 65536


def test_u16_axis_is_the_fp32_axis_on_the_grid(orc):
    """phi_q is phi (of the FP32-angle axis, pinned above) reduced mod pi and
    floored to the grid pi/65536; pi + 2 phi_q = Cq 2pi/65536; m is uniform."""
    ms = []
    for t in range(3000):
        phi = orc.axis(13, t)[0]
        phq, c, s, C64, cq = orc.axis_u16(13, t)
        d = math.fmod(phi, math.pi) - phq
        assert -1e-12 <= d < math.pi / 65536 + 1e-12, (t, phi, phq)
        assert c == math.cos(phq) and s == math.sin(phq)
        assert C64 == cq * U16_STEP
        assert math.cos(math.pi + 2 * phq) == pytest.approx(math.cos(C64), abs=1e-12)
        assert math.sin(math.pi + 2 * phq) == pytest.approx(math.sin(C64), abs=1e-12)
        ms.append(int(round(phq / (math.pi / 65536))))
    h = np.histogram(ms, bins=16, range=(0, 65536))[0]
    e = len(ms) / 16
    assert ((h - e) ** 2 / e).sum() < 15 + 5 * math.sqrt(30)


def test_u16_flip_is_exact_vector_reflection(orc):
    """Every flipped q' is the reflection s - 2 (s.r) r of q about the grid
    axis, to FP64 rounding; the projection on r is exactly negated (this is
    what makes the move exact); flipping twice restores every bit."""
    L, seed = 24, 8
    q0 = synth.angles(L * L, seed=14, dtype=np.uint16)
    for t in range(6):
        phq, c, s, C64, cq = orc.axis_u16(seed, t)
        right, down, _ = orc.bonds(q0, L, L, 1.0, seed, t)
        lab, _ = orc.label_bfs(right, down, L, L)
        q = q0.copy()
        fl = orc.flip(q, lab, L, L, seed, t, cq)
        old = q0.astype(np.float64) * U16_STEP
        new = q.astype(np.float64) * U16_STEP
        proj = np.cos(old) * c + np.sin(old) * s
        rx, ry = np.cos(old) - 2 * proj * c, np.sin(old) - 2 * proj * s
        d = np.abs(np.angle(np.exp(1j * (new - np.arctan2(ry, rx)))))
        assert np.all(d[fl == 1] < 1e-12)
        newproj = np.cos(new) * c + np.sin(new) * s
        assert np.all(np.abs(newproj[fl == 1] + proj[fl == 1]) < 1e-12)
        np.testing.assert_array_equal(q[fl == 0], q0[fl == 0])
        orc.flip(q, lab, L, L, seed, t, cq)
        np.testing.assert_array_equal(q, q0)


def test_u16_init_is_the_fp32_start_truncated(orc):
    """q = the top 16 of the 24 bits that the FP32 start scales by 2pi 2^-24."""
    th = orc.init_angles(64, 3, start=0)
    q = orc.init_angles(64, 3, start=0, dtype=np.uint16)
    assert q.dtype == np.uint16
    step = np.float32(2 * math.pi) * np.float32(2.0 ** -24)
    # the FP32 start rounds w24 * step to 24 bits, so w24 comes back within 1
    w24 = np.rint(th.astype(np.float64) / float(step)).astype(np.int64)
    ok = th > 0  # the FP32 start wraps a value that rounds to 2pi to 0
    d = (w24[ok] >> 8) - q[ok].astype(np.int64)
    edge = np.isin(w24[ok] & 255, (0, 255))
    assert np.all(d[~edge] == 0) and np.all(np.abs(d[edge]) <= 1)
    assert edge.sum() < 0.02 * ok.sum()
    assert not orc.init_angles(16, 3, start=1, dtype=np.uint16).any()


@pytest.mark.parametrize("L,k", [(16, 1), (32, 3)])
def test_u16_observables_twisted(orc, L, k):
    """q = k x 65536 / L is exactly a twist by 2 pi k / L."""
    y, x = np.mgrid[0:L, 0:L]
    q = ((k * x * (65536 // L)) % 65536).astype(np.uint16).ravel()
    o = orc.measure(q, L, L, 0.9)
    a = 2 * math.pi * k / L
    assert o["ex"] == pytest.approx(math.cos(a), abs=1e-14)
    assert o["sx"] == pytest.approx(-math.sin(a), abs=1e-14)
    assert o["ey"] == pytest.approx(1.0, abs=1e-14)
    assert o["m2"] == pytest.approx(0.0, abs=1e-14)


@pytest.mark.parametrize("beta", [1.0, 3.0])
def test_u16_open_chain_closed_form(orc, beta):
    """The 65536-state clock chain is the XY chain to ~1e-9: I1/I0 per link."""
    N, n = 64, 20000
    seed = 300 + int(beta * 10)
    q = orc.init_angles(N, seed, start=0, Ly=1, dtype=np.uint16)
    obs = orc.sw_run(q, N, 1, beta, seed, 0, n, per_x=0, per_y=0)
    t = iv(1, beta) / iv(0, beta)
    m, e = mean_err((obs["ex"] * N / (N - 1))[200:])
    assert abs(m - t) < 4 * e + 1e-4, (m, e, t)


def test_u16_chain_matches_fp32_chain(orc):
    """L = 16, beta = 1.0: u16 and FP32 chains sample the same distribution."""
    L, beta, n = 16, 1.0, 12000
    a = orc.sw_run(orc.init_angles(L, 41, 0), L, L, beta, 41, 0, n)
    b = orc.sw_run(orc.init_angles(L, 42, 0, dtype=np.uint16), L, L, beta, 42, 0, n)
    for f in ("energy_per_site", "m2"):
        ma, ea = mean_err(a[f][500:])
        mb, eb = mean_err(b[f][500:])
        assert abs(ma - mb) < 4 * math.hypot(ea, eb), (f, ma, ea, mb, eb)


def test_u16_bonds_use_the_grid_axis(orc):
    """Bonds project on the grid axis phi_q itself: spins exactly perpendicular
    to it (q = (m + 32768) / 2) get no bond even at beta = 1e12, spins along it
    (q = m / 2) all get one.  With the unrounded axis phi the perpendicular
    spins would project to ~pi/65536 and bond."""
    L, seed, tested = 8, 31, 0
    for t in range(40):
        phq, c, s, C64, cq = orc.axis_u16(seed, t)
        m = int(round(phq / (math.pi / 65536)))
        if m % 2:
            continue
        tested += 1
        perp = np.full(L * L, (m + 32768) // 2, np.uint16)
        r, d, _ = orc.bonds(perp, L, L, 1e12, seed, t)
        assert not r.any() and not d.any(), t
        par = np.full(L * L, m // 2, np.uint16)
        r, d, _ = orc.bonds(par, L, L, 1e12, seed, t)
        assert r.all() and d.all(), t
    assert tested >= 10
