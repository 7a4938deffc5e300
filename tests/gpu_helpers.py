"""Shared helpers of the GPU parity tests: tolerances and record comparison.

Observable tolerance (reading A19 of the hot-path scope: 1e-6 relative, with
sums that cancel compared against their L1 norm).  With REL = 1e-6 and, from
the oracle's record, l1_q = N^-1 sum |term| of the sum behind q:

    E/site, e_x, e_y, m_x, m_y, s_x, s_y   REL * l1_q
    Upsilon = e_x - beta N s_x^2           REL * (l1_ex + beta N s_x^2)
    M^2 = m_x^2 + m_y^2                    REL * max(M^2, |m_x| l1_mx + |m_y| l1_my)

For a sum that does not cancel (the ordered and critical configurations the
method runs at: E/site ~ -1.4, e_x ~ 0.7, M^2 = O(0.1 .. 1)) l1_q = |q| and
these are exactly 1e-6 relative; l1_q only matters where the terms cancel
(m, s, and e near infinite temperature).  Upsilon is compared against the
magnitudes of its two terms, and no term of any tolerance grows with N.

The kernel's error is far below these: every term is an FP32 product of the
kernel's own cos/sin (absolute error <= 1e-7, test_gpu_spins), rounded to a
2^-22 grid and summed exactly in integers, so the error of a per-site mean is
a sum of N independent roundings divided by N.  measured_errors() keeps the
largest error / tolerance seen per field; conftest writes it out when
XY_OBS_ERRLOG names a file.

chik (Eq. (9) at the smallest wave vector) is built from eight Fourier sums
F_c = sum_r {cos, sin}(theta_r) {cos, sin}(2 pi x / L) of terms within
EPS_WAVE = 3.6e-7 (FP32 cos/sin 1.2e-7, wave factor rounded from FP64 6e-8,
product rounding 6e-8, 2^-22 grid 1.2e-7), so |dF_c| <= dF = EPS_WAVE N; with
sum_c |F_c| <= 4 sqrt(N chik) the error of chik = sum_c F_c^2 / (2N) is at
most (4 dF sqrt(N chik) + 4 dF^2) / N (reading A20).
"""
import numpy as np

REL = 1e-6
EPS_WAVE = 3.6e-7

_worst: dict = {}


def measured_errors() -> dict:
    """Largest |gpu - oracle| / tolerance (and the error itself) per field."""
    return dict(_worst)


def _note(k, err, tol, val):
    w = _worst.get(k)
    r = err / tol if tol > 0 else (0.0 if err == 0 else float("inf"))
    if w is None or r > w["err_over_tol"]:
        _worst[k] = {"err_over_tol": r, "abs_err": err,
                     "rel_err": err / abs(val) if val else None}


def obs_tolerances(o: dict, N: int, beta: float) -> dict:
    """Tolerance of each compared observable, from the oracle record o."""
    tol = {"energy_per_site": REL * (o["l1_ex"] + o["l1_ey"])}
    for k in ("ex", "sx", "ey", "sy", "mx", "my"):
        tol[k] = REL * o["l1_" + k]
    tol["upsilon"] = REL * (o["l1_ex"] + beta * N * o["sx"] ** 2)
    tol["m2"] = REL * max(o["m2"], abs(o["mx"]) * o["l1_mx"] + abs(o["my"]) * o["l1_my"])
    return tol


def obs_close(g: dict, o: dict, N: int, beta: float, xi: bool = False, flips: bool = False):
    """Return a list of (field, gpu, oracle, tol) that violate the tolerance.
    xi: the GPU lattice measures chik; otherwise its chik must be exactly 0.
    flips: the GPU counts reflected sites (Wolff), compared exactly with the
    oracle's count; otherwise (SW) the count must be 0."""
    bad = []

    def chk(k, tol):
        err = abs(g[k] - o[k])
        _note(k, err, tol, o[k])
        if err > tol:
            bad.append((k, g[k], o[k], tol))

    for k, tol in obs_tolerances(o, N, beta).items():
        chk(k, tol)
    if xi:
        dF = EPS_WAVE * N
        chk("chik", max(REL * o["chik"], (4 * dF * np.sqrt(N * o["chik"]) + 4 * dF * dF) / N))
    elif g.get("chik", 0.0) != 0.0:
        bad.append(("chik", g["chik"], 0.0, 0.0))
    if g["beta"] != o["beta"]:
        bad.append(("beta", g["beta"], o["beta"], 0.0))
    if flips:
        if g["flipped"] != o["flipped"]:
            bad.append(("flipped", g["flipped"], o["flipped"], 0.0))  # a count: exact
    elif g.get("flipped", 0.0) != 0.0:
        bad.append(("flipped", g["flipped"], 0.0, 0.0))
    return bad


def rec_dict(rec) -> dict:
    return {k: float(rec[k]) for k in rec.dtype.names if k != "sweep"}


def band_mismatches(orc, theta, L, beta, seed, t, g_right, g_down, o_right, o_down):
    """Bond bits where GPU and oracle differ, split into those inside the
    |u - p| < 1e-12 exception band and those outside it."""
    inside, outside = [], []
    for direction, g, o in ((0, g_right, o_right), (1, g_down, o_down)):
        for i in np.nonzero(g != o)[0]:
            u, p = orc.bond_up(theta, L, L, beta, seed, t, int(i), direction)
            (inside if abs(u - p) < 1e-12 else outside).append((direction, int(i), u, p))
    return inside, outside


_SUM_FIELDS = ("sum_cos", "sum_sin", "sum_cos_r", "sum_sin_r", "sum_cos_d", "sum_sin_d",
               "abs_cos", "abs_sin", "abs_cos_r", "abs_sin_r", "abs_cos_d", "abs_sin_d")


def banded_measure(orc, theta, L: int, beta: float, band: int = 1024, omp: bool = True) -> dict:
    """The oracle's observables of an L x L periodic FP32 configuration,
    computed over bands of rows so that no more than a band is widened at
    once: each band [y0, y0 + h) is summed as an (h + 1)-row lattice, open
    in y (its down links reach the next band's first row), minus that extra
    row's own site and right-link terms.  Equal to orc.measure up to the
    order of summation.  omp: the oracle's OpenMP build."""
    tot = dict.fromkeys(_SUM_FIELDS, 0.0)
    for y0 in range(0, L, band):
        h = min(band, L - y0)
        if y0 + h < L:
            rows = theta[y0 * L:(y0 + h + 1) * L]
        else:
            rows = np.concatenate([theta[y0 * L:], theta[:L]])
        s = orc.sums(rows, L, h + 1, per_x=1, per_y=0, omp=omp)
        e = orc.sums(np.ascontiguousarray(rows[h * L:]), L, 1, per_x=1, per_y=0, omp=omp)
        for f in _SUM_FIELDS:
            tot[f] += getattr(s, f) - getattr(e, f)
    s = orc.Sums()
    for f in _SUM_FIELDS:
        setattr(s, f, tot[f])
    s.n_sites = s.n_links_r = s.n_links_d = float(L) * L
    return orc.derive(s, beta)
