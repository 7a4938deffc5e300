"""Shared helpers of the GPU parity tests: tolerances and record comparison.

Tolerances, derived from the arithmetic of the observable kernel.  Each site
term is evaluated in FP32 from the stored angles: cos/sin of an angle with
the kernel's own routine (Cody-Waite reduction and Taylor polynomials,
<= 1e-7 absolute, measured in test_gpu_spins; the bounds below allow
1.2e-7), and a link
term cos(ti - tj) = ci cj + si sj (or si cj - ci sj) with error
<= 1.2e-7 * (|ci| + |cj| + |si| + |sj|) + 1.2e-7 <= 4.6e-7.  Every term is then
rounded to a 2^-22 grid (<= 2^-23 = 1.2e-7) and summed exactly in integers.
Per site, a link sum (e_x, s_x, e_y, s_y) is therefore within
EPS_LINK = 6e-7 of the oracle's FP64 sum / N, a site sum (m_x, m_y) within
EPS_SITE = 2.4e-7, and E/site (two links per site) within 2 EPS_LINK.
The 1e-6 relative target for the observables holds on top of these wherever the value is
O(1) (E/site ~ -1.4, e_x ~ 0.7): the test takes max(1e-6 |value|, bound).
M^2 = mx^2 + my^2 and Upsilon = e_x - beta N s_x^2 inherit the bounds by
error propagation.

chik (Eq. (9) at the smallest wave vector) is built from eight Fourier sums
F_c = sum_r {cos, sin}(theta_r) {cos, sin}(2 pi x / L).  Each term is the
product of an FP32 cos/sin (<= 1.2e-7), a wave factor rounded from FP64 to
FP32 (<= 6e-8), the product's rounding (<= 6e-8) and the 2^-22 grid
(<= 1.2e-7): EPS_WAVE = 3.6e-7 per term, so |dF_c| <= dF = EPS_WAVE N.  With
sum_c |F_c| <= sqrt(8 sum_c F_c^2) = 4 sqrt(N chik), the error of
chik = sum_c F_c^2 / (2N) is at most (4 dF sqrt(N chik) + 4 dF^2) / N.
"""
import numpy as np

REL = 1e-6
EPS_LINK = 6e-7
EPS_SITE = 2.4e-7
EPS_WAVE = 3.6e-7


def obs_close(g: dict, o: dict, N: int, beta: float, xi: bool = False, flips: bool = False):
    """Return a list of (field, gpu, oracle, tol) that violate the tolerance.
    xi: the GPU lattice measures chik; otherwise its chik must be exactly 0.
    flips: the GPU counts reflected sites (Wolff), compared exactly with the
    oracle's count; otherwise (SW) the count must be 0."""
    bad = []

    def chk(k, tol):
        if abs(g[k] - o[k]) > tol:
            bad.append((k, g[k], o[k], tol))

    chk("energy_per_site", max(REL * abs(o["energy_per_site"]), 2 * EPS_LINK))
    for k in ("ex", "ey"):
        chk(k, max(REL * abs(o[k]), EPS_LINK))
    for k in ("sx", "sy"):
        chk(k, EPS_LINK)
    for k in ("mx", "my"):
        chk(k, EPS_SITE)
    chk("m2", max(REL * o["m2"],
                  2 * (abs(o["mx"]) + abs(o["my"]) + EPS_SITE) * EPS_SITE))
    chk("upsilon", max(REL * abs(o["upsilon"]),
                       EPS_LINK + beta * N * (2 * abs(o["sx"]) + EPS_LINK) * EPS_LINK))
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
