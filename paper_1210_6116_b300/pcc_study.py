"""beta_KT(L) by the paper's helicity-modulus PCC protocol, on many replicas.

The paper (Sec. 3) runs the PCC with dbeta = 0.0005, one beta step per block
of 1000 MCS driven by the block mean of beta*Upsilon against 0.636508,
discards the first part of the run, and reports the long-run mean of beta as
beta_KT(L) together with <m^2>_L (Table 1).  This runs that protocol for
several L at once: every (L, replica) pair is one lattice of an Engine, so
all of them advance with shared launches, and the error bars come from the
spread over independent replicas.  Every lattice also records chik, so each
row carries the second-moment correlation length xi_2nd(L)/L of Eq. (8).

    python -m paper_1210_6116_b300.pcc_study [--sizes 64 128 256 512]
        [--replicas 16] [--discard 20000] [--measure 200000]
"""
from __future__ import annotations

import argparse
import json
import math
import time

import numpy as np

import paper_1210_6116_b300 as xy

TABLE1 = {  # L: (beta_KT(L), err, <m^2>_L, err, xi_2nd/L, err) -- the paper's Table 1
    64: (1.09167, 0.00025, 0.34924, 0.00029, 0.7464, 0.0011),
    128: (1.09788, 0.00032, 0.29695, 0.00036, 0.7466, 0.0015),
    256: (1.10224, 0.00021, 0.25245, 0.00028, 0.7482, 0.0009),
    512: (1.10530, 0.00026, 0.21427, 0.00027, 0.7482, 0.0014),
    1024: (1.10768, 0.00019, 0.18195, 0.00016, 0.7488, 0.0011),
    2048: (1.10966, 0.00020, 0.15443, 0.00026, 0.7491, 0.0014),
    4096: (1.11097, 0.00008, 0.13085, 0.00015, 0.7495, 0.0012),
}
TARGET = 0.636508


def xi_2nd(chi0: float, chik: float, L: int) -> float:
    """Second-moment correlation length, Eq. (8): from the run averages of
    chi(0) = N <m^2> and chi(k_min) = <chik>, k_min = 2 pi / L."""
    return math.sqrt(chi0 / chik - 1.0) / (2.0 * math.sin(math.pi / L))


def run(sizes=(64, 128, 256, 512), replicas=16, discard=20000, measure=200000,
        beta0=1.10, seed0=11 << 20, tile_y=32, chunk=4000) -> dict:
    pcc = xy.xy_pcc_params(target=TARGET, dbeta0=0.0005, halve_every=0, block=1000)
    eng = xy.Engine(len(sizes) * replicas, tile_y=tile_y)
    slots = {L: [eng.admit(eng.config(L, beta0, seed0 + 1000 * L + k, record_cap=chunk,
                                      measure_xi=True), pcc)
                 for k in range(replicas)] for L in sizes}
    allslots = [s for L in sizes for s in slots[L]]
    sums = {s: np.zeros(4) for s in allslots}  # sum beta, sum m2, sum chik, count
    t0 = time.perf_counter()
    done = 0
    while done < discard + measure:
        n = min(chunk, discard + measure - done)
        if done < discard:
            n = min(n, discard - done)
        eng.step(n)
        for s in allslots:
            r = eng.measure(s)
            if done >= discard:
                sums[s] += (r["beta"].sum(), r["m2"].sum(), r["chik"].sum(), len(r))
        done += n
    wall = time.perf_counter() - t0
    out = {"protocol": f"PCC target {TARGET}, dbeta 0.0005, block 1000 sweeps, start beta {beta0}, "
                       f"{discard} sweeps discarded, {measure} measured, {replicas} replicas per L",
           "wall_s": round(wall, 1), "sizes": {}}
    for L in sizes:
        b = np.array([sums[s][0] / sums[s][3] for s in slots[L]])
        m = np.array([sums[s][1] / sums[s][3] for s in slots[L]])
        xl = np.array([xi_2nd(L * L * sums[s][1] / sums[s][3], sums[s][2] / sums[s][3], L) / L
                       for s in slots[L]])

        def err(a):
            return round(float(a.std(ddof=1) / math.sqrt(len(a))), 5)

        row = {"beta_kt": round(float(b.mean()), 5), "beta_err": err(b),
               "m2": round(float(m.mean()), 5), "m2_err": err(m),
               "xi_over_L": round(float(xl.mean()), 5), "xi_err": err(xl)}
        if L in TABLE1:
            tb, tbe, tm, tme, tx, txe = TABLE1[L]
            row["paper"] = {"beta_kt": tb, "beta_err": tbe, "m2": tm, "m2_err": tme,
                            "xi_over_L": tx, "xi_err": txe}
            row["beta_sigma"] = round((row["beta_kt"] - tb) / math.hypot(row["beta_err"], tbe), 2)
            row["m2_sigma"] = round((row["m2"] - tm) / math.hypot(row["m2_err"], tme), 2)
            row["xi_sigma"] = round((row["xi_over_L"] - tx) / math.hypot(row["xi_err"], txe), 2)
        out["sizes"][str(L)] = row
    eng.close()
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--sizes", type=int, nargs="+", default=[64, 128, 256, 512])
    ap.add_argument("--replicas", type=int, default=16)
    ap.add_argument("--discard", type=int, default=20000)
    ap.add_argument("--measure", type=int, default=200000)
    a = ap.parse_args()
    print(json.dumps(run(tuple(a.sizes), a.replicas, a.discard, a.measure), indent=1))


if __name__ == "__main__":
    main()
