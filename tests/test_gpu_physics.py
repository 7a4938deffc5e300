"""Physics on the GPU against the paper's Table 1.

* fixed beta = beta_KT(L) for L = 64, 128, 256 (8 independent replicas each,
  one engine): <m^2>_L and xi_2nd(L)/L (Eq. (8), from chi(0) = N <m^2> and
  <chik>) match Table 1 and <beta Upsilon> sits at the PCC target 0.636508
  (Sec. 2);
* the paper's own PCC protocol at L = 64 (blocks of 1000 sweeps,
  dbeta = 0.0005, target 0.636508; Sec. 3) on 16 replicas: the long-run mean
  of beta reproduces beta_KT(64) = 1.09167(25).
Errors come from the spread over independent replicas; |delta| < 4 sigma.
"""
import json
import math
from pathlib import Path

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1210_6116_b300 as xy  # noqa: E402
from paper_1210_6116_b300 import build as xybuild  # noqa: E402
from paper_1210_6116_b300.pcc_study import xi_2nd  # noqa: E402

xybuild.build()
GOLDEN = json.loads((Path(__file__).resolve().parent / "golden" / "table1.json").read_text())
TARGET = GOLDEN["critical_beta_upsilon"]["value"]


def _row(L):
    return next(r for r in GOLDEN["rows"] if r["L"] == L)


def _drain(eng, slots, n_steps, chunk=4000):
    out = {s: [] for s in slots}
    done = 0
    while done < n_steps:
        k = min(chunk, n_steps - done)
        eng.step(k)
        for s in slots:
            out[s].append(eng.measure(s))
        done += k
    return {s: np.concatenate(v) for s, v in out.items()}


def test_table1_fixed_beta_small_L():
    sizes, reps = (64, 128, 256), 8
    eng = xy.Engine(len(sizes) * reps, tile_y=32)
    slots = {L: [eng.admit(eng.config(L, _row(L)["beta_kt"], 5000 + 100 * L + k,
                                      measure_xi=True))
                 for k in range(reps)] for L in sizes}
    eng.step(1000)
    for L in sizes:
        for s in slots[L]:
            eng.measure(s)
    allslots = [s for L in sizes for s in slots[L]]
    recs = _drain(eng, allslots, 12000)
    for L in sizes:
        row = _row(L)
        m2 = np.array([recs[s]["m2"].mean() for s in slots[L]])
        bu = np.array([(recs[s]["beta"] * recs[s]["upsilon"]).mean() for s in slots[L]])
        e_m2 = m2.std(ddof=1) / math.sqrt(reps)
        e_bu = bu.std(ddof=1) / math.sqrt(reps)
        assert abs(m2.mean() - row["m2"]) < 4 * math.hypot(e_m2, row["m2_err"]), (L, m2.mean(), e_m2)
        xil = np.array([xi_2nd(L * L * recs[s]["m2"].mean(), recs[s]["chik"].mean(), L) / L
                        for s in slots[L]])
        e_xi = xil.std(ddof=1) / math.sqrt(reps)
        assert abs(xil.mean() - row["xi_over_L"]) < 4 * math.hypot(e_xi, row["xi_err"]), \
            (L, xil.mean(), e_xi)
        # beta*Upsilon moves by ~1.5 x the table's beta uncertainty
        assert abs(bu.mean() - TARGET) < 4 * math.hypot(e_bu, 1.5 * row["beta_err"]), (L, bu.mean(), e_bu)


def test_paper_protocol_pcc_finds_beta_kt_64():
    L, reps = 64, 16
    pcc = xy.xy_pcc_params(target=TARGET, dbeta0=0.0005, halve_every=0, block=1000)
    eng = xy.Engine(reps, tile_y=32)
    slots = [eng.admit(eng.config(L, 1.09, 7000 + k), pcc) for k in range(reps)]
    _drain(eng, slots, 20000)                 # discarded (the paper discards 60000)
    recs = _drain(eng, slots, 100000)
    means = np.array([recs[s]["beta"].mean() for s in slots])
    err = means.std(ddof=1) / math.sqrt(reps)
    row = _row(L)
    assert abs(means.mean() - row["beta_kt"]) < 4 * math.hypot(err, row["beta_err"]), \
        (means.mean(), err)
