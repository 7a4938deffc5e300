"""Serving: continuous batching of PCC requests.  A request's observable
series is the same bit for bit whether it is served alone or mixed with
others that join and leave around it; admission respects the HBM budget;
oversized requests are rejected; a cancelled request frees its slot."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1210_6116_b300 as xy  # noqa: E402
from paper_1210_6116_b300 import build as xybuild  # noqa: E402
from paper_1210_6116_b300.serve import PCC, Request, Server, run_loop  # noqa: E402

xybuild.build()


def _trace():
    rng = np.random.default_rng(11)
    return [Request(k, 0.0, int(rng.choice([64, 128, 256])), int(rng.integers(60, 220)),
                    (4 << 20) + k) for k in range(10)]


def test_mix_equals_alone():
    trace = _trace()
    srv = Server(max_slots=4, tile_y=32, chunk=25)  # 4 slots: requests join and leave
    mixed = {r.rid: r for r in srv.run(trace, realtime=False).results}
    srv.close()
    alone = {r.rid: r for r in run_loop(trace, realtime=False).results}
    assert set(mixed) == set(alone) == {r.rid for r in trace}
    for rid in mixed:
        np.testing.assert_array_equal(mixed[rid].records, alone[rid].records)
        assert mixed[rid].final_beta == alone[rid].final_beta
        assert len(mixed[rid].records) == next(r.budget for r in trace if r.rid == rid)


def test_admission_respects_hbm_budget():
    trace = [Request(k, 0.0, 256, 50, 900 + k) for k in range(6)]
    probe = Server(max_slots=8, tile_y=32)
    one = probe.footprint(trace[0])
    probe.close()
    srv = Server(max_slots=8, hbm_budget=int(2.5 * one), tile_y=32, chunk=10)
    st = srv.run(trace, realtime=False)
    srv.close()
    assert len(st.results) == 6 and not st.rejected
    assert st.peak_bytes <= 2 * one  # never more than two at a time


def test_oversized_request_rejected():
    srv = Server(max_slots=2, hbm_budget=1 << 20, tile_y=32)
    st = srv.run([Request(0, 0.0, 1024, 20, 5)], realtime=False)
    srv.close()
    assert not st.results and len(st.rejected) == 1


def test_cancel_frees_the_slot():
    trace = [Request(0, 0.0, 128, 400, 70), Request(1, 0.0, 128, 40, 71)]
    srv = Server(max_slots=1, tile_y=32, chunk=20, policy="fifo")
    st = srv.run(trace, realtime=False, should_cancel=lambda req, done: req.rid == 0 and done >= 40)
    srv.close()
    res = {r.rid: r for r in st.results}
    assert res[0].cancelled and len(res[0].records) == 40
    assert not res[1].cancelled and len(res[1].records) == 40
    assert res[1].admitted >= res[0].finished - 1e-3  # admitted only once slot 0 was freed
