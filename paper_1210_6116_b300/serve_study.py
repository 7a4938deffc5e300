"""Serving study on the PCC request workload: a finite seeded Poisson trace
of helicity-modulus PCC runs (L over {128, ..., 8192}, sweep budget uniform
in 500..5000, beta from 1.0, dbeta 0.01 halved every 500 sweeps, target
2/pi), served by the continuous-batching Server and by the plain
one-request-at-a-time loop on the same GPU.

    python -m paper_1210_6116_b300.serve_study [--requests 400] [--rates 2,5,10,20,50]
        [--sweep-requests 100] [--out FILE]

The full trace (400 requests at 50/s) is served once by each; then the
arrival rate is swept over --rates with the first --sweep-requests requests
of a trace of that rate, to show where the p99 latency of each diverges.
Every result is one JSON object per line.
"""
from __future__ import annotations

import argparse
import json
import sys

import synth
from paper_1210_6116_b300.serve import Request, Server, run_loop


def trace(n: int, rate: float, seed: int = 4):
    return [Request(k, r["arrival"], r["L"], r["budget"], r["seed"])
            for k, r in enumerate(synth.request_trace(n, rate, seed=seed))]


def offered(tr) -> float:
    """Offered load of a trace in spin updates/ns."""
    return sum(r.L * r.L * r.budget for r in tr) / (tr[-1].arrival * 1e9)


def serve_both(tr, chunk: int) -> dict:
    srv = Server(max_slots=64, chunk=chunk, policy="small-first")
    s = srv.run(tr, realtime=True).summary()
    srv.close()
    loop = run_loop(tr, realtime=True).summary()
    return {"server_small_first": s, "per_request_loop": loop,
            "sweeps_per_s_ratio": round(s["sweeps_per_s"] / loop["sweeps_per_s"], 3),
            "p99_ratio_loop_over_server": round(loop["p99_latency_s"] / s["p99_latency_s"], 3)}


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--requests", type=int, default=400)
    ap.add_argument("--rate", type=float, default=50.0)
    ap.add_argument("--rates", default="2,5,10,20,50")
    ap.add_argument("--sweep-requests", dest="sweep_requests", type=int, default=100)
    ap.add_argument("--chunk", type=int, default=100)
    ap.add_argument("--out", default=None)
    args = ap.parse_args(argv)
    out = open(args.out, "w") if args.out else sys.stdout

    def emit(d):
        print(json.dumps(d), file=out, flush=True)

    tr = trace(args.requests, args.rate)
    emit({"trace": f"{len(tr)} requests, Poisson rate {args.rate}/s (seed 4)",
          "offered_updates_per_ns": round(offered(tr), 3), **serve_both(tr, args.chunk)})
    for rate in (float(x) for x in args.rates.split(",") if x):
        tr = trace(args.requests, rate)[: args.sweep_requests]
        emit({"trace": f"first {len(tr)} requests of a Poisson trace at {rate}/s (seed 4)",
              "rate": rate, "offered_updates_per_ns": round(offered(tr), 3),
              **serve_both(tr, args.chunk)})


if __name__ == "__main__":
    main()
