"""Benchmark of the Swendsen-Wang XY sweep on B300: one JSON line.

A step is one full SW sweep (axis, bonds, labels, flip, observables, record)
of an L = 4096 periodic lattice (16.8M spins, FP32 angles, beta = 1.12,
Philox random start) -- the single-lattice workload the spin-updates/ns metric
is quoted on.  The working set of a sweep (two angle buffers, labels, bit
planes: 204 MB) is larger than the 126 MB L2, so sweeps run back to back
without an explicit flush.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun (N > 1) every rank runs its own independent lattice (replicas
only: the method has no data-path exchange); rank 0 prints the line.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time
from pathlib import Path

import numpy as np

ROOT = Path(__file__).resolve().parent
sys.path.insert(0, str(ROOT))

METRIC = "spin updates/ns per SW sweep (L=4096, 65536) & %HBM roofline; batched sweeps/s, p50/p99"
UNIT = "spin updates/ns"

PROFILE_EVERY = 16  # kernel-timing stride inside timed regions

# Byte models of a sweep, per site, FP32 angles (the hot-path scope's
# measurement section):
#   M_alg   the method's minimum: angles read in the bond pass (4), read and
#           written in the flip pass after global connectivity (4 + 4), bond
#           bits written and read (0.25 + 0.25)                    = 12.5
#   M_canon M_alg + one uint32 canonical label written once        = 16.5
# Each kernel's share of M_alg (the roofline of the dominant kernel is taken
# against its share): the bond + label kernel reads the angles and writes the
# bond bits, the flip kernel reads and writes the angles and (in the model)
# reads the bond bits back.
M_ALG = 4.0 + 4.0 + 4.0 + 0.25 + 0.25
M_CANON = M_ALG + 4.0
ALG_SHARE = {"bond_label": 4.0 + 0.25, "flip_measure": 4.0 + 4.0 + 0.25}
# Bytes the built pipeline moves per site (its own intermediates included):
# bond + label kernel: angles in, tile labels out, bond planes, coin bits,
# tile edge table; merge and compress ~0.5 each (upper figures); flip kernel:
# labels in, angles in and out.
BUILT_SHARE = {"bond_label": 4.0 + 4.0 + 0.25 + 0.125 + 0.375, "flip_measure": 12.0}
M_BUILT = BUILT_SHARE["bond_label"] + 0.5 + 0.5 + BUILT_SHARE["flip_measure"]


def _sm_max_mhz():
    p = ROOT / "MEASURED_PEAKS.json"
    if p.exists():
        return float(json.loads(p.read_text()).get("sm_max_mhz", 2032.0))
    return 2032.0


def _peaks():
    p = ROOT / "MEASURED_PEAKS.json"
    if p.exists():
        d = json.loads(p.read_text())
        return float(d["hbm_gbs"]), "measured"
    return 6400.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled every 200 ms from before
    the warm-up until after the timed region.  The GPU is named by its UUID
    (the process's device 0 need not be nvidia-smi's index 0).  The summary
    takes the samples inside the timed region, or, when the region is shorter
    than the sampling interval, the samples nearest to it."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None
        self.samples = []  # (monotonic time, fields)
        self.window = None
        self.error = None

    def start(self):
        import threading

        import torch

        try:
            gpu = "GPU-" + str(torch.cuda.get_device_properties(self.device).uuid)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", gpu, f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True)
        except (OSError, AssertionError, RuntimeError) as e:
            self.error = f"nvidia-smi not started: {e}"
            return self

        def reader():
            for line in self.proc.stdout:
                f = [x.strip() for x in line.split(",")]
                if len(f) >= 9:
                    self.samples.append((time.monotonic(), f))

        self.thread = threading.Thread(target=reader, daemon=True)
        self.thread.start()
        t0 = time.monotonic()
        while not self.samples and time.monotonic() - t0 < 3.0 and self.proc.poll() is None:
            time.sleep(0.02)
        return self

    def mark(self, t0: float, t1: float):
        self.window = (t0, t1)

    def stop(self):
        if self.proc is None:
            return
        time.sleep(0.25)  # one more sample after the timed region
        self.proc.terminate()
        try:
            _, err = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            _, err = self.proc.communicate()
        if not self.samples:
            self.error = "nvidia-smi gave no samples: " + (err or "").strip()[:200]

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [],
                    "error": self.error or "no samples"}
        t0, t1 = self.window or (self.samples[0][0], self.samples[-1][0])
        inside = [f for t, f in self.samples if t0 <= t <= t1]
        how = "samples inside the timed region"
        if not inside:
            near = sorted(self.samples, key=lambda s: min(abs(s[0] - t0), abs(s[0] - t1)))[:2]
            inside = [f for _, f in near]
            how = ("timed region shorter than the 200 ms sampling interval: "
                   "the samples nearest to it")

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None

        sm = [v for v in (num(f[1]) for f in inside) if v is not None]
        mx = [v for v in (num(f[2]) for f in inside) if v is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for f in inside for k in range(4)
                          if f[5 + k].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(inside), "how": how}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def aggregate(dist, ws: int, sites_per_step: int, steps: int, t_local: float, device=None):
    """Whole-job rate over ranks: every rank ran `steps` sweeps of its own
    lattice; the job takes as long as the slowest rank (max over ranks).
    dist is torch.distributed (or None for one rank)."""
    t = t_local
    if dist is not None and ws > 1:
        import torch

        tt = torch.tensor([t_local], dtype=torch.float64, device=device)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        t = float(tt.item())
    return ws * sites_per_step * steps / (t * 1e9), t


def run_ours(args):
    import torch

    import paper_1210_6116_b300 as xy
    from paper_1210_6116_b300 import build as xybuild

    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    pg = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
        pg = dist
    if rank == 0:
        xybuild.build()
    if pg:
        pg.barrier()
    L, beta = args.L, args.beta
    N = L * L
    clk = ClockSampler(local).start()
    lat = xy.Lattice(L, beta, seed=1000 + rank, tile_y=args.tile_y, exact=bool(args.exact))
    stream = lat.stream
    lat.sweep(args.warmup)
    lat.measure(max_records=0)
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    if pg:
        pg.barrier()
    torch.cuda.synchronize()

    def sweeps():
        done = 0
        while done < args.steps:
            n = min(1024, args.steps - done)
            lat.sweep(n)
            done += n

    # the timed region: the sweeps exactly as a caller runs them
    t_start = time.monotonic()
    ev0.record(stream)
    sweeps()
    ev1.record(stream)
    torch.cuda.synchronize()
    clk.mark(t_start, time.monotonic())
    if pg:
        pg.barrier()
    ms = ev0.elapsed_time(ev1)
    recs = lat.measure()
    # kernel durations: a second window of as many sweeps, with CUDA events
    # around the kernels of every 16th sweep (events between a sweep's kernels
    # cost it ~12 us, and a timed sweep is launched directly, not replayed
    # from xy_sweep's chunk graph, so the window runs slower than the first)
    lat.profile(True, every=PROFILE_EVERY)
    evp0 = torch.cuda.Event(enable_timing=True)
    evp1 = torch.cuda.Event(enable_timing=True)
    evp0.record(stream)
    sweeps()
    evp1.record(stream)
    torch.cuda.synchronize()
    kt = lat.profile_read()
    lat.profile(False)
    lat.measure(max_records=0)
    ms_prof = evp0.elapsed_time(evp1)
    value, t_sec = aggregate(pg, ws, N, args.steps, ms / 1e3, device="cuda")
    ms_per_step = t_sec * 1e3 / args.steps
    launches = (xy.LAUNCHES_PER_SWEEP * args.steps
                + xy.LAUNCHES_PER_CALL * math.ceil(args.steps / 1024))

    out = None
    if rank == 0:
        peak, peak_kind = _peaks()
        # dominant kernel, against its share of the method's bytes (M_alg)
        dom = max(ALG_SHARE, key=lambda k: kt[k][0])
        dms = kt[dom][0] / kt[dom][1]
        achieved = ALG_SHARE[dom] * N / (dms * 1e-3) / 1e9
        achieved_built = BUILT_SHARE[dom] * N / (dms * 1e-3) / 1e9
        tot = sum(x[0] for x in kt.values())
        kernels = {k: {"ms_per_launch": round(v[0] / v[1], 5), "share": round(v[0] / tot, 4)}
                   for k, v in kt.items() if v[1]}
        traffic, alu = _traffic_and_alu(dom, L, dms)
        out = {
            "metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_per_step, 5),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic",
            "config": bench_config(args, ws),
            "roofline": {"bound": "hbm", "kernel": dom, "achieved": round(achieved, 1),
                         "peak": peak, "peak_kind": f"{peak_kind} (burst copy; of measured)",
                         "unit": "GB/s", "frac": round(achieved / peak, 4), "traffic": traffic,
                         "bytes_per_site": ALG_SHARE[dom],
                         "model": "the kernel's share of M_alg (angles in, bond bits out)",
                         "achieved_built_bytes": round(achieved_built, 1),
                         "frac_built_bytes": round(achieved_built / peak, 4),
                         "built_bytes_per_site": BUILT_SHARE[dom]},
            "roofline_alu": alu,
            "sweep_roofline": {"M_alg_B_per_site": M_ALG, "M_canon_B_per_site": M_CANON,
                               "M_built_B_per_site": M_BUILT,
                               "frac_alg": round(value / ws * M_ALG / peak, 4),
                               "frac_canon": round(value / ws * M_CANON / peak, 4),
                               "frac_built": round(value / ws * M_BUILT / peak, 4)},
            "kernels": kernels,
            "kernel_timing": (f"CUDA events around the kernels of every {PROFILE_EVERY}th sweep of a "
                              f"second window of {args.steps} sweeps right after the timed region"),
            "profiled_window": {"value": round(N * args.steps / (ms_prof * 1e6), 3), "unit": UNIT,
                                "ms_per_step": round(ms_prof / args.steps, 5)},
            "gpu_launches": launches,
            "last_energy_per_site": float(recs[-1]["energy_per_site"]) if len(recs) else None,
        }
    # end to end through the C ABI with pinned host buffers
    e2e = run_e2e(lat, args, N, pg, ws)
    clk.stop()
    if rank == 0:
        out["clocks"] = clk.summary()
        out["e2e"] = e2e
        # the single-GPU reports run at N = 1 only (under torchrun the other
        # ranks would hold their GPUs at the final barrier meanwhile)
        extras = ws == 1
        if args.protocol and extras:
            out["cfg1_protocol"] = run_cfg1_protocol(xy, args)
        if args.exact_report and extras:
            out["exact_mode"] = exact_report(xy, L, beta, args)
            out["storage"] = storage_report(xy, L, beta, args)
            out["wolff"] = wolff_report(xy, L, beta, args)
            out["wolff"]["sw_reflected_sites_per_ns"] = round(0.5 * value / ws, 3)
        if args.big and extras:
            out["l65536"] = run_big(xy, args)
        if args.batched and extras:
            out["batched"] = run_batched(xy, args)
        if args.precision and extras:
            out["precision"] = run_precision(xy, args)
        if args.serving and extras:
            out["serving"] = run_serving(xy, args)
        if not args.no_cpu and extras:
            out["cpu_baseline"] = cpu_baseline(args)
        print(json.dumps(out), flush=True)
    lat.close()
    if pg:
        pg.barrier()
        pg.destroy_process_group()


def _traffic_and_alu(dom: str, L: int, dms: float):
    """DRAM bytes per launch of the dominant kernel (ncu, profiles/traffic.json)
    and its executed instructions against the issue ceiling, while the kernel
    source is the one the capture was taken from (else null)."""
    import hashlib

    tfile = ROOT / "profiles" / "traffic.json"
    if not tfile.exists():
        return None, None
    tj = json.loads(tfile.read_text())
    src = ROOT / "paper_1210_6116_b300" / "csrc" / "sweep_kernels.cuh"
    same = hashlib.sha256(src.read_bytes()).hexdigest()[:16] == tj.get("kernels_source_sha256_16")
    if not (same and tj.get("kernel") == dom and tj.get("L") == L):
        return None, None
    traffic = tj.get("bytes_per_launch")
    alu = None
    if tj.get("thread_inst_per_launch"):
        # instruction issue ceiling: 148 SMs x 4 schedulers x 32 lanes x SM clock
        peak_ti = 148 * 4 * 32 * _sm_max_mhz() * 1e6 / 1e12
        ach_ti = tj["thread_inst_per_launch"] / (dms * 1e-3) / 1e12
        alu = {"bound": "alu", "kernel": dom, "achieved": round(ach_ti, 2),
               "peak": round(peak_ti, 2), "unit": "T thread-instructions/s",
               "frac": round(ach_ti / peak_ti, 4),
               "thread_inst_per_launch": tj["thread_inst_per_launch"],
               "how": "executed instructions from the ncu capture in profiles/, "
                      "duration from this run's CUDA events"}
    return traffic, alu


def run_cfg1_protocol(xy, args):
    """The L = 4096 workload's own protocol: beta in {1.10, 1.12, 1.14}, each
    on a fresh lattice (seed 1000 + k) thermalised by 10^3 sweeps, then five
    windows of 10^3 sweeps timed with CUDA events; the rate is the median of
    the windows."""
    import torch

    L, N = args.L, args.L * args.L
    out = {"L": L, "thermalisation_sweeps": args.therm, "windows": args.windows,
           "window_sweeps": args.window_sweeps, "thresholds": "fp64-exact" if args.exact else "fp32"}
    per_beta = {}
    for k, beta in enumerate((1.10, 1.12, 1.14)):
        lat = xy.Lattice(L, beta, seed=1000 + k, tile_y=args.tile_y, exact=bool(args.exact))
        lat.sweep(args.therm)
        lat.measure(max_records=0)
        rates = []
        for _ in range(args.windows):
            t = _event_time(lambda: lat.sweep(args.window_sweeps), lat.stream)
            rates.append(N * args.window_sweeps / (t * 1e9))
        recs = lat.measure()
        per_beta[f"{beta:.2f}"] = {
            "median_updates_per_ns": round(statistics.median(rates), 3),
            "windows_updates_per_ns": [round(r, 3) for r in rates],
            "mean_energy_per_site": round(float(recs["energy_per_site"].mean()), 6),
            "mean_beta_upsilon": round(float((recs["beta"] * recs["upsilon"]).mean()), 5)}
        lat.close()
    out["per_beta"] = per_beta
    out["median_updates_per_ns"] = round(statistics.median(
        v["median_updates_per_ns"] for v in per_beta.values()), 3)
    return out


def run_e2e(lat, args, N, dist=None, ws: int = 1):
    """The metric through the public API with host buffers: every step copies
    its input angles from pinned host memory, sweeps once and copies the
    sweep's record back.  Two lattices on their own streams alternate
    (xy_run_host_async, at most two steps in flight), so one step's copy
    overlaps the other's sweep, as a user after throughput would run it."""
    import numpy as np
    import torch

    import paper_1210_6116_b300 as xy

    n_steps = max(4, min(args.e2e_steps, args.steps))
    lats = [xy.Lattice(args.L, args.beta, seed=2000 + k, tile_y=args.tile_y, exact=bool(args.exact),
                       stream=torch.cuda.Stream()) for k in range(2)]
    angles = lat.get_angles()
    ins, outs, keep = [], [], []
    for k in range(2):
        h_in = torch.empty(N, dtype=torch.float32, pin_memory=True)
        h_in.numpy()[:] = angles
        h_out = torch.empty(xy.OBS_DTYPE.itemsize, dtype=torch.uint8, pin_memory=True)
        keep += [h_in, h_out]
        ins.append(h_in.numpy())
        outs.append(h_out.numpy().view(xy.OBS_DTYPE))
    for k in range(2):  # warm
        lats[k].run_host(ins[k], 1, outs[k])
    t0 = time.perf_counter()
    for step in range(n_steps):
        k = step & 1
        if step >= 2:
            lats[k].sync()  # step - 2 on this lattice is done
        lats[k].run_host_async(ins[k], 1, outs[k])
    for k in range(2):
        lats[k].sync()
    elapsed = time.perf_counter() - t0
    for x in lats:
        x.close()
    # whole job: every rank ran n_steps steps of its own lattices at once;
    # the job takes as long as the slowest rank
    value, _ = aggregate(dist, ws, N, n_steps, elapsed, device="cuda")
    return {"value": round(value, 3), "unit": UNIT, "h2d_bytes_per_step": 4 * N * ws,
            "d2h_bytes_per_step": int(xy.OBS_DTYPE.itemsize) * ws, "steps": n_steps,
            "how": "xy_run_host_async per step on two alternating lattices per rank (own streams, "
                   "at most two steps in flight): pinned host angles in, one sweep, the sweep's "
                   "record out; bytes counted over all ranks"}


def exact_report(xy, L, beta, args):
    import torch

    lat = xy.Lattice(L, beta, seed=4242, tile_y=args.tile_y, exact=True)
    lat.sweep(5)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    n = max(20, min(200, args.steps))
    e0.record(lat.stream)
    lat.sweep(n)
    e1.record(lat.stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / n
    n64, wrong = lat.band_stats()
    bonds = 2 * L * L * (n + 5)
    lat.close()
    return {"value": round(L * L / (ms * 1e6), 3), "unit": UNIT, "ms_per_step": round(ms, 5),
            "fp64_band_fraction": n64 / bonds, "fp32_bond_mismatch_rate": wrong / bonds}


def storage_report(xy, L, beta, args):
    """The same sweep (FP32 thresholds) with FP32, FP16 and u16 angle
    storage: rate and per-kernel times at the benchmark size."""
    import torch

    out = {}
    n = max(20, min(200, args.steps))
    for dt in ("f32", "f16", "u16"):
        lat = xy.Lattice(L, beta, seed=4343, tile_y=args.tile_y, exact=bool(args.exact), dtype=dt)
        lat.sweep(5)
        torch.cuda.synchronize()
        lat.profile(True, every=PROFILE_EVERY)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(lat.stream)
        lat.sweep(n)
        e1.record(lat.stream)
        torch.cuda.synchronize()
        kt = lat.profile_read()
        lat.profile(False)
        ms = e0.elapsed_time(e1) / n
        out[dt] = {"value": round(L * L / (ms * 1e6), 3), "unit": UNIT, "ms_per_step": round(ms, 5),
                   "bytes_per_angle": {"f32": 4, "f16": 2, "u16": 2}[dt],
                   "kernels_ms": {k: round(v[0] / v[1], 4) for k, v in kt.items() if v[1]}}
        lat.close()
    return out


def wolff_report(xy, L, beta, args):
    """Wolff single-cluster updates at the benchmark size: update rate, mean
    cluster fraction and reflected sites per ns, beside the SW sweep's
    (which reflects N/2 sites on average)."""
    import torch

    # equilibrate with SW sweeps first: from a random start a single-cluster
    # update reflects only a few sites, and L^2 / <|C|> updates make a sweep
    sw = xy.Lattice(L, beta, seed=4545, tile_y=args.tile_y, exact=bool(args.exact))
    sw.sweep(300)
    eq = sw.get_angles()
    sw.close()
    lat = xy.Lattice(L, beta, seed=4546, tile_y=args.tile_y, exact=bool(args.exact),
                     update="wolff", record_cap=4096)
    lat.set_angles(eq)
    lat.sweep(20)
    torch.cuda.synchronize()
    lat.measure()
    n = max(20, min(400, args.steps))
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(lat.stream)
    lat.sweep(n)
    e1.record(lat.stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / n
    frac = float(lat.measure()["flipped"].mean()) / (L * L)
    lat.close()
    return {"updates_per_s": round(1e3 / ms, 1), "ms_per_update": round(ms, 5),
            "mean_cluster_fraction": round(frac, 6),
            "reflected_sites_per_ns": round(frac * L * L / (ms * 1e6), 3),
            "how": f"L={L}, beta={beta}, from 300 SW sweeps, {n} updates after 20; cluster "
                   "found by the sweep's bond and label kernels (one launch set per update)"}


def run_big(xy, args):
    """L = 65536 (2^32 spins, the paper's largest lattice): 100 sweeps timed
    from the ordered start at beta = 1.1199 (the workload as specified), then,
    after --big-therm more sweeps, another timed window on the thermalised
    lattice, whose clusters have the equilibrium structure."""
    import torch

    L = 65536
    free, total = torch.cuda.mem_get_info()
    cfg_bytes = xy.xy_workspace_size(xy.xy_config(L=L, tile_y=args.tile_y, seed=2, beta=1.1199,
                                                  angle_dtype=0, threshold_mode=args.exact,
                                                  start=1, record_cap=0))
    if cfg_bytes > 0.9 * free:
        return {"skipped": f"needs {cfg_bytes/1e9:.1f} GB, {free/1e9:.1f} GB free"}
    lat = xy.Lattice(L, 1.1199, seed=2, start="ordered", tile_y=args.tile_y, exact=bool(args.exact))
    peak, _ = _peaks()

    def window(n):
        lat.profile(True, every=max(1, n // 10))
        t = _event_time(lambda: lat.sweep(n), lat.stream)
        kt = lat.profile_read()
        lat.profile(False)
        recs = lat.measure()
        v = L * L * n / (t * 1e9)
        return {"value": round(v, 3), "unit": UNIT, "ms_per_step": round(t * 1e3 / n, 4), "steps": n,
                "frac_alg": round(v * M_ALG / peak, 4), "frac_canon": round(v * M_CANON / peak, 4),
                "frac_built": round(v * M_BUILT / peak, 4),
                "kernels_ms": {k: round(val[0] / val[1], 4) for k, val in kt.items() if val[1]},
                "mean_energy_per_site": round(float(recs["energy_per_site"].mean()), 6),
                "last_m2": float(recs[-1]["m2"])}

    out = {"L": L, "beta": 1.1199, "start": "ordered", "seed": 2,
           "workspace_GB": round(cfg_bytes / 1e9, 2),
           "bytes_per_sweep_M_alg": M_ALG * L * L, "bytes_per_sweep_M_canon": M_CANON * L * L}
    out["from_ordered_start"] = window(args.big_steps)
    if args.big_therm > 0:
        lat.sweep(args.big_therm)
        lat.measure(max_records=0)
        out["thermalised"] = window(args.big_steps)
        out["thermalised"]["after_sweeps"] = args.big_steps + args.big_therm
    lat.close()
    del lat
    torch.cuda.empty_cache()
    out["value"] = out["from_ordered_start"]["value"]
    return out


def _event_time(fn, stream):
    import torch

    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / 1e3


def run_batched(xy, args):
    """256 independent replicas (L from {64..2048}, beta ~ U[1.0, 1.3]) advanced
    by one launch per kernel per sweep for all of them (CUDA graph replay),
    tile autotuned per table; against the same replicas run one at a time."""
    import torch

    import synth
    from paper_1210_6116_b300 import autotune

    table = synth.replica_table(args.replicas, seed=3)
    n_sites = sum(r["L"] ** 2 for r in table)
    out = {"replicas": len(table), "sizes": "L uniform over {64,128,256,512,1024,2048}",
           "beta": "uniform [1.0, 1.3]", "sites_per_step": n_sites, "sweeps": args.batch_sweeps}
    stream = torch.cuda.current_stream()
    for dtype in ("f32", "f16"):
        ty, times = autotune.best_tile_table(table, dtype=dtype, sweeps=3, use_cache=False)
        eng = xy.Engine(len(table), dtype=dtype, tile_y=ty)
        slots = [eng.admit(eng.config(r["L"], r["beta"], r["seed"])) for r in table]
        eng.step(3)
        t = _event_time(lambda: eng.step(args.batch_sweeps), stream)
        e_mean = float(np.mean([eng.measure(s_)[-1]["energy_per_site"] for s_ in slots]))
        out[dtype] = {"tile": f"32x{ty}", "autotune_ms_per_step": {str(k): round(v, 4) for k, v in times.items()},
                      "replica_sweeps_per_s": round(len(table) * args.batch_sweeps / t, 1),
                      "updates_per_ns": round(n_sites * args.batch_sweeps / (t * 1e9), 3),
                      "ms_per_step": round(t * 1e3 / args.batch_sweeps, 4),
                      "mean_final_energy_per_site": round(e_mean, 6)}
        eng.close()
        del eng
        torch.cuda.empty_cache()
    # the second reading of the size set: multiples of 64 from 64 to 2048
    # (32 sizes, most not powers of two), FP32, the same replica count
    table64 = synth.replica_table(args.replicas, seed=3, sizes=tuple(range(64, 2049, 64)))
    n64 = sum(r["L"] ** 2 for r in table64)
    ty, _ = autotune.best_tile_table(table64, dtype="f32", sweeps=3, use_cache=False)
    eng = xy.Engine(len(table64), dtype="f32", tile_y=ty)
    for r in table64:
        eng.admit(eng.config(r["L"], r["beta"], r["seed"]))
    eng.step(3)
    t = _event_time(lambda: eng.step(args.batch_sweeps), stream)
    out["f32_step64_sizes"] = {"sizes": "L uniform over {64, 128, 192, ..., 2048}", "tile": f"32x{ty}",
                               "sites_per_step": n64,
                               "replica_sweeps_per_s": round(len(table64) * args.batch_sweeps / t, 1),
                               "updates_per_ns": round(n64 * args.batch_sweeps / (t * 1e9), 3),
                               "ms_per_step": round(t * 1e3 / args.batch_sweeps, 4)}
    eng.close()
    del eng
    torch.cuda.empty_cache()
    # per-request loop: the same replicas, one lattice at a time
    n_base = args.batch_base_sweeps
    total = 0.0
    lats = []
    for r in table:
        lat = xy.Lattice(r["L"], r["beta"], r["seed"], tile_y=32 if r["L"] <= 256 else 64)
        lat.sweep(2)
        total += _event_time(lambda: lat.sweep(n_base), stream)
        lat.close()
    out["per_request_loop"] = {"replica_sweeps_per_s": round(len(table) * n_base / total, 1),
                               "updates_per_ns": round(n_sites * n_base / (total * 1e9), 3),
                               "sweeps_per_replica": n_base, "dtype": "f32"}
    out["speedup_vs_loop_f32"] = round(out["f32"]["replica_sweeps_per_s"]
                                       / out["per_request_loop"]["replica_sweeps_per_s"], 2)
    return out


def run_serving(xy, args):
    """Poisson stream of PCC requests (finite, seeded): continuous batching in
    the engine against the plain one-at-a-time loop on the same trace."""
    import synth
    from paper_1210_6116_b300.serve import Request, Server, run_loop

    trace = [Request(k, r["arrival"], r["L"], r["budget"], r["seed"])
             for k, r in enumerate(synth.request_trace(args.requests, args.rate, seed=4))]
    out = {"trace": f"{len(trace)} requests, Poisson rate {args.rate}/s, L log-uniform over "
                    "{128..8192} (powers of 2), budget uniform 500..5000 sweeps, PCC from "
                    "beta=1.0, dbeta 0.01 halved every 500 sweeps, target 2/pi",
           "offered_updates_per_ns": round(sum(r.L * r.L * r.budget for r in trace)
                                           / (trace[-1].arrival * 1e9), 3)}
    for policy in ("small-first", "fifo"):
        srv = Server(max_slots=64, chunk=args.serve_chunk, policy=policy)
        st = srv.run(trace, realtime=True)
        srv.close()
        out[f"server_{policy}"] = st.summary()
    out["per_request_loop"] = run_loop(trace, realtime=True).summary()
    return out


def run_precision(xy, args):
    """Observable shift of FP32 thresholds and of FP16 and u16 angle storage
    against the exact (FP64-threshold) mode on the same seeds, and the FP32
    bond mismatch rate measured by exact mode."""
    import numpy as np

    L, beta, n = args.prec_L, 1.12, args.prec_sweeps
    res = {}
    for name, kw in (("exact_f32", dict(exact=True)), ("thr_f32", dict(exact=False)),
                     ("thr_f32_f16", dict(exact=False, dtype="f16")),
                     ("thr_f32_u16", dict(exact=False, dtype="u16"))):
        lat = xy.Lattice(L, beta, 2024, **kw)
        lat.sweep(200)
        lat.measure()
        lat.sweep(n)
        r = lat.measure()
        if name == "exact_f32":
            n64, wrong = lat.band_stats()
            res["fp32_bond_mismatch_rate"] = wrong / (2.0 * L * L * (n + 200))
        lat.close()
        stats = {}
        for f, x in (("energy_per_site", r["energy_per_site"]), ("m2", r["m2"]),
                     ("beta_upsilon", r["beta"] * r["upsilon"])):
            nb = 20
            blocks = x[: len(x) // nb * nb].reshape(nb, -1).mean(axis=1)
            stats[f] = (float(blocks.mean()), float(blocks.std(ddof=1) / np.sqrt(nb)))
        res[name] = {f: {"mean": round(m, 8), "err": round(e, 8)} for f, (m, e) in stats.items()}
    for name in ("thr_f32", "thr_f32_f16", "thr_f32_u16"):
        res[name]["shift_vs_exact"] = {
            f: round(res[name][f]["mean"] - res["exact_f32"][f]["mean"], 8)
            for f in ("energy_per_site", "m2", "beta_upsilon")}
    res["config"] = f"L={L}, beta={beta}, {n} sweeps after 200, binned errors (20 bins)"
    return res


def cpu_baseline(args):
    """The oracle as it stands on the host cores: its OpenMP build on every
    core (bonds, flip and observables parallel, labeling sequential) over
    --cpu-sweeps sweeps of the benchmark lattice, and beside it the plain
    single-threaded oracle over one sweep."""
    import oracle

    oracle.build()
    L = args.L
    cores = os.cpu_count() or 1
    threads = oracle.omp_threads(cores)
    th = oracle.init_angles(L, 1000, 0)
    n = args.cpu_sweeps
    t0 = time.perf_counter()
    oracle.sw_run(th, L, L, args.beta, 1000, 0, n, omp=True)
    dt = time.perf_counter() - t0
    th1 = oracle.init_angles(L, 1000, 0)
    t1 = time.perf_counter()
    oracle.sw_run(th1, L, L, args.beta, 1000, 0, 1)
    dt1 = time.perf_counter() - t1
    return {"value": round(n * L * L / (dt * 1e9), 6), "unit": UNIT, "cores": threads,
            "kind": "oracle",
            "sample": f"{n} sweeps of the L={L} lattice (beta={args.beta}) from the random start, "
                      f"{dt:.1f} s, OpenMP build on {threads} threads (labeling sequential)",
            "single_thread": {"value": round(L * L / (dt1 * 1e9), 6), "unit": UNIT, "cores": 1,
                              "sample": f"1 sweep of the same lattice, {dt1:.1f} s"},
            "host_cores_available": cores}


def bench_config(args, ws: int) -> dict:
    """The workload both arms report and time (the reference arm runs it on
    the host cores, see its cpu_baseline)."""
    L, N = args.L, args.L * args.L
    return {"workload": f"SW sweep, 2D XY, L={L} periodic ({N} spins), beta={args.beta}, "
                        "FP32 angles, Philox random start",
            "L": L, "beta": args.beta, "tile": f"32x{args.tile_y or 'auto'}",
            "thresholds": "fp64-exact" if args.exact else "fp32",
            "parallelism": f"replicas x{ws}",
            "l2": (f"working set {N * 12.75 / 1e6:.0f} MB > 126 MB L2; no flush"
                   if N * 12.75 > 126e6 else
                   f"working set {N * 12.75 / 1e6:.1f} MB fits in L2; sweeps back to back")}


def run_reference(args):
    """The oracle timed as the reference arm (rank 0 only): its OpenMP build
    on all host cores, one sweep of the benchmark lattice (L = --L) per
    step -- the same workload and steps as the GPU arm."""
    ws, rank, _ = _dist()
    if rank != 0:
        return
    import oracle

    oracle.build()
    L = args.L
    cores = os.cpu_count() or 1
    threads = oracle.omp_threads(cores)
    th = oracle.init_angles(L, 1000, 0)
    oracle.sw_run(th, L, L, args.beta, 1000, 0, args.warmup, record=False, omp=True)
    t0 = time.perf_counter()
    oracle.sw_run(th, L, L, args.beta, 1000, args.warmup, args.steps, record=False, omp=True)
    dt = time.perf_counter() - t0
    v = args.steps * L * L / (dt * 1e9)
    sample = (f"{args.steps} timed sweeps of the L={L} lattice (beta={args.beta}) after "
              f"{args.warmup} warm-up sweeps, one sweep per step; OpenMP build on {threads} "
              "threads (labeling sequential)")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": round(v, 6), "unit": UNIT, "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(dt * 1e3 / args.steps, 4),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": bench_config(args, ws),
        "cpu_baseline": {"value": round(v, 6), "unit": UNIT, "cores": threads, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": round(v, 6), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=100)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--L", type=int, default=4096)
    ap.add_argument("--beta", type=float, default=1.12)
    ap.add_argument("--tile-y", dest="tile_y", type=int, default=64)
    ap.add_argument("--exact", type=int, default=0)
    ap.add_argument("--e2e-steps", dest="e2e_steps", type=int, default=50)
    ap.add_argument("--cpu-sweeps", dest="cpu_sweeps", type=int, default=8)
    ap.add_argument("--big-steps", dest="big_steps", type=int, default=100)
    ap.add_argument("--big-therm", dest="big_therm", type=int, default=200)
    ap.add_argument("--therm", type=int, default=1000)
    ap.add_argument("--windows", type=int, default=5)
    ap.add_argument("--window-sweeps", dest="window_sweeps", type=int, default=1000)
    ap.add_argument("--no-protocol", dest="protocol", action="store_false")
    ap.add_argument("--no-big", dest="big", action="store_false")
    ap.add_argument("--no-batched", dest="batched", action="store_false")
    ap.add_argument("--no-precision", dest="precision", action="store_false")
    ap.add_argument("--no-serving", dest="serving", action="store_false")
    ap.add_argument("--requests", type=int, default=24)
    ap.add_argument("--rate", type=float, default=50.0)
    ap.add_argument("--serve-chunk", dest="serve_chunk", type=int, default=100)
    ap.add_argument("--replicas", type=int, default=256)
    ap.add_argument("--batch-sweeps", dest="batch_sweeps", type=int, default=500)
    ap.add_argument("--batch-base-sweeps", dest="batch_base_sweeps", type=int, default=100)
    ap.add_argument("--prec-L", dest="prec_L", type=int, default=256)
    ap.add_argument("--prec-sweeps", dest="prec_sweeps", type=int, default=4000)
    ap.add_argument("--no-cpu", dest="no_cpu", action="store_true")
    ap.add_argument("--no-exact-report", dest="exact_report", action="store_false")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
