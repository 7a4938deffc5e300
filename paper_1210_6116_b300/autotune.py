"""Labeling-tile autotuner.

Tiles are 32 columns wide (one warp ballot word per row) and TY rows high;
TY in {16, 32, 64, 128} trades shared-memory union-find work inside a tile
against the number of tile edges merged in global memory.  The tuner times a
few sweeps of each candidate on the actual lattice (or replica table) with
CUDA events and keeps the fastest, cached per (L, dtype, threshold mode) --
for a table, per its sorted tuple of sizes.
"""
from __future__ import annotations

import json
from pathlib import Path

import numpy as np

CANDIDATES = (16, 32, 64, 128)
_CACHE_FILE = Path(__file__).resolve().parent / "tile_cache.json"
_cache: dict | None = None


def _load():
    global _cache
    if _cache is None:
        try:
            _cache = json.loads(_CACHE_FILE.read_text())
        except (OSError, ValueError):
            _cache = {}
    return _cache


def _store(key: str, value: int):
    c = _load()
    c[key] = value
    try:
        _CACHE_FILE.write_text(json.dumps(c, indent=1, sort_keys=True))
    except OSError:
        pass


def _time(fn, n: int) -> float:
    import torch

    s = torch.cuda.current_stream()
    fn(2)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(s)
    fn(n)
    e1.record(s)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / n


def best_tile(L: int, *, dtype: str = "f32", exact: bool = False, sweeps: int = 10,
              candidates=CANDIDATES, use_cache: bool = True) -> tuple[int, dict]:
    """Fastest tile height for one L x L lattice; returns (TY, {TY: ms/sweep})."""
    import paper_1210_6116_b300 as xy

    key = f"single:{L}:{dtype}:{int(exact)}"
    if use_cache and key in _load():
        return int(_load()[key]), {}
    times = {}
    for ty in candidates:
        lat = xy.Lattice(L, 1.1, 12345, dtype=dtype, exact=exact, tile_y=ty)
        times[ty] = _time(lat.sweep, sweeps)
        lat.close()
    best = min(times, key=times.get)
    _store(key, best)
    return best, times


def best_tile_table(table: list[dict], *, dtype: str = "f32", exact: bool = False,
                    sweeps: int = 5, candidates=CANDIDATES, use_cache: bool = True):
    """Fastest shared tile height for an engine running `table` (dicts with
    L, beta, seed); returns (TY, {TY: ms per engine step})."""
    import paper_1210_6116_b300 as xy

    sizes = tuple(sorted(int(r["L"]) for r in table))
    key = f"table:{hash(sizes) & 0xFFFFFFFF:08x}:{len(sizes)}:{dtype}:{int(exact)}"
    if use_cache and key in _load():
        return int(_load()[key]), {}
    times = {}
    for ty in candidates:
        eng = xy.Engine(len(table), dtype=dtype, exact=exact, tile_y=ty)
        for r in table:
            eng.admit(eng.config(r["L"], r["beta"], r["seed"]))
        times[ty] = _time(eng.step, sweeps)
        eng.close()
    best = min(times, key=times.get)
    _store(key, best)
    return best, times
