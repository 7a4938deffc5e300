"""Seeded synthetic inputs shared by the tests, the oracle checks and the bench.

This module holds no arithmetic of the method: it only draws the inputs that
both the CUDA path and the CPU oracle are fed (angle fields, bond masks for
labeling checks, replica tables and request traces).  Every generator takes an
explicit seed and uses numpy's PCG64 stream, so a test can rebuild the same
input on any host.
"""
from __future__ import annotations

import math

import numpy as np

TWO_PI_F32 = np.float32(2.0 * math.pi)


def angles(n: int, seed: int, dtype=np.float32) -> np.ndarray:
    """n angles uniform in [0, 2pi) stored as dtype: float32, float16, or
    uint16 (fixed point: theta = q 2pi / 65536, q uniform over all 65536)."""
    rng = np.random.default_rng(seed)
    if dtype == np.uint16:
        return rng.integers(0, 65536, size=n, dtype=np.uint16)
    a = rng.uniform(0.0, 2.0 * math.pi, size=n).astype(np.float32)
    a[a >= TWO_PI_F32] = 0.0
    if dtype == np.float16:
        h = a.astype(np.float16)
        h[h.astype(np.float32) >= TWO_PI_F32] = np.float16(0.0)
        return h
    return a


def ordered_angles(n: int, value: float = 0.0, dtype=np.float32) -> np.ndarray:
    return np.full(n, value, dtype=dtype)


def twisted_angles(L: int, k: int, axis: int = 0) -> np.ndarray:
    """theta(x, y) = 2 pi k x / L (axis 0) or 2 pi k y / L (axis 1), in [0, 2pi)."""
    y, x = np.mgrid[0:L, 0:L]
    c = x if axis == 0 else y
    a = ((2.0 * math.pi * k * c / L) % (2.0 * math.pi)).astype(np.float32).ravel()
    a[a >= TWO_PI_F32] = 0.0
    return a


def bond_masks(Lx: int, Ly: int, density: float, seed: int):
    """Random right/down bond bytes with the given density of active bonds."""
    rng = np.random.default_rng(seed)
    right = (rng.random(Lx * Ly) < density).astype(np.uint8)
    down = (rng.random(Lx * Ly) < density).astype(np.uint8)
    return right, down


def spiral_masks(L: int):
    """One self-avoiding path that spirals inward from the corner with a gap of
    one site between its arms: a single long cluster whose tile-local pieces
    need many merges; the gap sites stay isolated."""
    right = np.zeros(L * L, np.uint8)
    down = np.zeros(L * L, np.uint8)
    seen = np.zeros((L, L), bool)
    x, y, d = 0, 0, 0
    steps = ((1, 0), (0, 1), (-1, 0), (0, -1))
    seen[y, x] = True

    def free(cx, cy):
        return 0 <= cx < L and 0 <= cy < L and not seen[cy, cx]

    turns = 0
    while turns < 2:
        dx, dy = steps[d]
        nx, ny = x + dx, y + dy
        if free(nx, ny) and (not (0 <= nx + dx < L and 0 <= ny + dy < L) or not seen[ny + dy, nx + dx]):
            if dx == 1:
                right[y * L + x] = 1
            elif dx == -1:
                right[ny * L + nx] = 1
            elif dy == 1:
                down[y * L + x] = 1
            else:
                down[ny * L + nx] = 1
            x, y = nx, ny
            seen[y, x] = True
            turns = 0
        else:
            d = (d + 1) % 4
            turns += 1
    return right, down


def wrap_masks(L: int):
    """Clusters that only close through the periodic boundary: full rows of
    right bonds on even rows, and a column of down bonds that wraps y."""
    right = np.zeros(L * L, np.uint8)
    down = np.zeros(L * L, np.uint8)
    for y in range(0, L, 2):
        right[y * L:(y + 1) * L] = 1
    for y in range(L):
        down[y * L + (L - 1)] = 1 if y % 3 == 0 else 0
    return right, down


def replica_table(n: int, seed: int, sizes=(64, 128, 256, 512, 1024, 2048),
                  beta_range=(1.0, 1.3)):
    """Batched workload: per replica an L drawn uniformly from `sizes`, a beta
    uniform in beta_range and a distinct seed."""
    rng = np.random.default_rng(seed)
    Ls = rng.choice(np.asarray(sizes), size=n)
    betas = rng.uniform(beta_range[0], beta_range[1], size=n)
    seeds = (3 << 20) + np.arange(n)
    return [dict(L=int(L), beta=float(b), seed=int(s)) for L, b, s in zip(Ls, betas, seeds)]


def request_trace(n: int, rate: float, seed: int,
                  sizes=(128, 256, 512, 1024, 2048, 4096, 8192),
                  budget=(500, 5000)):
    """Finite Poisson request stream of PCC runs: arrival time (s), L, sweep
    budget and run seed per request, sorted by arrival."""
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate, size=n)
    arrivals = np.cumsum(gaps)
    Ls = rng.choice(np.asarray(sizes), size=n)
    budgets = rng.integers(budget[0], budget[1] + 1, size=n)
    seeds = (4 << 20) + np.arange(n)
    return [dict(arrival=float(a), L=int(L), budget=int(b), seed=int(s))
            for a, L, b, s in zip(arrivals, Ls, budgets, seeds)]
