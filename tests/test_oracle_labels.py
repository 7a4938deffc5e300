"""Pins of the oracle's cluster labeling (step 3 of the sweep).

The label of a site is the minimum site index of its connected component over
the active bonds.  BFS and union-find are two independent copies inside the
oracle; networkx's connected_components is an outside library routine for the
same definition.  Exhaustive enumeration covers every bond mask of the 2x2 and
3x3 periodic lattices.
"""
import itertools

import networkx as nx
import numpy as np
import pytest

import synth


def _nx_labels(right, down, Lx, Ly, per_x=1, per_y=1):
    g = nx.MultiGraph()
    n = Lx * Ly
    g.add_nodes_from(range(n))
    for i in range(n):
        x, y = i % Lx, i // Lx
        if right[i] and (x + 1 < Lx or per_x):
            g.add_edge(i, y * Lx + (x + 1) % Lx)
        if down[i] and (y + 1 < Ly or per_y):
            g.add_edge(i, ((y + 1) % Ly) * Lx + x)
    lab = np.zeros(n, np.uint32)
    for comp in nx.connected_components(g):
        m = min(comp)
        for i in comp:
            lab[i] = m
    return lab


@pytest.mark.parametrize("L", [4, 5, 8, 16, 17, 64])
@pytest.mark.parametrize("density", [0.0, 0.3, 0.5, 0.7, 1.0])
def test_bfs_matches_networkx(orc, L, density):
    right, down = synth.bond_masks(L, L, density, seed=1000 * L + int(density * 10))
    bfs, comps = orc.label_bfs(right, down, L, L)
    ref = _nx_labels(right, down, L, L)
    np.testing.assert_array_equal(bfs, ref)
    assert comps == len(np.unique(ref))
    uf, comps_uf = orc.label_uf(right, down, L, L)
    np.testing.assert_array_equal(uf, bfs)
    assert comps_uf == comps


@pytest.mark.parametrize("L", [9, 16, 33])
def test_structured_masks(orc, L):
    for right, down in (synth.spiral_masks(L), synth.wrap_masks(L)):
        bfs, _ = orc.label_bfs(right, down, L, L)
        np.testing.assert_array_equal(bfs, _nx_labels(right, down, L, L))
        uf, _ = orc.label_uf(right, down, L, L)
        np.testing.assert_array_equal(uf, bfs)


def test_open_boundaries_and_rectangles(orc):
    for Lx, Ly, px, py in [(7, 3, 0, 0), (5, 9, 1, 0), (64, 1, 0, 0), (6, 4, 0, 1)]:
        right, down = synth.bond_masks(Lx, Ly, 0.6, seed=Lx * 31 + Ly)
        bfs, _ = orc.label_bfs(right, down, Lx, Ly, px, py)
        np.testing.assert_array_equal(bfs, _nx_labels(right, down, Lx, Ly, px, py))


def test_exhaustive_2x2_vs_networkx(orc):
    L = 2
    for bits in range(1 << 8):
        m = np.array([(bits >> k) & 1 for k in range(8)], np.uint8)
        right, down = m[:4].copy(), m[4:].copy()
        bfs, _ = orc.label_bfs(right, down, L, L)
        np.testing.assert_array_equal(bfs, _nx_labels(right, down, L, L))


def test_exhaustive_3x3_bfs_vs_uf(orc):
    """All 2^18 masks of the 3x3 periodic lattice: BFS == union-find, and a
    sample against networkx."""
    L = 3
    rng = np.random.default_rng(7)
    sample = set(rng.integers(0, 1 << 18, size=300).tolist())
    for bits in range(1 << 18):
        m = ((bits >> np.arange(18)) & 1).astype(np.uint8)
        right, down = m[:9].copy(), m[9:].copy()
        bfs, _ = orc.label_bfs(right, down, L, L)
        uf, _ = orc.label_uf(right, down, L, L)
        if not np.array_equal(bfs, uf):
            raise AssertionError(f"mask {bits:#x}: bfs {bfs} uf {uf}")
        if bits in sample:
            np.testing.assert_array_equal(bfs, _nx_labels(right, down, L, L))


def test_label_is_minimum_and_idempotent(orc):
    right, down = synth.bond_masks(32, 32, 0.5, seed=3)
    lab, _ = orc.label_bfs(right, down, 32, 32)
    idx = np.arange(32 * 32)
    assert np.all(lab <= idx)
    assert np.all(lab[lab] == lab)  # a root labels itself
