"""Pins of the oracle's Philox4x32-10 against an independent implementation.

cuRAND's host-side generator (CURAND_RNG_PSEUDO_PHILOX4_32_10, which runs on
the CPU and needs no GPU) emits block b of its stream as Philox4x32-10 with
key = (seed_lo, seed_hi) and counter (b // 65536, 0, b % 65536, 0).  Matching
4M words of that stream for several seeds pins the rounds, the multipliers,
the Weyl key schedule and the output word order of the oracle's copy.
"""
import ctypes
import os

import numpy as np
import pytest

CURAND_RNG_PSEUDO_PHILOX4_32_10 = 161


def _curand():
    path = "/usr/local/cuda/lib64/libcurand.so"
    if not os.path.exists(path):
        pytest.skip("libcurand not available")
    return ctypes.CDLL(path)


def _curand_stream(seed: int, n_words: int) -> np.ndarray:
    cr = _curand()
    gen = ctypes.c_void_p()
    assert cr.curandCreateGeneratorHost(ctypes.byref(gen), CURAND_RNG_PSEUDO_PHILOX4_32_10) == 0
    cr.curandSetPseudoRandomGeneratorSeed.argtypes = [ctypes.c_void_p, ctypes.c_ulonglong]
    assert cr.curandSetPseudoRandomGeneratorSeed(gen, seed) == 0
    out = np.zeros(n_words, np.uint32)
    assert cr.curandGenerate(gen, out.ctypes.data_as(ctypes.c_void_p),
                             ctypes.c_size_t(n_words)) == 0
    cr.curandDestroyGenerator(gen)
    return out


@pytest.mark.parametrize("seed", [0, 1, 0x0123456789ABCDEF, 0xFFFFFFFFFFFFFFFF])
def test_philox_matches_curand_host_stream(orc, seed):
    per = 1 << 16
    n_c0 = 16
    ref = _curand_stream(seed, 4 * per * n_c0).reshape(n_c0, per, 4)
    for c0 in range(n_c0):
        mine = orc.philox_stream(seed, [c0, 0, 0, 0], 2, per)
        np.testing.assert_array_equal(mine, ref[c0])


def test_philox_counter_words_1_and_3_change_output(orc):
    """Counter words 1 and 3 (site high word, domain) must enter the output."""
    base = orc.philox([5, 0, 7, 0], [11, 13])
    assert not np.array_equal(base, orc.philox([5, 1, 7, 0], [11, 13]))
    assert not np.array_equal(base, orc.philox([5, 0, 7, 1], [11, 13]))


def test_philox_uniformity(orc):
    """Chi-square of the byte histogram over 2^20 words stays in a 5-sigma band."""
    w = orc.philox_stream(42, [0, 0, 9, 0], 0, 1 << 18).ravel()
    b = w.view(np.uint8)
    h = np.bincount(b, minlength=256).astype(np.float64)
    e = len(b) / 256.0
    chi2 = float(((h - e) ** 2 / e).sum())
    assert abs(chi2 - 255.0) < 5 * np.sqrt(2 * 255.0)


def test_bond_words_pair_two_rows(orc):
    """One BOND draw serves the vertical pair (x, 2m), (x, 2m + 1): counter
    (m L + x, 0, t, BOND); row 2m reads words 0 (right) and 1 (down), row
    2m + 1 words 2 and 3; u = ((w >> 1) + 1/2) 2^-31 and the coin is bit 0
    of the right-bond word.  Checked against the Philox function pinned
    above, for even and odd rows and for the last row of an odd L."""
    seed, t = 0x0123456789ABCDEF, 5
    key = np.array([seed & 0xFFFFFFFF, seed >> 32], np.uint32)
    for L in (8, 9):
        theta = np.zeros(L * L, np.float32)
        for i in range(L * L):
            x, y = i % L, i // L
            w = orc.philox(np.array([(y >> 1) * L + x, 0, t, 0], np.uint32), key)
            wr, wd = (w[2], w[3]) if y & 1 else (w[0], w[1])
            u_r, _ = orc.bond_up(theta, L, L, 1.0, seed, t, i, 0)
            u_d, _ = orc.bond_up(theta, L, L, 1.0, seed, t, i, 1)
            assert u_r == ((int(wr) >> 1) + 0.5) * 2.0 ** -31
            assert u_d == ((int(wd) >> 1) + 0.5) * 2.0 ** -31
            assert orc.coin(seed, t, i, L) == int(wr) & 1
