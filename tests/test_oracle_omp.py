"""The OpenMP build of the oracle (used only to time the CPU baseline on all
host cores) runs the same chain as the plain oracle: identical angles and
flip counts; observables equal up to the order of the parallel sums."""
import numpy as np


def test_openmp_build_matches_plain_oracle(orc):
    L, beta, seed = 96, 1.12, 1000
    th0 = orc.init_angles(L, seed, 0)
    a, b = th0.copy(), th0.copy()
    ra = orc.sw_run(a, L, L, beta, seed, 0, 5)
    assert orc.omp_threads() >= 1
    rb = orc.sw_run(b, L, L, beta, seed, 0, 5, omp=True)
    np.testing.assert_array_equal(a, b)
    np.testing.assert_array_equal(ra["flipped"], rb["flipped"])
    for f in ("energy_per_site", "m2", "ex", "sx", "upsilon", "chik"):
        np.testing.assert_allclose(ra[f], rb[f], rtol=1e-12, atol=1e-15)
