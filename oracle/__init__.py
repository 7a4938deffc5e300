"""Plain CPU oracle of the Swendsen-Wang XY sweep (ctypes wrapper).

TEST INFRASTRUCTURE ONLY.  The C code in ``oracle.c`` is the slow, obviously
correct reference the CUDA library is checked against.  Only the test suite,
``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg and reference
arm (``--impl reference``, which times the oracle on the host cores) may
import this package.  It does not import the CUDA library and the CUDA library does
not import it; they share only the seeded input generators of ``synth``.

Each wrapper below follows one step of the sweep (see ``oracle.h``):
axis -> bonds -> labels -> flip -> observables -> PCC.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from pathlib import Path

import numpy as np

_HERE = Path(__file__).resolve().parent
_SRC = _HERE / "oracle.c"
_LIB = _HERE / "liboracle.so"
# the same source built with -fopenmp: bonds, flip and observables on all
# host cores (labeling sequential); used only to time the CPU baseline
_LIB_OMP = _HERE / "liboracle_omp.so"

_lib = None
_lib_omp = None


def _compile(out: Path, extra: list, force: bool):
    if force or not out.exists() or out.stat().st_mtime < max(
        _SRC.stat().st_mtime, (_HERE / "oracle.h").stat().st_mtime
    ):
        tmp = out.with_suffix(f".so.tmp{os.getpid()}")
        cmd = [
            "gcc", "-O2", "-std=gnu11", "-fPIC", "-shared",
            "-ffp-contract=off", "-fno-fast-math", *extra,
            str(_SRC), "-o", str(tmp), "-lm",
        ]
        subprocess.run(cmd, check=True)
        os.replace(tmp, out)


def build(force: bool = False) -> Path:
    """Compile oracle.c into liboracle.so with plain IEEE FP64 semantics, and
    the OpenMP timing build liboracle_omp.so."""
    _compile(_LIB, [], force)
    _compile(_LIB_OMP, ["-fopenmp"], force)
    return _LIB


class Sums(ctypes.Structure):
    _fields_ = [(n, ctypes.c_double) for n in (
        "sum_cos", "sum_sin", "sum_cos_r", "sum_sin_r", "sum_cos_d",
        "sum_sin_d", "n_sites", "n_links_r", "n_links_d")] + [
        ("fx", ctypes.c_double * 4), ("fy", ctypes.c_double * 4)] + [
        (n, ctypes.c_double) for n in ("abs_cos", "abs_sin", "abs_cos_r", "abs_sin_r",
                                       "abs_cos_d", "abs_sin_d")]


OBS_FIELDS = ("energy_per_site", "m2", "mx", "my", "ex", "sx", "ey", "sy",
              "upsilon", "beta", "chik")


# L1 norms per site of the sums behind mx, my, ex, sx, ey, sy (sum |term| / N):
# the scale a cancelling sum is compared against (tolerance reading A19)
L1_FIELDS = ("l1_mx", "l1_my", "l1_ex", "l1_sx", "l1_ey", "l1_sy")


class Obs(ctypes.Structure):
    _fields_ = [(n, ctypes.c_double) for n in OBS_FIELDS + ("flipped",) + L1_FIELDS]


# per-update records: the observables, the number of reflected sites and the
# L1 norms
OBS_DTYPE = np.dtype([(n, np.float64) for n in OBS_FIELDS + ("flipped",) + L1_FIELDS])

_P = ctypes.c_void_p
_I = ctypes.c_int
_U32 = ctypes.c_uint32
_U64 = ctypes.c_uint64
_D = ctypes.c_double


def lib(omp: bool = False):
    """The plain oracle library, or (omp=True) its OpenMP timing build."""
    global _lib, _lib_omp
    if (_lib_omp if omp else _lib) is None:
        build()
        L = ctypes.CDLL(str(_LIB_OMP if omp else _LIB))
        sig = {
            "orc_threads": (_I, [_I]),
            "orc_philox4x32_10": (None, [_P, _P, _P]),
            "orc_philox_stream": (None, [_U64, _P, _I, _U64, _P]),
            "orc_axis": (None, [_U64, _U32, _P, _P]),
            "orc_axis_u16": (None, [_U64, _U32, _P, _P]),
            "orc_init_angles_u16": (None, [_I, _I, _U64, _I, _P]),
            "orc_bonds_u16": (ctypes.c_long, [_I, _I, _I, _I, _P, _D, _U64, _U32, _P, _P]),
            "orc_bond_up_u16": (None, [_I, _I, _I, _I, _P, _D, _U64, _U32, ctypes.c_int64, _I, _P, _P]),
            "orc_flip_u16": (ctypes.c_long, [_I, _I, _P, _P, _U64, _U32, ctypes.c_uint16, _P]),
            "orc_sums_u16": (None, [_I, _I, _I, _I, _P, _P]),
            "orc_sw_run_u16": (None, [_I, _I, _I, _I, _P, _D, _U64, _U32, _U32, _P, _P, _P, _P, _P]),
            "orc_init_angles_f32": (None, [_I, _I, _U64, _I, _P]),
            "orc_init_angles_f16": (None, [_I, _I, _U64, _I, _P]),
            "orc_bonds_f32": (ctypes.c_long, [_I, _I, _I, _I, _P, _D, _U64, _U32, _P, _P]),
            "orc_bonds_f16": (ctypes.c_long, [_I, _I, _I, _I, _P, _D, _U64, _U32, _P, _P]),
            "orc_bond_up_f32": (None, [_I, _I, _I, _I, _P, _D, _U64, _U32, ctypes.c_int64, _I, _P, _P]),
            "orc_bonds_rows_f32": (ctypes.c_long, [_I, _P, ctypes.c_int64, _I, _D, _U64, _U32, _P, _P,
                                                   _P, _P]),
            "orc_label_bfs": (ctypes.c_long, [_I, _I, _I, _I, _P, _P, _P, _P]),
            "orc_label_uf": (ctypes.c_long, [_I, _I, _I, _I, _P, _P, _P]),
            "orc_flip_f32": (ctypes.c_long, [_I, _I, _P, _P, _U64, _U32, ctypes.c_float, _P]),
            "orc_flip_f16": (ctypes.c_long, [_I, _I, _P, _P, _U64, _U32, ctypes.c_float, _P]),
            "orc_coin": (_I, [_U64, _U32, _I, _U32]),
            "orc_sums_f32": (None, [_I, _I, _I, _I, _P, _P]),
            "orc_sums_f16": (None, [_I, _I, _I, _I, _P, _P]),
            "orc_derive": (None, [_P, _D, _P]),
            "orc_pcc_next_beta": (_D, [_D, _D, _D, _D]),
            "orc_pcc_dbeta": (_D, [_D, _U32, _U32]),
            "orc_sw_run_f32": (None, [_I, _I, _I, _I, _P, _D, _U64, _U32, _U32, _P, _P, _P, _P, _P]),
            "orc_sw_run_f16": (None, [_I, _I, _I, _I, _P, _D, _U64, _U32, _U32, _P, _P, _P, _P, _P]),
            "orc_pcc_run_f32": (None, [_I, _P, _P, _D, _D, _U32, _U32, _U64, _U32, _U32, _U32,
                                       _P, _P, _P, _P, _P, _P, _P]),
            "orc_seed_site": (_U64, [_U64, _U32, _U64]),
            "orc_wolff_cluster": (ctypes.c_long, [_I, _I, _I, _I, _P, _D, _D, _D, _U64, _U32,
                                                  _U64, _P, _P]),
            "orc_wolff_run_f32": (None, [_I, _I, _I, _I, _P, _D, _U64, _U32, _U32, _P, _P, _P]),
            "orc_wolff_run_f16": (None, [_I, _I, _I, _I, _P, _D, _U64, _U32, _U32, _P, _P, _P]),
            "orc_wolff_run_u16": (None, [_I, _I, _I, _I, _P, _D, _U64, _U32, _U32, _P, _P, _P]),
            "orc_metropolis_run": (None, [_I, _I, _P, _D, _D, _U64, _U32, _U32, _P, _P]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        if omp:
            _lib_omp = L
        else:
            _lib = L
    return _lib_omp if omp else _lib


def omp_threads(n: int = 0) -> int:
    """Threads of the OpenMP timing build (n > 0 sets them); returns the count."""
    return int(lib(omp=True).orc_threads(n))


def _ptr(a: np.ndarray):
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.c_void_p)


# ---- Philox -------------------------------------------------------------
def philox(ctr, key) -> np.ndarray:
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, np.uint32)
    lib().orc_philox4x32_10(_ptr(c), _ptr(k), _ptr(out))
    return out


def philox_stream(seed: int, ctr, word: int, n_calls: int) -> np.ndarray:
    """(n_calls, 4) words: Philox(ctr with counter word `word` advanced by k)."""
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    out = np.zeros((n_calls, 4), np.uint32)
    lib().orc_philox_stream(seed, _ptr(c), word, n_calls, _ptr(out))
    return out


# ---- sweep steps ----------------------------------------------------------
def axis(seed: int, t: int):
    """(phi, cos phi, sin phi, C64, C32) of sweep t."""
    out = np.zeros(4, np.float64)
    c32 = np.zeros(1, np.float32)
    lib().orc_axis(seed, t, _ptr(out), _ptr(c32))
    return float(out[0]), float(out[1]), float(out[2]), float(out[3]), np.float32(c32[0])


def axis_u16(seed: int, t: int):
    """(phi_q, cos phi_q, sin phi_q, C64, Cq) of sweep t for u16 angles."""
    out = np.zeros(4, np.float64)
    cq = np.zeros(1, np.uint16)
    lib().orc_axis_u16(seed, t, _ptr(out), _ptr(cq))
    return float(out[0]), float(out[1]), float(out[2]), float(out[3]), int(cq[0])


# Angle arrays: float32 (FP32), float16 (FP16 bits) or uint16 (u16 fixed
# point, theta = q 2 pi / 65536); every step below dispatches on the dtype.
def init_angles(L: int, seed: int, start: int, dtype=np.float32, Ly: int | None = None) -> np.ndarray:
    Ly = L if Ly is None else Ly
    if dtype == np.float32:
        th = np.zeros(L * Ly, np.float32)
        lib().orc_init_angles_f32(L, Ly, seed, start, _ptr(th))
    elif dtype == np.uint16:
        th = np.zeros(L * Ly, np.uint16)
        lib().orc_init_angles_u16(L, Ly, seed, start, _ptr(th))
    else:
        th = np.zeros(L * Ly, np.uint16)
        lib().orc_init_angles_f16(L, Ly, seed, start, _ptr(th))
        th = th.view(np.float16)
    return th


def bonds(theta: np.ndarray, Lx: int, Ly: int, beta: float, seed: int, t: int,
          per_x: int = 1, per_y: int = 1):
    """(right, down, n_band): per-site 0/1 bond bytes and the count of bonds
    with |u - p| < 1e-12."""
    n = Lx * Ly
    right = np.zeros(n, np.uint8)
    down = np.zeros(n, np.uint8)
    if theta.dtype == np.float32:
        band = lib().orc_bonds_f32(Lx, Ly, per_x, per_y, _ptr(theta), beta, seed, t,
                                   _ptr(right), _ptr(down))
    elif theta.dtype == np.uint16:
        band = lib().orc_bonds_u16(Lx, Ly, per_x, per_y, _ptr(theta), beta, seed, t,
                                   _ptr(right), _ptr(down))
    else:
        band = lib().orc_bonds_f16(Lx, Ly, per_x, per_y, _ptr(theta.view(np.uint16)), beta,
                                   seed, t, _ptr(right), _ptr(down))
    return right, down, int(band)


def bond_up(theta: np.ndarray, Lx: int, Ly: int, beta: float, seed: int, t: int,
            i: int, direction: int, per_x: int = 1, per_y: int = 1):
    u = np.zeros(1, np.float64)
    p = np.zeros(1, np.float64)
    f = lib().orc_bond_up_u16 if theta.dtype == np.uint16 else lib().orc_bond_up_f32
    f(Lx, Ly, per_x, per_y, _ptr(theta), beta, seed, t, i, direction, _ptr(u), _ptr(p))
    return float(u[0]), float(p[0])


def label_bfs(right, down, Lx: int, Ly: int, per_x: int = 1, per_y: int = 1):
    n = Lx * Ly
    lab = np.zeros(n, np.uint32)
    q = np.zeros(n, np.uint32)
    comps = lib().orc_label_bfs(Lx, Ly, per_x, per_y, _ptr(np.ascontiguousarray(right, np.uint8)),
                                _ptr(np.ascontiguousarray(down, np.uint8)), _ptr(lab), _ptr(q))
    return lab, int(comps)


def label_uf(right, down, Lx: int, Ly: int, per_x: int = 1, per_y: int = 1):
    n = Lx * Ly
    lab = np.zeros(n, np.uint32)
    comps = lib().orc_label_uf(Lx, Ly, per_x, per_y, _ptr(np.ascontiguousarray(right, np.uint8)),
                               _ptr(np.ascontiguousarray(down, np.uint8)), _ptr(lab))
    return lab, int(comps)


def coin(seed: int, t: int, root: int, Lx: int) -> int:
    """Cluster coin of root site `root` in sweep t of an Lx-wide lattice."""
    return int(lib().orc_coin(seed, t, Lx, root))


def flip(theta: np.ndarray, label: np.ndarray, Lx: int, Ly: int, seed: int, t: int, c32):
    """Flips theta in place; returns the per-site flip set.  c32 is C32 of
    axis() for FP32/FP16 angles and Cq of axis_u16() for u16 angles."""
    fl = np.zeros(Lx * Ly, np.uint8)
    lab = np.ascontiguousarray(label, np.uint32)
    if theta.dtype == np.float32:
        lib().orc_flip_f32(Lx, Ly, _ptr(theta), _ptr(lab), seed, t, float(c32), _ptr(fl))
    elif theta.dtype == np.uint16:
        lib().orc_flip_u16(Lx, Ly, _ptr(theta), _ptr(lab), seed, t, int(c32), _ptr(fl))
    else:
        lib().orc_flip_f16(Lx, Ly, _ptr(theta.view(np.uint16)), _ptr(lab), seed, t, float(c32),
                           _ptr(fl))
    return fl


def bonds_rows(theta_rows: np.ndarray, L: int, y0: int, nrows: int, beta: float, seed: int,
               t: int):
    """Bonds of rows y0 .. y0+nrows-1 of the L x L periodic lattice of sweep t
    from the FP32 angles of rows y0 .. y0+nrows ((nrows + 1) x L); returns
    (right, down, gap_right, gap_down): nrows x L bonds each, and u - p of
    each bond."""
    th = np.ascontiguousarray(theta_rows, np.float32)
    assert th.size == (nrows + 1) * L
    right = np.zeros(nrows * L, np.uint8)
    down = np.zeros(nrows * L, np.uint8)
    gr = np.zeros(nrows * L, np.float64)
    gd = np.zeros(nrows * L, np.float64)
    lib().orc_bonds_rows_f32(L, _ptr(th), y0, nrows, beta, seed, t, _ptr(right), _ptr(down),
                             _ptr(gr), _ptr(gd))
    return right, down, gr, gd


def sums(theta: np.ndarray, Lx: int, Ly: int, per_x: int = 1, per_y: int = 1,
         omp: bool = False) -> Sums:
    """Observable sums of a configuration; omp=True runs the OpenMP build
    (FP32 angles), which adds the same terms in another order."""
    s = Sums()
    if omp:
        assert theta.dtype == np.float32
        lib(omp=True).orc_sums_f32(Lx, Ly, per_x, per_y, _ptr(theta), ctypes.byref(s))
    elif theta.dtype == np.float32:
        lib().orc_sums_f32(Lx, Ly, per_x, per_y, _ptr(theta), ctypes.byref(s))
    elif theta.dtype == np.uint16:
        lib().orc_sums_u16(Lx, Ly, per_x, per_y, _ptr(theta), ctypes.byref(s))
    else:
        lib().orc_sums_f16(Lx, Ly, per_x, per_y, _ptr(theta.view(np.uint16)), ctypes.byref(s))
    return s


def derive(s: Sums, beta: float) -> dict:
    o = Obs()
    lib().orc_derive(ctypes.byref(s), beta, ctypes.byref(o))
    return {n: getattr(o, n) for n in OBS_FIELDS + L1_FIELDS}


def measure(theta: np.ndarray, Lx: int, Ly: int, beta: float, per_x: int = 1, per_y: int = 1) -> dict:
    return derive(sums(theta, Lx, Ly, per_x, per_y), beta)


def pcc_next_beta(beta: float, beta_upsilon: float, target: float, dbeta: float) -> float:
    return float(lib().orc_pcc_next_beta(beta, beta_upsilon, target, dbeta))


def pcc_dbeta(dbeta0: float, halve_every: int, k: int) -> float:
    return float(lib().orc_pcc_dbeta(dbeta0, halve_every, k))


# ---- whole runs -----------------------------------------------------------
class _Scratch:
    def __init__(self, n: int):
        self.right = np.zeros(n, np.uint8)
        self.down = np.zeros(n, np.uint8)
        self.label = np.zeros(n, np.uint32)
        self.queue = np.zeros(n, np.uint32)


def sw_run(theta: np.ndarray, Lx: int, Ly: int, beta: float, seed: int, t0: int, n: int,
           per_x: int = 1, per_y: int = 1, record: bool = True, omp: bool = False) -> np.ndarray:
    """n fixed-beta sweeps t0..t0+n-1 in place; returns the per-sweep records.
    omp=True runs the OpenMP timing build (FP32 angles only)."""
    sc = _Scratch(Lx * Ly)
    obs = np.zeros(n, OBS_DTYPE) if record else None
    optr = _ptr(obs) if record else None
    if omp:
        assert theta.dtype == np.float32
        lib(omp=True).orc_sw_run_f32(Lx, Ly, per_x, per_y, _ptr(theta), beta, seed, t0, n,
                                     _ptr(sc.right), _ptr(sc.down), _ptr(sc.label),
                                     _ptr(sc.queue), optr)
    elif theta.dtype == np.float32:
        lib().orc_sw_run_f32(Lx, Ly, per_x, per_y, _ptr(theta), beta, seed, t0, n,
                             _ptr(sc.right), _ptr(sc.down), _ptr(sc.label), _ptr(sc.queue), optr)
    elif theta.dtype == np.uint16:
        lib().orc_sw_run_u16(Lx, Ly, per_x, per_y, _ptr(theta), beta, seed, t0, n,
                             _ptr(sc.right), _ptr(sc.down), _ptr(sc.label), _ptr(sc.queue), optr)
    else:
        lib().orc_sw_run_f16(Lx, Ly, per_x, per_y, _ptr(theta.view(np.uint16)), beta, seed, t0,
                             n, _ptr(sc.right), _ptr(sc.down), _ptr(sc.label), _ptr(sc.queue),
                             optr)
    return obs


class PCCState:
    def __init__(self, beta: float):
        self.beta = np.array([beta], np.float64)
        self.blk_acc = np.zeros(1, np.float64)
        self.blk_count = np.zeros(1, np.uint32)


def pcc_run(theta: np.ndarray, L: int, state: PCCState, target: float, dbeta0: float,
            halve_every: int, block: int, seed: int, t0: int, k0: int, n: int) -> np.ndarray:
    sc = _Scratch(L * L)
    obs = np.zeros(n, OBS_DTYPE)
    lib().orc_pcc_run_f32(L, _ptr(theta), _ptr(state.beta), target, dbeta0, halve_every, block,
                          seed, t0, k0, n, _ptr(state.blk_acc), _ptr(state.blk_count),
                          _ptr(sc.right), _ptr(sc.down), _ptr(sc.label), _ptr(sc.queue),
                          _ptr(obs))
    return obs


def metropolis_run(theta64: np.ndarray, L: int, beta: float, delta: float, seed: int, t0: int,
                   n: int):
    obs = np.zeros(n, OBS_DTYPE)
    acc = ctypes.c_long(0)
    lib().orc_metropolis_run(L, L, _ptr(theta64), beta, delta, seed, t0, n, _ptr(obs),
                             ctypes.byref(acc))
    return obs, acc.value


# ---- Wolff single-cluster updates -----------------------------------------
def seed_site(seed: int, t: int, n: int) -> int:
    return int(lib().orc_seed_site(seed, t, n))


def _widen(theta: np.ndarray) -> np.ndarray:
    if theta.dtype == np.uint16:
        return theta.astype(np.float64) * (6.283185307179586 / 65536.0)
    return theta.astype(np.float64)


def wolff_cluster(theta: np.ndarray, Lx: int, Ly: int, beta: float, seed: int, t: int,
                  per_x: int = 1, per_y: int = 1):
    """(in_cluster bytes, size) of update t's cluster, grown from its seed
    site on the angles theta (not modified)."""
    n = Lx * Ly
    ax = axis_u16(seed, t) if theta.dtype == np.uint16 else axis(seed, t)
    ang = np.ascontiguousarray(_widen(theta))
    inc = np.zeros(n, np.uint8)
    q = np.zeros(n, np.uint32)
    size = lib().orc_wolff_cluster(Lx, Ly, per_x, per_y, _ptr(ang), ax[1], ax[2], beta, seed, t,
                                   seed_site(seed, t, n), _ptr(inc), _ptr(q))
    return inc, int(size)


def wolff_run(theta: np.ndarray, Lx: int, Ly: int, beta: float, seed: int, t0: int, n: int,
              per_x: int = 1, per_y: int = 1, record: bool = True) -> np.ndarray:
    """n Wolff updates t0..t0+n-1 in place; returns the per-update records
    (flipped = cluster size)."""
    N = Lx * Ly
    inc = np.zeros(N, np.uint8)
    q = np.zeros(N, np.uint32)
    obs = np.zeros(n, OBS_DTYPE) if record else None
    optr = _ptr(obs) if record else None
    if theta.dtype == np.float32:
        f, th = lib().orc_wolff_run_f32, theta
    elif theta.dtype == np.uint16:
        f, th = lib().orc_wolff_run_u16, theta
    else:
        f, th = lib().orc_wolff_run_f16, theta.view(np.uint16)
    f(Lx, Ly, per_x, per_y, _ptr(th), beta, seed, t0, n, _ptr(inc), _ptr(q), optr)
    return obs
