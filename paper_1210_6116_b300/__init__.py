"""B300 (sm_103a) Swendsen-Wang sweep of the 2D classical XY model.

Thin ctypes binding of the C ABI in ``include/xy.h`` (libxy.so, built
in-tree).  Every step of a sweep runs in the library's CUDA kernels; this
module only marshals arguments.  PyTorch provides the device workspace and the
stream.  There is no CPU fallback: importing the package on a machine where
libxy.so cannot be loaded raises.

Functions with the C names (``xy_init``, ``xy_sweep``, ``xy_measure``,
``xy_pcc_step`` ...) mirror the ABI one to one; ``Lattice`` bundles a handle
with its workspace tensor.
"""
from __future__ import annotations

import ctypes
import math
import os
from pathlib import Path

import numpy as np

_PKG = Path(__file__).resolve().parent
# XY_BOUNDS_CHECK=1 selects the bounds-checked build of the library
LIB_PATH = _PKG / ("libxy_checked.so" if os.environ.get("XY_BOUNDS_CHECK") == "1" else "libxy.so")

XY_OK, XY_EINVAL, XY_ENOMEM, XY_ECUDA, XY_ETIMEOUT, XY_EINTERNAL, XY_EUNSUPPORTED = range(7)
XY_F32, XY_F16, XY_U16 = 0, 1, 2
# angle storage by name: (xy_angle_t, numpy dtype of xy_get/set_angles)
DTYPES = {"f32": (XY_F32, np.float32), "f16": (XY_F16, np.float16), "u16": (XY_U16, np.uint16)}


XY_UPDATE_SW, XY_UPDATE_WOLFF = 0, 1


def _update(name: str) -> int:
    """'sw': Swendsen-Wang sweep; 'wolff': Wolff single-cluster update."""
    codes = {"sw": XY_UPDATE_SW, "wolff": XY_UPDATE_WOLFF}
    if name not in codes:
        raise ValueError("update must be 'sw' or 'wolff'")
    return codes[name]


def _dtype(name: str):
    if name not in DTYPES:
        raise ValueError(f"dtype must be one of {sorted(DTYPES)}")
    return DTYPES[name]
XY_THR_F32, XY_THR_F64 = 0, 1

STATUS_NAMES = {0: "XY_OK", 1: "XY_EINVAL", 2: "XY_ENOMEM", 3: "XY_ECUDA", 4: "XY_ETIMEOUT",
                5: "XY_EINTERNAL", 6: "XY_EUNSUPPORTED"}

# every entry point declared in include/xy.h
EXPORTS = (
    "xy_last_error", "xy_workspace_size", "xy_init", "xy_sweep", "xy_pcc_step",
    "xy_measure", "xy_get_state", "xy_destroy", "xy_get_angles", "xy_set_angles",
    "xy_get_bonds", "xy_get_labels", "xy_get_sites", "xy_get_spins", "xy_label_bonds", "xy_get_band_stats",
    "xy_save", "xy_load", "xy_run_host", "xy_run_host_async", "xy_sync", "xy_profile",
    "xy_profile_read", "xy_label_bonds_static", "xy_set_loop_bound", "xy_set_link_cap",
    "xy_build_arch",
    "xy_engine_workspace_size", "xy_engine_create", "xy_engine_admit", "xy_engine_retire",
    "xy_engine_step", "xy_engine_measure", "xy_engine_get_angles", "xy_engine_get_state",
    "xy_engine_destroy",
)
KERNEL_NAMES = ("bond_label", "merge", "compress", "flip_measure", "finalize")
# kernel launches of one single-lattice sweep: xy_sweep runs 4 per sweep
# (its finalize step is folded into the next sweep's first kernel) plus 2 per
# call (the PCC switch and the last record); xy_pcc_step runs 5 per sweep
# plus 1 per call
LAUNCHES_PER_SWEEP = 4
LAUNCHES_PER_CALL = 2
LAUNCHES_PER_PCC_SWEEP = 5


class XyError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class xy_config(ctypes.Structure):
    _fields_ = [("L", ctypes.c_uint32), ("tile_y", ctypes.c_uint32), ("seed", ctypes.c_uint64),
                ("beta", ctypes.c_double), ("angle_dtype", ctypes.c_int32),
                ("threshold_mode", ctypes.c_int32), ("start", ctypes.c_int32),
                ("record_cap", ctypes.c_uint32), ("measure_xi", ctypes.c_uint32),
                ("update", ctypes.c_uint32)]


OBS_FIELDS = ("energy_per_site", "m2", "mx", "my", "ex", "sx", "ey", "sy", "upsilon", "beta")


class xy_obs(ctypes.Structure):
    _fields_ = ([(n, ctypes.c_double) for n in OBS_FIELDS] + [("sweep", ctypes.c_uint64)]
                + [("chik", ctypes.c_double), ("flipped", ctypes.c_uint64)])


OBS_DTYPE = np.dtype([(n, np.float64) for n in OBS_FIELDS] + [("sweep", np.uint64),
                                                             ("chik", np.float64),
                                                             ("flipped", np.uint64)])
assert OBS_DTYPE.itemsize == ctypes.sizeof(xy_obs)


class xy_kernel_times(ctypes.Structure):
    _fields_ = [("ms", ctypes.c_double * 5), ("launches", ctypes.c_uint64 * 5)]


class xy_pcc_params(ctypes.Structure):
    _fields_ = [("target", ctypes.c_double), ("dbeta0", ctypes.c_double),
                ("halve_every", ctypes.c_uint32), ("block", ctypes.c_uint32)]


_lib = None


def load_library() -> ctypes.CDLL:
    """Load libxy.so (raises if it is missing: there is no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not LIB_PATH.exists():
        raise RuntimeError(f"{LIB_PATH} is missing; build it with "
                           "`python -m paper_1210_6116_b300.build`")
    L = ctypes.CDLL(str(LIB_PATH))
    P, U32, U64, I, D = ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int, ctypes.c_double
    sigs = {
        "xy_last_error": (ctypes.c_char_p, []),
        "xy_workspace_size": (I, [P, P]),
        "xy_init": (I, [P, P, ctypes.c_size_t, P, P]),
        "xy_sweep": (I, [P, U32]),
        "xy_pcc_step": (I, [P, P, U32]),
        "xy_measure": (I, [P, P, U32, P, I]),
        "xy_get_state": (I, [P, P, P]),
        "xy_destroy": (I, [P]),
        "xy_get_angles": (I, [P, P]),
        "xy_set_angles": (I, [P, P]),
        "xy_get_bonds": (I, [P, P, P]),
        "xy_get_labels": (I, [P, P]),
        "xy_get_sites": (I, [P, P, ctypes.c_uint32, P, P, P]),
        "xy_get_spins": (I, [P, P, P]),
        "xy_label_bonds": (I, [P, P, P, P]),
        "xy_get_band_stats": (I, [P, P, P]),
        "xy_save": (I, [P, P, P]),
        "xy_load": (I, [P, P, ctypes.c_size_t]),
        "xy_run_host": (I, [P, P, U32, P, P]),
        "xy_run_host_async": (I, [P, P, ctypes.c_uint32, P, P]),
        "xy_sync": (I, [P]),
        "xy_profile": (I, [P, I]),
        "xy_profile_read": (I, [P, P]),
        "xy_label_bonds_static": (I, [U32, P, P, P, P, I]),
        "xy_set_loop_bound": (I, [P, U32]),
        "xy_set_link_cap": (I, [P, U32]),
        "xy_build_arch": (I, [P]),
        "xy_engine_workspace_size": (I, [U32, P]),
        "xy_engine_create": (I, [U32, I, I, U32, P, ctypes.c_size_t, P, P]),
        "xy_engine_admit": (I, [P, P, P, P, ctypes.c_size_t, P]),
        "xy_engine_retire": (I, [P, U32]),
        "xy_engine_step": (I, [P, U32]),
        "xy_engine_measure": (I, [P, U32, P, U32, P]),
        "xy_engine_get_angles": (I, [P, U32, P]),
        "xy_engine_get_state": (I, [P, U32, P, P]),
        "xy_engine_destroy": (I, [P]),
    }
    for name, (res, args) in sigs.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def _check(status: int):
    if status != XY_OK:
        raise XyError(status, load_library().xy_last_error().decode())


def _ptr(a: np.ndarray):
    assert a.flags["C_CONTIGUOUS"]
    return ctypes.c_void_p(a.ctypes.data)


# ---------------------------------------------------------------------------
# C-named wrappers
# ---------------------------------------------------------------------------
def xy_workspace_size(cfg: xy_config) -> int:
    n = ctypes.c_size_t(0)
    _check(load_library().xy_workspace_size(ctypes.byref(cfg), ctypes.byref(n)))
    return n.value


def xy_init(cfg: xy_config, d_workspace: int, nbytes: int, stream: int) -> ctypes.c_void_p:
    h = ctypes.c_void_p()
    _check(load_library().xy_init(ctypes.byref(cfg), ctypes.c_void_p(d_workspace), nbytes,
                                  ctypes.c_void_p(stream), ctypes.byref(h)))
    return h


def xy_sweep(h, n: int):
    _check(load_library().xy_sweep(h, n))


def xy_pcc_step(h, params: xy_pcc_params, n: int):
    _check(load_library().xy_pcc_step(h, ctypes.byref(params), n))


def xy_measure(h, max_records: int, sync: int = 1) -> np.ndarray:
    out = np.zeros(max_records, OBS_DTYPE)
    n = ctypes.c_uint32(0)
    _check(load_library().xy_measure(h, _ptr(out) if max_records else None, max_records,
                                     ctypes.byref(n), sync))
    return out[: n.value]


def xy_get_state(h):
    b = ctypes.c_double(0)
    t = ctypes.c_uint64(0)
    _check(load_library().xy_get_state(h, ctypes.byref(b), ctypes.byref(t)))
    return b.value, t.value


def xy_destroy(h):
    _check(load_library().xy_destroy(h))


def xy_last_error() -> str:
    return load_library().xy_last_error().decode()


def xy_build_arch() -> int:
    """Compute capability of the loaded device code (103 for sm_103a)."""
    v = ctypes.c_int(0)
    _check(load_library().xy_build_arch(ctypes.byref(v)))
    return v.value


XY_STATIC_MAX_L = 1024


def xy_label_bonds_static(L: int, d_right: int, d_down: int, d_labels: int, stream: int,
                          sync: int = 1):
    """Label device bond bytes into device labels without any workspace
    (see include/xy.h): pointers are device addresses."""
    _check(load_library().xy_label_bonds_static(L, ctypes.c_void_p(d_right),
                                                ctypes.c_void_p(d_down),
                                                ctypes.c_void_p(d_labels),
                                                ctypes.c_void_p(stream), sync))


# ---------------------------------------------------------------------------
# Lattice: a handle plus its torch-owned workspace
# ---------------------------------------------------------------------------
class Lattice:
    """One L x L periodic lattice resident in device memory.

    The workspace is a torch uint8 tensor on the current CUDA device; all
    launches go to ``stream`` (default: torch's current stream)."""

    def __init__(self, L: int, beta: float, seed: int, *, dtype: str = "f32",
                 exact: bool = True, start: str = "random", tile_y: int = 0,
                 record_cap: int = 0, measure_xi: bool = False, update: str = "sw",
                 stream=None):
        import torch  # plumbing: device memory and streams

        self.L = int(L)
        self.dtype = dtype
        code, self.np_dtype = _dtype(dtype)
        self.cfg = xy_config(L=self.L, tile_y=tile_y, seed=seed, beta=beta,
                             angle_dtype=code,
                             threshold_mode=XY_THR_F64 if exact else XY_THR_F32,
                             start=0 if start == "random" else 1, record_cap=record_cap,
                             measure_xi=1 if measure_xi else 0, update=_update(update))
        self.nbytes = xy_workspace_size(self.cfg)
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.workspace = torch.empty(self.nbytes, dtype=torch.uint8, device="cuda")
        self.handle = xy_init(self.cfg, self.workspace.data_ptr(), self.nbytes,
                              self.stream.cuda_stream)

    # -- chain ---------------------------------------------------------------
    def sweep(self, n: int = 1):
        xy_sweep(self.handle, n)

    def pcc_step(self, n: int, target: float = 0.636508, dbeta0: float = 0.0005,
                 halve_every: int = 0, block: int = 1000):
        xy_pcc_step(self.handle, xy_pcc_params(target=target, dbeta0=dbeta0,
                                               halve_every=halve_every, block=block), n)

    def measure(self, max_records: int = 1 << 20, sync: bool = True) -> np.ndarray:
        return xy_measure(self.handle, max_records, 1 if sync else 0)

    def state(self):
        return xy_get_state(self.handle)

    # -- host copies ---------------------------------------------------------
    @property
    def n(self) -> int:
        return self.L * self.L

    def get_angles(self) -> np.ndarray:
        out = np.zeros(self.n, self.np_dtype)
        _check(load_library().xy_get_angles(self.handle, _ptr(out)))
        return out

    def set_angles(self, a: np.ndarray):
        a = np.ascontiguousarray(a, dtype=self.np_dtype)
        assert a.size == self.n
        _check(load_library().xy_set_angles(self.handle, _ptr(a)))

    def get_spins(self):
        """(cos theta, sin theta) of the current angles, float32 arrays of N,
        from the observables' device cos/sin routine."""
        c = np.zeros(self.n, np.float32)
        s = np.zeros(self.n, np.float32)
        _check(load_library().xy_get_spins(self.handle, _ptr(c), _ptr(s)))
        return c, s

    def get_bonds(self):
        r = np.zeros(self.n, np.uint8)
        d = np.zeros(self.n, np.uint8)
        _check(load_library().xy_get_bonds(self.handle, _ptr(r), _ptr(d)))
        return r, d

    def get_labels(self) -> np.ndarray:
        out = np.zeros(self.n, np.uint32)
        _check(load_library().xy_get_labels(self.handle, _ptr(out)))
        return out

    def get_sites(self, sites):
        """(angles, labels, bonds) of the listed sites after the last sweep;
        bonds: bit 0 right, bit 1 down."""
        sites = np.ascontiguousarray(sites, dtype=np.uint64)
        th = np.zeros(sites.size, self.np_dtype)
        lab = np.zeros(sites.size, np.uint32)
        bd = np.zeros(sites.size, np.uint8)
        _check(load_library().xy_get_sites(self.handle, _ptr(sites), sites.size, _ptr(th),
                                           _ptr(lab), _ptr(bd)))
        return th, lab, bd

    def label_bonds(self, right: np.ndarray, down: np.ndarray) -> np.ndarray:
        r = np.ascontiguousarray(right, np.uint8)
        d = np.ascontiguousarray(down, np.uint8)
        out = np.zeros(self.n, np.uint32)
        _check(load_library().xy_label_bonds(self.handle, _ptr(r), _ptr(d), _ptr(out)))
        return out

    def set_loop_bound(self, cap: int):
        """Bound on the device-side find/union loops (0: the default)."""
        _check(load_library().xy_set_loop_bound(self.handle, int(cap)))

    def set_link_cap(self, cap: int):
        """Link slots a tile may fill per sweep (0: the default)."""
        _check(load_library().xy_set_link_cap(self.handle, int(cap)))

    def band_stats(self):
        a = ctypes.c_uint64(0)
        b = ctypes.c_uint64(0)
        _check(load_library().xy_get_band_stats(self.handle, ctypes.byref(a), ctypes.byref(b)))
        return a.value, b.value

    def run_host(self, angles_in, n_sweeps: int, obs_out=None, angles_out=None):
        """xy_run_host with numpy (optionally pinned) host buffers."""
        pin = (lambda a: None if a is None else ctypes.c_void_p(a.ctypes.data))
        _check(load_library().xy_run_host(self.handle, pin(angles_in), n_sweeps,
                                          pin(obs_out), pin(angles_out)))

    def run_host_async(self, angles_in, n_sweeps: int, obs_out=None, angles_out=None):
        """xy_run_host_async: enqueue only; the buffers must stay alive and
        unread until sync()."""
        pin = (lambda a: None if a is None else ctypes.c_void_p(a.ctypes.data))
        _check(load_library().xy_run_host_async(self.handle, pin(angles_in), n_sweeps,
                                                pin(obs_out), pin(angles_out)))

    def sync(self):
        _check(load_library().xy_sync(self.handle))

    def profile(self, enable: bool, every: int = 1):
        """Time the kernels of every `every`-th sweep with CUDA events (the
        events slow the timed sweeps by a few us each)."""
        _check(load_library().xy_profile(self.handle, int(every) if enable else 0))

    def profile_read(self) -> dict:
        t = xy_kernel_times()
        _check(load_library().xy_profile_read(self.handle, ctypes.byref(t)))
        return {name: (t.ms[k], int(t.launches[k])) for k, name in enumerate(KERNEL_NAMES)}

    def save(self) -> bytes:
        n = ctypes.c_size_t(0)
        _check(load_library().xy_save(self.handle, None, ctypes.byref(n)))
        buf = (ctypes.c_char * n.value)()
        _check(load_library().xy_save(self.handle, buf, ctypes.byref(n)))
        return bytes(buf)

    def load(self, blob: bytes):
        buf = ctypes.create_string_buffer(blob, len(blob))
        _check(load_library().xy_load(self.handle, buf, len(blob)))

    def close(self):
        if getattr(self, "handle", None):
            xy_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Engine:
    """Many lattices advanced by shared launches (xy_engine_* of the C ABI).

    Every admitted lattice gets its own torch workspace; the engine's table
    lives in one more.  All lattices share dtype, threshold mode and tile."""

    def __init__(self, max_slots: int, *, dtype: str = "f32", exact: bool = False,
                 tile_y: int = 64, stream=None):
        import torch

        self.dtype = dtype
        code, self.np_dtype = _dtype(dtype)
        self.exact = exact
        self.tile_y = tile_y
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        n = ctypes.c_size_t(0)
        _check(load_library().xy_engine_workspace_size(max_slots, ctypes.byref(n)))
        self.table = torch.empty(n.value, dtype=torch.uint8, device="cuda")
        self.handle = ctypes.c_void_p()
        _check(load_library().xy_engine_create(
            max_slots, code,
            XY_THR_F64 if exact else XY_THR_F32, tile_y,
            ctypes.c_void_p(self.table.data_ptr()), n.value,
            ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(self.handle)))
        self.workspaces = {}
        self.L = {}

    def config(self, L: int, beta: float, seed: int, start: str = "random",
               record_cap: int = 0, measure_xi: bool = False, update: str = "sw") -> xy_config:
        return xy_config(L=L, tile_y=self.tile_y, seed=seed, beta=beta,
                         angle_dtype=_dtype(self.dtype)[0],
                         threshold_mode=XY_THR_F64 if self.exact else XY_THR_F32,
                         start=0 if start == "random" else 1, record_cap=record_cap,
                         measure_xi=1 if measure_xi else 0, update=_update(update))

    @staticmethod
    def footprint(cfg: xy_config) -> int:
        return xy_workspace_size(cfg)

    def admit(self, cfg: xy_config, pcc: xy_pcc_params | None = None) -> int:
        import torch

        nbytes = xy_workspace_size(cfg)
        ws = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
        slot = ctypes.c_uint32(0)
        _check(load_library().xy_engine_admit(
            self.handle, ctypes.byref(cfg), ctypes.byref(pcc) if pcc is not None else None,
            ctypes.c_void_p(ws.data_ptr()), nbytes, ctypes.byref(slot)))
        self.workspaces[slot.value] = ws
        self.L[slot.value] = cfg.L
        return slot.value

    def retire(self, slot: int):
        _check(load_library().xy_engine_retire(self.handle, slot))
        self.workspaces.pop(slot, None)
        self.L.pop(slot, None)

    def step(self, n: int = 1):
        _check(load_library().xy_engine_step(self.handle, n))

    def measure(self, slot: int, max_records: int = 1 << 20) -> np.ndarray:
        out = np.zeros(max_records, OBS_DTYPE)
        n = ctypes.c_uint32(0)
        _check(load_library().xy_engine_measure(self.handle, slot, _ptr(out), max_records,
                                                ctypes.byref(n)))
        return out[: n.value]

    def get_angles(self, slot: int) -> np.ndarray:
        out = np.zeros(self.L[slot] ** 2, self.np_dtype)
        _check(load_library().xy_engine_get_angles(self.handle, slot, _ptr(out)))
        return out

    def state(self, slot: int):
        b = ctypes.c_double(0)
        t = ctypes.c_uint64(0)
        _check(load_library().xy_engine_get_state(self.handle, slot, ctypes.byref(b),
                                                  ctypes.byref(t)))
        return b.value, t.value

    def close(self):
        if getattr(self, "handle", None):
            _check(load_library().xy_engine_destroy(self.handle))
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


TWO_PI_F32 = np.float32(2.0 * math.pi)
