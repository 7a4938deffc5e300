"""The C ABI library loads and exports every entry point declared in
include/xy.h; host-side argument checks work without a GPU."""
import ctypes
import re
from pathlib import Path

import pytest

import paper_1210_6116_b300 as xy
from paper_1210_6116_b300 import build as xybuild

ROOT = Path(__file__).resolve().parent.parent


@pytest.fixture(scope="module")
def lib():
    xybuild.build()
    return xy.load_library()


def _declared():
    text = (ROOT / "include" / "xy.h").read_text()
    return sorted(set(re.findall(r"^\s*(?:xy_status|const char \*)\s*(xy_\w+)\s*\(", text, re.M)))


def test_header_declares_the_boundary():
    names = _declared()
    for must in ("xy_init", "xy_sweep", "xy_measure", "xy_pcc_step", "xy_workspace_size",
                 "xy_destroy"):
        assert must in names
    assert set(names) == set(xy.EXPORTS)


def test_library_exports_every_declared_symbol(lib):
    for name in _declared():
        assert hasattr(lib, name), name


def test_bounds_checked_library_exports_every_declared_symbol():
    checked = ctypes.CDLL(str(xybuild.build(checked=True)))
    for name in _declared():
        assert hasattr(checked, name), name


def test_library_build_targets_sm_103a_only():
    """The build compiles device code for sm_103a and nothing else (the
    loaded image's compute capability is checked on a GPU by
    test_gpu_failure.py through xy_build_arch)."""
    assert xybuild.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def _cfg(**kw):
    base = dict(L=64, tile_y=0, seed=1, beta=1.12, angle_dtype=xy.XY_F32,
                threshold_mode=xy.XY_THR_F64, start=0, record_cap=0)
    base.update(kw)
    return xy.xy_config(**base)


def test_workspace_size_grows_with_L(lib):
    a = xy.xy_workspace_size(_cfg(L=64))
    b = xy.xy_workspace_size(_cfg(L=128))
    c = xy.xy_workspace_size(_cfg(L=4096))
    assert a < b < c
    n = 4096 * 4096
    # two FP32 angle buffers + labels + bit planes + coin bits
    assert c >= n * (4 + 4 + 4) + n // 4
    assert xy.xy_workspace_size(_cfg(L=4096, angle_dtype=xy.XY_F16)) < c


def test_workspace_size_at_L65536_fits_one_b300(lib):
    n = xy.xy_workspace_size(_cfg(L=65536))
    assert 50e9 < n < 60e9


@pytest.mark.parametrize("bad", [dict(L=1), dict(L=65537), dict(beta=-1.0),
                                 dict(beta=float("nan")), dict(angle_dtype=7),
                                 dict(threshold_mode=3), dict(start=2), dict(tile_y=48)])
def test_invalid_configs_rejected(lib, bad):
    with pytest.raises(xy.XyError) as e:
        xy.xy_workspace_size(_cfg(**bad))
    assert e.value.status == xy.XY_EINVAL
    assert xy.xy_last_error()


def test_init_rejects_null_and_small_workspace(lib):
    cfg = _cfg()
    h = ctypes.c_void_p()
    assert lib.xy_init(ctypes.byref(cfg), None, 1 << 30, None, ctypes.byref(h)) == xy.XY_EINVAL
    need = xy.xy_workspace_size(cfg)
    # a fake, aligned, non-NULL pointer: rejected before any device access
    assert lib.xy_init(ctypes.byref(cfg), ctypes.c_void_p(1 << 20), need - 1, None,
                       ctypes.byref(h)) == xy.XY_ENOMEM
    assert lib.xy_init(ctypes.byref(cfg), ctypes.c_void_p((1 << 20) + 8), need, None,
                       ctypes.byref(h)) == xy.XY_EINVAL


def test_null_handle_calls_rejected(lib):
    assert lib.xy_sweep(None, 1) == xy.XY_EINVAL
    n = ctypes.c_uint32()
    assert lib.xy_measure(None, None, 0, ctypes.byref(n), 1) == xy.XY_EINVAL
    assert lib.xy_pcc_step(None, None, 1) == xy.XY_EINVAL
    assert lib.xy_destroy(None) == xy.XY_EINVAL
