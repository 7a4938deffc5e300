"""The workspace-free labeling entry point (xy_label_bonds_static).

Some callers cannot allocate device memory -- a plugin that its host
application hands only input and output buffers, or a loop that must not
allocate once it runs -- so they cannot give a lattice handle its workspace.
xy_label_bonds_static serves them from a scratch array built into the
library.  This checks, through the C ABI, that two calls in a row (the second
on top of whatever the first left in the shared scratch) label exactly as the
workspace-based xy_label_bonds does, and that sizes beyond the built-in limit
are refused.  The file is named to be collected last.
"""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1210_6116_b300 as xy  # noqa: E402
from paper_1210_6116_b300 import build as xybuild  # noqa: E402

xybuild.build()


def _static_labels(L, right, down):
    r = torch.from_numpy(right).cuda()
    d = torch.from_numpy(down).cuda()
    out = torch.empty(L * L, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream()
    xy.xy_label_bonds_static(L, r.data_ptr(), d.data_ptr(), out.data_ptr(), stream.cuda_stream, 1)
    return out.cpu().numpy().view(np.uint32)


# L = 2: the periodic wrap makes a site its own right and down neighbour's
# neighbour twice; L <= 32: one tile column (the single-column tile geometry);
# 17 and 100: ragged tiles; 1024: the largest size the scratch holds.
@pytest.mark.parametrize("L", [2, 17, 32, 100, 1024])
def test_static_labels_match_workspace_labels_twice(L):
    lat = xy.Lattice(L, 1.0, 1, tile_y=32)
    for call, density in enumerate((0.55, 0.45)):
        right, down = synth.bond_masks(L, L, density, seed=7000 + 10 * L + call)
        want = lat.label_bonds(right, down)
        got = _static_labels(L, right, down)
        np.testing.assert_array_equal(got, want)


def test_static_bond_bytes_above_one_are_active():
    """The static entry point takes any nonzero byte as an active bond; the
    workspace path takes 0 / 1 only, so it labels the 0 / 1 version."""
    L = 100
    lat = xy.Lattice(L, 1.0, 1, tile_y=32)
    right, down = synth.bond_masks(L, L, 0.5, seed=9100)
    want = lat.label_bonds(right, down)
    rng = np.random.default_rng(9101)
    big_r = right * rng.choice(np.array([1, 2, 255], np.uint8), size=right.size)
    big_d = down * rng.choice(np.array([1, 2, 255], np.uint8), size=down.size)
    assert (big_r > 1).any() and (big_d > 1).any()
    np.testing.assert_array_equal(_static_labels(L, big_r, big_d), want)


def test_static_async_on_a_side_stream():
    """sync = 0 on a stream of its own: the call only enqueues; after the
    caller synchronises that stream the labels are complete."""
    L = 256
    lat = xy.Lattice(L, 1.0, 1, tile_y=32)
    right, down = synth.bond_masks(L, L, 0.5, seed=9200)
    want = lat.label_bonds(right, down)
    r = torch.from_numpy(right).cuda()
    d = torch.from_numpy(down).cuda()
    out = torch.full((L * L,), -1, dtype=torch.int32, device="cuda")
    torch.cuda.synchronize()
    side = torch.cuda.Stream()
    xy.xy_label_bonds_static(L, r.data_ptr(), d.data_ptr(), out.data_ptr(), side.cuda_stream, 0)
    side.synchronize()
    np.testing.assert_array_equal(out.cpu().numpy().view(np.uint32), want)


def test_static_labels_reject_sizes_beyond_the_scratch():
    L = xy.XY_STATIC_MAX_L + 1
    buf = torch.zeros(16, dtype=torch.uint8, device="cuda")
    with pytest.raises(xy.XyError) as e:
        xy.xy_label_bonds_static(L, buf.data_ptr(), buf.data_ptr(), buf.data_ptr(),
                                 torch.cuda.current_stream().cuda_stream, 1)
    assert e.value.status == xy.XY_EINVAL
    assert "scratch" in xy.xy_last_error()
