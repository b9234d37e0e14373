"""The tiled volume layout of the ground-truth lookup v(x) (Sec. 4.3.1): the copy that
srn_tile_volume writes follows the layout the header documents, the lookup that reads it
gives the same values bit for bit as the lookup of the x-fastest volume (and the
oracle's v(x) within float32 rounding), and a training step on it samples the same
batch and targets."""
import numpy as np
import pytest

from oracle import apmgsrn as ap
from paper_2308_02494_gb300 import synth
from gpu_util import ensure_built, make_model

pytestmark = pytest.mark.gpu

SHAPE_K16 = synth.ModelShape(8, 16, 2, 64)    # M = 8 grids of 16^3 x 2: K = 16
SHAPE_K32 = synth.ModelShape(16, 16, 2, 64)   # K = 32


@pytest.fixture(scope="module", autouse=True)
def _built():
    ensure_built()


def _torch():
    import torch
    return torch


def _volume(shape_zyx, seed):
    return np.random.default_rng(seed).normal(size=shape_zyx).astype(np.float32)


def _layout(vol):
    """The documented tiled layout, written out on the host: 4^3 tiles in x-fastest tile
    order, x-fastest inside a tile, each extent padded with zeros to whole tiles."""
    vz, vy, vx = vol.shape
    tz, ty, tx = (vz + 3) // 4, (vy + 3) // 4, (vx + 3) // 4
    pad = np.zeros((tz * 4, ty * 4, tx * 4), dtype=np.float32)
    pad[:vz, :vy, :vx] = vol
    # [tz][4][ty][4][tx][4] -> [tz][ty][tx][4 z][4 y][4 x]
    return pad.reshape(tz, 4, ty, 4, tx, 4).transpose(0, 2, 4, 1, 3, 5).ravel()


def test_tiled_copy_follows_the_documented_layout():
    torch = _torch()
    from paper_2308_02494_gb300.model import TiledVolume
    for shape in [(9, 6, 13), (8, 8, 8), (2, 3, 2)]:
        vol = _volume(shape, 3)
        tv = TiledVolume(torch.as_tensor(vol, device="cuda"))
        got = tv.data.cpu().numpy()
        want = _layout(vol)
        assert got.shape == want.shape, shape
        np.testing.assert_array_equal(got, want)


def test_tiled_lookup_equals_linear_lookup_and_the_oracle():
    torch = _torch()
    from paper_2308_02494_gb300.model import TiledVolume
    vol = _volume((37, 22, 45), 11)              # [z][y][x]: no extent a multiple of 4
    boxes = np.array([[0, 0, 0, 23, 12, 19], [21, 9, 17, 44, 21, 36], [3, 1, 2, 5, 4, 3],
                      [0, 0, 0, 44, 21, 36], [40, 18, 33, 44, 21, 36], [7, 7, 7, 8, 8, 8],
                      [10, 0, 20, 30, 21, 36], [0, 10, 0, 44, 20, 35]], dtype=np.int64)
    counts = [150, 7, 0, 300, 41, 5, 64, 65]
    m, _ = make_model(SHAPE_K16, 8, "fp32", 1024, seed=31)
    r = np.random.default_rng(12)
    xs = [r.uniform(-1, 1, size=(c, 3)).astype(np.float32) for c in counts]
    # the faces and corners of the boxes: the last cell of an axis and its upper node
    xs[0][:6] = [[-1, -1, -1], [1, 1, 1], [1, -1, 0.5], [0, 0, 0], [-1, 1, -1], [1, 1, -1]]
    xs[3][:2] = [[1, 1, 1], [-1, -1, -1]]
    off = m.offsets_of(counts)
    xyz = torch.as_tensor(np.concatenate(xs), device="cuda")
    vd = torch.as_tensor(vol, device="cuda")
    tv = TiledVolume(vd)
    lin = m.sample_target(vd, boxes, xyz, off).cpu().numpy()
    til = m.sample_target(tv, boxes, xyz, off).cpu().numpy()
    np.testing.assert_array_equal(til, lin)
    for b in range(8):
        if counts[b]:
            want = ap.volume_sample(vol, xs[b].astype(np.float64), boxes[b])
            assert np.max(np.abs(til[off[b]:off[b + 1]] - want)) <= 1e-5 * np.max(np.abs(vol)), b


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_train_step_on_the_tiled_volume_samples_the_same_targets(precision):
    torch = _torch()
    from paper_2308_02494_gb300.model import TiledVolume
    shape = SHAPE_K32 if precision == "bf16" else SHAPE_K16
    V = 41
    vol = _volume((V, V, V), 5)
    boxes = synth.brick_boxes(V, (2, 2, 2), ghost=2)
    counts = [1024, 512, 2048, 256, 1024, 768, 128, 1536]
    outs = []
    for tiled in (False, True):
        m, _ = make_model(shape, 8, precision, sum(counts), seed=32)
        off = m.offsets_of(counts)
        xyz = torch.empty((sum(counts), 3), dtype=torch.float32, device="cuda")
        tgt = torch.empty(sum(counts), dtype=torch.float32, device="cuda")
        vd = torch.as_tensor(vol, device="cuda")
        src = TiledVolume(vd) if tiled else vd
        losses = m.train_step(9, src, boxes, off, True, xyz, tgt)
        torch.cuda.synchronize()
        outs.append((xyz.cpu().numpy(), tgt.cpu().numpy(), losses.cpu().numpy().copy()))
    # the sampler's counting sort orders the points of one bin as its atomics come, so
    # compare each brick's (point, target) pairs as sets
    off = np.concatenate([[0], np.cumsum(counts)])
    for b in range(8):
        pairs = []
        for xyz, tgt, _ in outs:
            rows = np.concatenate([xyz[off[b]:off[b + 1]], tgt[off[b]:off[b + 1], None]], axis=1)
            pairs.append(rows[np.lexsort(rows[:, 2::-1].T)])
        np.testing.assert_array_equal(pairs[1], pairs[0])
    # the losses come from the same batch and targets (their sums may add in another order)
    np.testing.assert_allclose(outs[1][2], outs[0][2], rtol=1e-6, atol=1e-12)
