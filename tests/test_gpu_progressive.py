"""GPU parity of progressive rendering (Sec. 6): the image-hierarchy order of the
pixels each pass evaluates, the in-progress preview, and the finished frame."""
import numpy as np
import pytest

from oracle import render as orr
from paper_2308_02494_gb300 import synth
from gpu_util import TOL, ensure_built, make_model, rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    ensure_built()


def _scene(precision, n_bricks, max_points=2048):
    shape = synth.ModelShape(8, 6, 2, 64)
    m, ref = make_model(shape, n_bricks, precision, max_points, seed=61, shrink=0.2)
    if n_bricks == 1:
        grid, V, boxes = (1, 1, 1), 64, [[0, 0, 0, 63, 63, 63]]
    else:
        grid, V = (2, 2, 2), 65
        boxes = synth.brick_boxes(V, grid, ghost=2)
    lut = synth.random_lut(5, max_opacity=0.01)
    cam = synth.orbit_camera(1.1, 0.35, ortho=False)
    return m, ref, grid, V, boxes, lut, cam


@pytest.mark.parametrize("precision,n_bricks", [("fp32", 8), ("bf16", 1)])
def test_passes_follow_the_hierarchy_order_and_finish_the_frame(precision, n_bricks):
    import torch
    m, ref, grid, V, boxes, lut, cam = _scene(precision, n_bricks)
    W, H, S = 23, 17, 24
    lut_d = torch.as_tensor(lut, device="cuda")
    order = orr.hierarchy_order(W, H)
    rgba = torch.full((H, W, 4), float("nan"), device="cuda")
    preview = torch.empty_like(rgba)
    done = 0
    for count in (1, 5, 37, 100, W * H - 143):
        m.render_progressive(cam, lut_d, -0.5, 1.5, W, H, S, grid, boxes, V, done, count, rgba, preview)
        done += count
        img = rgba.cpu().numpy()
        written = ~np.isnan(img.reshape(-1, 4)).any(axis=1)
        assert set(np.flatnonzero(written)) == set(order[:done]), done
        want = orr.progressive_preview(np.nan_to_num(img, nan=0.0), done)
        np.testing.assert_allclose(preview.cpu().numpy(), want, rtol=0, atol=2e-6)
    full = m.render(cam, lut_d, -0.5, 1.5, W, H, S, grid, boxes, V).cpu().numpy()
    # the same per-pixel computation in another order and batching
    np.testing.assert_allclose(rgba.cpu().numpy(), full, rtol=0, atol=1e-6)
    want = orr.render(ref, boxes, grid, V, cam, lut, -0.5, 1.5, W, H, S)
    assert rel_l2(full, want) <= TOL[precision] * 5, rel_l2(full, want)


def test_preview_of_nothing_is_zero_and_bad_ranges_are_rejected():
    import torch
    from paper_2308_02494_gb300.srn import SrnError
    m, ref, grid, V, boxes, lut, cam = _scene("fp32", 1)
    W, H, S = 9, 6, 8
    lut_d = torch.as_tensor(lut, device="cuda")
    rgba = torch.zeros((H, W, 4), device="cuda")
    preview = torch.full_like(rgba, 3.0)
    m.render_progressive(cam, lut_d, -0.5, 1.5, W, H, S, grid, boxes, V, 0, 0, rgba, preview)
    assert torch.all(preview == 0)
    for first, count in ((0, W * H + 1), (-1, 2), (W * H, 1), (3, -1)):
        with pytest.raises(SrnError):
            m.render_progressive(cam, lut_d, -0.5, 1.5, W, H, S, grid, boxes, V, first, count, rgba, preview)
    with pytest.raises(SrnError):
        m.render_progressive(cam, lut_d, -0.5, 1.5, W, H, S, grid, boxes, V, 0, 4, rgba, rgba)
