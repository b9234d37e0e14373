"""Full-volume decode (srn_decode) against the oracle: every voxel of a small lattice
through the brick decomposition, batches small enough to split planes and rows."""
import numpy as np
import pytest

from oracle import apmgsrn as ap
from paper_2308_02494_gb300 import synth

from gpu_util import RND, TOL, make_model, rel_l2

pytestmark = pytest.mark.gpu


def _oracle_decode(models, grid, boxes, vox, rnd):
    i = np.arange(vox, dtype=np.float64)
    z, y, x = np.meshgrid(i, i, i, indexing="ij")
    p = np.stack([x.ravel(), y.ravel(), z.ravel()], axis=1) * 2.0 / (vox - 1) - 1.0
    b = ap.brick_index(p, grid)
    want = np.empty(len(p))
    keep = np.ones(len(p), dtype=bool)
    for k, prm in enumerate(models):
        sel = b == k
        loc = ap.global_to_brick_local(p[sel], boxes[k], vox)
        want[sel] = ap.query(prm, loc, rnd)
        # the inclusive mask of Eq. 2 is an FP-decided switch: drop voxels on a grid face
        u = ap.local_coords(prm["G"], loc)
        keep[np.nonzero(sel)[0]] = np.all(np.abs(np.abs(u) - 1.0) > 1e-5, axis=(1, 2))
    return want.reshape(vox, vox, vox), keep.reshape(vox, vox, vox)


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
@pytest.mark.parametrize("max_points", [4096, 90, 7])
def test_decode_matches_oracle(precision, max_points):
    import torch
    V, grid = 19, (2, 2, 2)
    boxes = synth.brick_boxes(V, grid, ghost=2)
    m, ref = make_model(synth.ModelShape(8, 6, 2, 64), 8, precision, max_points, seed=31, shrink=0.2)
    got = m.decode(grid, boxes, V).cpu().numpy()
    want, keep = _oracle_decode(ref, grid, boxes, V, RND[precision])
    assert keep.mean() > 0.9
    assert rel_l2(got[keep], want[keep]) <= TOL[precision], rel_l2(got[keep], want[keep])


def test_decode_rejects_a_grid_that_does_not_match_the_bricks():
    from paper_2308_02494_gb300 import srn as S
    m, _ = make_model(synth.ModelShape(8, 6, 2, 64), 8, "fp32", 64, seed=32)
    with pytest.raises(S.SrnError):
        m.decode((2, 2, 1), synth.brick_boxes(9, (2, 2, 1), ghost=1), 9)
