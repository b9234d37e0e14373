"""The allocation-free sampler entry point, srn_sample_points_static.

It exists for callers that cannot allocate device memory at all (a plug-in inside a
host application that owns the GPU memory budget, or a real-time loop that must not
enter an allocator), so they cannot build a handle with a workspace.  Its scratch lives
in a static device array inside the library.  This file is named to be collected last:
if it fails, a run that stops at the first failure has already run every other test.
"""
import numpy as np
import pytest

from oracle import sampler as osp
from paper_2308_02494_gb300 import srn as S
from paper_2308_02494_gb300 import synth
from gpu_util import ensure_built, make_model

pytestmark = pytest.mark.gpu


def _as_set(a):
    return a[np.lexsort((a[:, 2], a[:, 1], a[:, 0]))]


def _morton(a):
    cell = np.minimum(((a.astype(np.float64) + 1) * 16).astype(int), 31)
    code = np.zeros(len(a), dtype=np.int64)
    for bit in range(5):
        for ax in range(3):
            code |= ((cell[:, ax] >> bit) & 1) << (3 * bit + ax)
    return code


def test_static_sampler_matches_the_workspace_sampler_on_two_calls_in_a_row():
    import torch
    ensure_built()
    counts = [50000, 0, 31337, 777]
    off = [0] + list(np.cumsum(counts))
    m, _ = make_model(synth.ModelShape(8, 16, 2, 64), 4, "fp32", off[-1], seed=3)
    stream = torch.cuda.current_stream().cuda_stream
    for seed, step in ((0xC0FFEE, 3), (0xC0FFEE, 4)):
        want = m.sample_points(seed=seed, step=step, offsets=off).cpu().numpy()
        got_t = torch.full((off[-1], 3), float("nan"), device="cuda")
        S.srn_sample_points_static(stream, seed, step, 4, off, got_t.data_ptr())
        got = got_t.cpu().numpy()
        for b in range(4):
            g, w = got[off[b]:off[b + 1]], want[off[b]:off[b + 1]]
            np.testing.assert_array_equal(_as_set(g), _as_set(w))   # same draws
            # and the draws are the published Philox4x32-10 ones of the oracle's sampler
            np.testing.assert_array_equal(_as_set(g), _as_set(osp.sample_points(seed, step, b, counts[b])))
            if len(g):
                assert np.all(np.diff(_morton(g)) >= 0)                # same bin order


def test_static_sampler_rejects_requests_beyond_its_array():
    ensure_built()
    with pytest.raises(S.SrnError) as e:
        S.srn_sample_points_static(0, 1, 0, 1, [0, S.SRN_STATIC_SAMPLER_MAX_POINTS + 1], 16)
    assert e.value.status == S.SRN_ERR_INVALID_ARG and "131072" in str(e.value)
    with pytest.raises(S.SrnError):
        S.srn_sample_points_static(0, 1, 0, S.SRN_STATIC_SAMPLER_MAX_BRICKS + 1, [0] * 10, 16)
