"""The measurement hook (srn_set_timing / srn_read_timing): each target brackets the
launches it names with CUDA events, and nothing else."""
import numpy as np
import pytest

from paper_2308_02494_gb300 import synth

from gpu_util import make_model

pytestmark = pytest.mark.gpu


def test_timing_targets():
    import torch
    from paper_2308_02494_gb300 import srn as S
    from paper_2308_02494_gb300.model import SRN

    shape = synth.ModelShape(8, 16, 2, 64)
    counts = np.array([3000, 1777])
    off = SRN.offsets_of(counts)
    m, _ = make_model(shape, 2, "bf16", int(counts.sum()), seed=5)
    xyz = torch.from_numpy(synth.uniform_points(int(counts.sum()), 3)).float().cuda()
    tgt = torch.rand(int(counts.sum()), device="cuda")
    for which in (S.SRN_TIME_QUERY, S.SRN_TIME_ENCODER, S.SRN_TIME_DECODER, S.SRN_TIME_SCATTER):
        S.srn_set_timing(m.handle, which)
        m.backward(xyz, tgt, off, density=True)
        m.backward(xyz, tgt, off, density=False)
        torch.cuda.synchronize()
        ms, n = S.srn_read_timing(m.handle)
        assert n == 2 and ms > 0.0, (which, ms, n)
    # one kernel of the training pass: a forward query launches none of them
    S.srn_set_timing(m.handle, S.SRN_TIME_SCATTER)
    m.forward(xyz, off)
    torch.cuda.synchronize()
    assert S.srn_read_timing(m.handle) == (0.0, 0)
    S.srn_set_timing(m.handle, S.SRN_TIME_OFF)
    m.backward(xyz, tgt, off)
    torch.cuda.synchronize()
    assert S.srn_read_timing(m.handle) == (0.0, 0)
    with pytest.raises(S.SrnError):
        S.srn_set_timing(m.handle, 5)
