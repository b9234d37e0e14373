"""Failure detection through the device status word, with the failure made on the host:
a NaN target makes one brick's losses non-finite; srn_get_status reports
SRN_ERR_NONFINITE once, clears it, and a clean pass afterwards reports OK."""
import numpy as np
import pytest

from paper_2308_02494_gb300 import synth
from gpu_util import ensure_built, make_model
from test_gpu_parity import SHAPES

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    ensure_built()


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_nonfinite_loss_is_reported_once_and_cleared(precision):
    import torch
    from paper_2308_02494_gb300 import srn as S
    counts = [700, 300]
    m, _ = make_model(SHAPES["m8r16c2"], 2, precision, 2048, seed=90)
    off = m.offsets_of(counts)
    xyz = torch.as_tensor(synth.uniform_points(1000, 91), device="cuda").float()
    tgt = torch.rand(1000, device="cuda")
    m.status()                                   # nothing recorded yet
    tgt[5] = float("nan")                        # a point of brick 0
    losses = m.backward(xyz, tgt, off, density=True).cpu().numpy()
    assert np.isnan(losses[0, 0]) and np.isfinite(losses[1, 0])
    with pytest.raises(S.SrnError) as ei:
        m.status()
    assert ei.value.status == S.SRN_ERR_NONFINITE
    m.status()                                   # reported once, then cleared
    tgt[5] = 0.5
    losses = m.backward(xyz, tgt, off, density=True).cpu().numpy()
    assert np.all(np.isfinite(losses))
    m.status()
