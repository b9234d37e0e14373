"""Checkpoint and resume: a model saved after some training steps and loaded into a
fresh handle continues exactly as the original (same batches from the restored
sampler step; results equal up to the summation order of float atomics)."""
import numpy as np
import pytest

from paper_2308_02494_gb300 import synth

from gpu_util import make_model

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_checkpoint_resumes_the_run(tmp_path, precision):
    import torch
    from paper_2308_02494_gb300 import srn as S
    from paper_2308_02494_gb300.model import SRN
    shape = synth.ModelShape(8, 16, 2, 64)
    counts = [700, 300]
    off = SRN.offsets_of(counts)
    vol_np, _ = synth.gaussian_volume(32, 16, seed=2)
    vol = torch.as_tensor(np.asarray(vol_np, dtype=np.float32), device="cuda")
    boxes = synth.brick_boxes(32, (2, 1, 1), ghost=1)
    xyz = torch.empty((sum(counts), 3), dtype=torch.float32, device="cuda")
    tgt = torch.empty(sum(counts), dtype=torch.float32, device="cuda")

    def run(m, steps):
        for _ in range(steps):
            m.train_step(5, vol, boxes, off, True, xyz, tgt)
        torch.cuda.synchronize()
        return m.params.clone(), m.adam_v.clone(), m.losses.clone()

    m1, _ = make_model(shape, 2, precision, 1024, seed=40)
    run(m1, 4)
    path = str(tmp_path / "ckpt.npz")
    m1.save(path)
    p1, v1, l1 = run(m1, 3)

    m2, _ = make_model(shape, 2, precision, 1024, seed=41)   # other parameters: all overwritten
    m2.load(path)
    assert S.srn_save_state(m2.handle, torch.cuda.current_stream().cuda_stream) == bytes(np.load(path)["state"])
    p2, v2, l2 = run(m2, 3)
    tol = 1e-5 if precision == "fp32" else 2e-3
    assert torch.linalg.norm(p2 - p1) <= tol * torch.linalg.norm(p1)
    assert torch.linalg.norm(v2 - v1) <= tol * torch.linalg.norm(v1)
    assert torch.allclose(l2, l1, rtol=tol, atol=0)


def test_checkpoint_of_another_shape_is_rejected(tmp_path):
    m1, _ = make_model(synth.ModelShape(8, 16, 2, 64), 2, "fp32", 256, seed=42)
    path = str(tmp_path / "a.npz")
    m1.save(path)
    m2, _ = make_model(synth.ModelShape(8, 16, 2, 64), 3, "fp32", 256, seed=43)
    with pytest.raises(ValueError):
        m2.load(path)
