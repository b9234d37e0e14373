"""The device-side training routine (SRN_SCHEDULE) against its plain restatement
(tests/schedule_ref.py), step by step on a real training run, and its effect on the
parameters: a finished brick is no longer updated, G only moves while density is on."""
import numpy as np
import pytest

from paper_2308_02494_gb300 import synth
from schedule_ref import BrickRoutine

pytestmark = pytest.mark.gpu

ROUTINE = dict(delay=3, window=4, rel=1e-4, frac=0.8, total=60, pwin=2, prel=1e-4, pfactor=0.5, pmax=3)


def _model(precision):
    import torch
    from paper_2308_02494_gb300.model import SRN
    shape = synth.ModelShape(8, 16, 2, 64)
    # a tiny feature learning rate: L_rec stays noisy, so plateaus come quickly
    m = SRN(shape, n_bricks=2, precision=precision, max_points=1024, lr_feat=1e-6)
    m.set_params([synth.parity_model(shape, 60 + b) for b in range(2)])
    torch.cuda.synchronize()
    return m


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_device_routine_follows_the_plain_one(precision):
    import torch
    from paper_2308_02494_gb300.model import SRN
    m = _model(precision)
    r = ROUTINE
    m.set_schedule(delay_iters=r["delay"], density_window=r["window"], density_rel=r["rel"],
                   density_frac=r["frac"], total_iters=r["total"], plateau_window=r["pwin"],
                   plateau_rel=r["prel"], plateau_factor=r["pfactor"], plateau_max=r["pmax"])
    refs = [BrickRoutine(**r) for _ in range(2)]
    counts = [600, 400]
    off = SRN.offsets_of(counts)
    vol_np, _ = synth.gaussian_volume(32, 16, seed=3)
    vol = torch.as_tensor(np.asarray(vol_np, dtype=np.float32), device="cuda")
    boxes = synth.brick_boxes(32, (2, 1, 1), ghost=1)
    xyz = torch.empty((sum(counts), 3), dtype=torch.float32, device="cuda")
    tgt = torch.empty(sum(counts), dtype=torch.float32, device="cuda")
    seen = {"plateau": 0, "finished": 0, "stopped": 0, "density": 0}
    for step in range(r["total"]):
        dec = m.read_schedule()                       # the decisions for this iteration
        before = [{k: v.clone() for k, v in m._views(m.params, b).items()} for b in range(2)]
        m.train_step(7, vol, boxes, off, True, xyz, tgt, schedule=True)
        torch.cuda.synchronize()
        losses = m.losses.cpu().numpy()
        for b in range(2):
            after = m._views(m.params, b)
            moved = {k: not torch.equal(before[b][k], after[k]) for k in after}
            if dec[b]["finished"]:
                assert not any(moved.values()), (step, b)
            else:
                assert moved["F"], (step, b)
            assert moved["G"] == bool(dec[b]["density_on"] and not dec[b]["finished"]), (step, b)
            if not dec[b]["density_on"]:
                assert losses[b, 1] == 0.0
            refs[b].update(float(losses[b, 0]), float(losses[b, 1]))
        st = m.read_schedule()
        for b in range(2):
            ref, got = refs[b], st[b]
            assert got["iteration"] == ref.it
            assert got["plateaus"] == ref.plateaus, (step, b)
            assert bool(got["finished"]) == ref.finished, (step, b)
            assert bool(got["density_on"]) == ref.den_on, (step, b)
            assert bool(got["density_stopped"]) == ref.den_stopped, (step, b)
            assert got["density_iters"] == len(ref.den_hist), (step, b)
            assert abs(got["lr_scale"] - ref.lr_scale) <= 1e-6
            seen["plateau"] += got["plateaus"] > 0
            seen["finished"] += bool(got["finished"])
            seen["stopped"] += bool(got["density_stopped"])
            seen["density"] += bool(got["density_on"])
    assert all(v > 0 for v in seen.values()), seen      # every transition happened


def test_schedule_flag_needs_a_routine():
    import torch
    from paper_2308_02494_gb300 import srn as S
    from paper_2308_02494_gb300.model import SRN
    m = _model("fp32")
    vol = torch.zeros((8, 8, 8), device="cuda")
    xyz = torch.empty((10, 3), device="cuda")
    tgt = torch.empty(10, device="cuda")
    with pytest.raises(S.SrnError):
        m.train_step(1, vol, synth.brick_boxes(8, (2, 1, 1), ghost=1), SRN.offsets_of([5, 5]), True, xyz, tgt,
                     schedule=True)
    with pytest.raises(S.SrnError):
        m.set_schedule(density_window=5000)


def test_finished_bricks_give_their_share_to_the_others():
    """After a brick finishes, srn_rebalance moves its share of the batch to the bricks
    still training; the next steps run on the new offsets (a new CUDA graph), the finished
    brick keeps its minimum share and stays frozen."""
    import torch
    from paper_2308_02494_gb300 import srn as S
    m = _model("bf16")
    r = ROUTINE
    m.set_schedule(delay_iters=r["delay"], density_window=r["window"], density_rel=r["rel"],
                   density_frac=r["frac"], total_iters=r["total"], plateau_window=r["pwin"],
                   plateau_rel=r["prel"], plateau_factor=r["pfactor"], plateau_max=r["pmax"])
    base = [600, 400]
    off = [0, 600, 1000]
    vol_np, _ = synth.gaussian_volume(32, 16, seed=3)
    vol = torch.as_tensor(np.asarray(vol_np, dtype=np.float32), device="cuda")
    boxes = synth.brick_boxes(32, (2, 1, 1), ghost=1)
    xyz = torch.empty((1000, 3), dtype=torch.float32, device="cuda")
    tgt = torch.empty(1000, dtype=torch.float32, device="cuda")
    stream = torch.cuda.Stream()
    state = m.read_schedule()
    for _ in range(r["total"]):
        with torch.cuda.stream(stream):
            m.train_step(7, vol, boxes, off, True, xyz, tgt, stream=stream, schedule=True)
        state = m.read_schedule(stream)
        if any(s["finished"] for s in state):
            break
    fin = [bool(s["finished"]) for s in state]
    assert any(fin)
    new = m.rebalanced_offsets(base, min_points=64, stream=stream)
    assert new == S.srn_rebalance(base, fin, 64) and new[-1] == 1000
    if not all(fin):
        for b in range(2):
            assert (new[b + 1] - new[b] == 64) if fin[b] else (new[b + 1] - new[b] > base[b])
    frozen = [{k: v.clone() for k, v in m._views(m.params, b).items()} for b in range(2)]
    for _ in range(3):   # eager, capture, replay of the new offsets' graph
        with torch.cuda.stream(stream):
            m.train_step(7, vol, boxes, new, True, xyz, tgt, stream=stream, schedule=True)
    stream.synchronize()
    m.status(stream)
    losses = m.losses.cpu().numpy()
    assert list(losses[:, 3]) == [new[1] - new[0], new[2] - new[1]]   # points per brick
    for b in range(2):
        after = m._views(m.params, b)
        moved = not torch.equal(frozen[b]["F"], after["F"])
        assert moved == (not fin[b]), b
