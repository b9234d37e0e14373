"""The BF16 training pass's launch shape (srn_get_tuning / srn_set_tuning /
srn_autotune): every tile shape the library accepts gives the oracle's losses and
gradients, the autotuner installs one of its candidates without touching the
parameters or the Adam state, and a new tuning is picked up by the training step's
CUDA graphs."""
import numpy as np
import pytest

from paper_2308_02494_gb300 import synth
from gpu_util import RND, TOL, dG_error, density_grad_scale, ensure_built, make_model, morton_sorted, \
    points_off_faces, points_off_kinks, rel_l2
from test_gpu_parity import SHAPES, _oracle_backward

pytestmark = pytest.mark.gpu

POINTS = (256, 512, 768, 1024)
LEVELS = (2, 3, 4, 6, 9)


@pytest.fixture(scope="module", autouse=True)
def _built():
    ensure_built()


def _dense(ref, n, seed, lo, hi):
    x = points_off_kinks(ref, points_off_faces(ref["G"], 2 * n + 64, seed, lo=lo, hi=hi), RND["bf16"])
    assert len(x) >= n
    return morton_sorted(x[:n])


def test_default_tuning_and_argument_checks():
    from paper_2308_02494_gb300 import srn as S
    m, _ = make_model(SHAPES["m8r16c2"], 1, "bf16", 1024, seed=70)
    assert m.tuning == {"tile_points": 1024, "tile_level": 9, "density_ctas": 2}
    for bad in ((64, 9, 2), (1056, 9, 2), (300, 9, 2), (512, -1, 2), (512, 10, 2), (512, 4, 0), (512, 4, 5)):
        with pytest.raises(S.SrnError) as ei:
            m.set_tuning(*bad)
        assert ei.value.status == S.SRN_ERR_INVALID_ARG, bad
    assert m.tuning["tile_points"] == 1024
    m.set_tuning(128, 0, 4)
    assert m.tuning == {"tile_points": 128, "tile_level": 0, "density_ctas": 4}
    f, _ = make_model(SHAPES["m8r16c2"], 1, "fp32", 1024, seed=70)
    import torch
    x = torch.zeros((8, 3), device="cuda")
    with pytest.raises(S.SrnError) as ei:
        f.autotune(x, torch.zeros(8, device="cuda"), [0, 8])
    assert ei.value.status == S.SRN_ERR_UNSUPPORTED


@pytest.mark.parametrize("tuning", [(128, 0, 1), (256, 2, 4), (512, 4, 3), (160, 9, 1), (1024, 1, 2)])
def test_every_tile_shape_matches_the_oracle(tuning):
    """Small tiles and low levels cut the same batch into many more, smaller tiles (at
    level 0 every Morton unit is its own block); each tuning keeps the oracle's results."""
    import torch
    n = 2500
    m, ref = make_model(SHAPES["m64r32c2"], 1, "bf16", 4096, seed=71)
    x = _dense(ref[0], n, 72, -0.3, 0.2)
    v = np.random.default_rng(73).uniform(-0.5, 1.5, n).astype(np.float32)
    m.set_tuning(*tuning)
    losses = m.backward(torch.as_tensor(x, device="cuda"), torch.as_tensor(v, device="cuda"),
                        [0, n], density=True).cpu().numpy()
    gr = m.get("grads")[0]
    o = _oracle_backward(ref[0], x, v, True, RND["bf16"])
    tol = TOL["bf16"]
    assert abs(losses[0, 0] - o["L_rec"]) <= tol * abs(o["L_rec"])
    assert abs(losses[0, 1] - o["L_den"]) <= tol * abs(o["L_den"]) + 1e-12
    for k, ok in (("F", "dF"), ("W1", "dW1"), ("W2", "dW2"), ("w3", "dw3")):
        assert rel_l2(gr[k], o[ok]) <= tol, (k, rel_l2(gr[k], o[ok]))
    assert dG_error(gr["G"], o["dG"], density_grad_scale(ref[0]["G"], x, o["h"])) <= tol


def test_small_tiles_over_uneven_bricks_of_the_sub_lane_layout():
    """M = 8 (several points per warp in every grid) over two uneven bricks."""
    import torch
    counts = [2000, 777]
    m, ref = make_model(SHAPES["m8r16c2"], 2, "bf16", 4096, seed=74)
    xs = [_dense(ref[b], counts[b], 75 + b, -0.4 + 0.1 * b, 0.3) for b in range(2)]
    vs = [np.random.default_rng(77 + b).uniform(-0.5, 1.5, counts[b]).astype(np.float32) for b in range(2)]
    off = m.offsets_of(counts)
    m.set_tuning(128, 2, 2)
    m.backward(torch.as_tensor(np.concatenate(xs), device="cuda"),
               torch.as_tensor(np.concatenate(vs), device="cuda"), off, density=False)
    grads = m.get("grads")
    for b in range(2):
        o = _oracle_backward(ref[b], xs[b], vs[b], False, RND["bf16"])
        for k, ok in (("F", "dF"), ("W1", "dW1"), ("W2", "dW2"), ("w3", "dw3")):
            assert rel_l2(grads[b][k], o[ok]) <= TOL["bf16"], (b, k)


def test_autotune_installs_a_candidate_and_changes_no_parameter():
    import torch
    counts = [3000, 1777]
    m, _ = make_model(SHAPES["m8r16c2"], 2, "bf16", 8192, seed=80)
    off = m.offsets_of(counts)
    xyz = m.sample_points(81, 0, off)
    vol_np, _ = synth.gaussian_volume(32, 16, seed=82)
    vol = torch.as_tensor(np.asarray(vol_np, dtype=np.float32), device="cuda")
    boxes = synth.brick_boxes(32, (2, 1, 1), ghost=1)
    tgt = m.sample_target(vol, boxes, xyz, off)
    m.set_tuning(1024, 9, 3)
    before = {k: t.clone() for k, t in (("p", m.params), ("m", m.adam_m), ("v", m.adam_v))}
    got = m.autotune(xyz, tgt, off, density=True, reps=2)
    torch.cuda.synchronize()
    assert m.tuning == got
    assert got["density_ctas"] == 3
    assert (got["tile_points"], got["tile_level"]) in [(p, lv) for p in POINTS for lv in LEVELS]
    for k, t in (("p", m.params), ("m", m.adam_m), ("v", m.adam_v)):
        assert torch.equal(t, before[k]), k
    # the gradient buffer holds the installed tuning's backward pass (up to the order of
    # the float atomics that flush each tile's node sums)
    g_tuned = m.grads.clone()
    m.backward(xyz, tgt, off, density=True)
    torch.cuda.synchronize()
    assert rel_l2(g_tuned.cpu().numpy(), m.grads.cpu().numpy()) <= 1e-5
    m.status()


def test_train_step_graphs_follow_a_new_tuning():
    """Steps on a stream are captured into a CUDA graph; after srn_set_tuning the next
    step re-captures, and its results equal an eager step's under the same tuning."""
    import torch
    off = [0, 900, 1400]   # uneven bricks
    vol_np, _ = synth.gaussian_volume(32, 16, seed=84)
    vol = torch.as_tensor(np.asarray(vol_np, dtype=np.float32), device="cuda")
    boxes = synth.brick_boxes(32, (2, 1, 1), ghost=1)

    def run(stream, tunings):
        m, _ = make_model(SHAPES["m8r16c2"], 2, "bf16", 2048, seed=85)
        xyz = torch.empty((1400, 3), device="cuda")
        tgt = torch.empty(1400, device="cuda")
        for t in tunings:
            m.set_tuning(*t)
            with torch.cuda.stream(stream):
                m.train_step(86, vol, boxes, off, True, xyz, tgt, stream=stream)
        torch.cuda.synchronize()
        m.status(stream)
        return m.params.clone(), m.losses.clone()

    seq = [(1024, 9, 2)] * 3 + [(128, 1, 1)] * 3   # eager, capture, replay; after each tuning
    p_graph, l_graph = run(torch.cuda.Stream(), seq)
    p_eager, l_eager = run(torch.cuda.default_stream(), seq)
    assert torch.isfinite(l_graph).all()
    assert rel_l2(l_graph.cpu().numpy(), l_eager.cpu().numpy()) <= 1e-5
    assert rel_l2(p_graph.cpu().numpy(), p_eager.cpu().numpy()) <= 1e-5
