"""GPU parity at the benchmark's sizes.

* One paper-scale model (M=64 grids of 32^3 x 2, MLP 128-64-64-1) trained on a
  2^18-point batch: the full backward (losses, every gradient) against the oracle,
  in FP32 and BF16.  The batch is the oracle sampler's Philox batch in the library
  sampler's Morton order, so the kernel runs its per-tile box path as in training.
* The 8-brick domain decomposition with uneven per-brick batches (the benchmark's
  launch configuration): forward values at 2000 sampled points per run, computed
  one by one by the oracle.
"""
import numpy as np
import pytest

from oracle import apmgsrn as ap
from oracle import sampler as osp
from paper_2308_02494_gb300 import synth
from gpu_util import (RND, TOL, dG_error, density_grad_scale, ensure_built, make_model,
                      morton_sorted, points_off_kinks, rel_l2)

pytestmark = pytest.mark.gpu

SHAPE = synth.ModelShape(64, 32, 2, 64)


@pytest.fixture(scope="module", autouse=True)
def _built():
    ensure_built()


def _batch(ref, n, seed, rnd):
    x = osp.sample_points(seed, 3, 0, n + n // 2)
    u = ap.local_coords(ref["G"], x.astype(np.float64))
    x = x[np.all(np.abs(np.abs(u) - 1.0) > 1e-5, axis=(1, 2))]
    x = points_off_kinks(ref, x, rnd)[:n]
    assert len(x) == n
    return morton_sorted(x)


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_paper_scale_backward_at_full_batch(precision):
    import torch
    n = 1 << 18
    m, refs = make_model(SHAPE, 1, precision, n, seed=31, shrink=0.3)
    ref = refs[0]
    x = _batch(ref, n, 77, RND[precision])
    v = np.random.default_rng(5).uniform(-0.5, 1.5, n).astype(np.float32)
    losses = m.backward(torch.as_tensor(x, device="cuda"), torch.as_tensor(v, device="cuda"),
                        [0, n], density=True).cpu().numpy()
    g = m.get("grads")[0]
    o = ap.grad_rec(ref, x.astype(np.float64), v.astype(np.float64), rnd=RND[precision])
    d = ap.grad_density(ref["G"], x.astype(np.float64), o["h"])
    tol = TOL[precision]
    assert abs(losses[0, 0] - o["L_rec"]) <= tol * o["L_rec"]
    assert abs(losses[0, 1] - d["L_den"]) <= tol * abs(d["L_den"])
    errs = {k: rel_l2(g[k], ref_g) for k, ref_g in (("F", o["dF"]), ("W1", o["dW1"]), ("W2", o["dW2"]),
                                                   ("w3", o["dw3"]))}
    errs["G"] = dG_error(g["G"], d["dG"], density_grad_scale(ref["G"], x, o["h"]))
    assert all(e <= tol for e in errs.values()), errs


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_eight_brick_forward_sampled(precision):
    import torch
    counts = synth.uneven_counts(8, 1 << 16, 1 << 19, seed=1)
    m, refs = make_model(SHAPE, 8, precision, int(counts.sum()), seed=41, shrink=0.3)
    off = m.offsets_of(counts)
    xs = [morton_sorted(osp.sample_points(9, 0, b, int(c))) for b, c in enumerate(counts)]
    f = m.forward(torch.as_tensor(np.concatenate(xs), device="cuda"), off).cpu().numpy()
    r = np.random.default_rng(3)
    for b in range(8):
        pick = r.choice(int(counts[b]), size=250, replace=False)
        xb = xs[b][pick].astype(np.float64)
        u = ap.local_coords(refs[b]["G"], xb)
        keep = np.all(np.abs(np.abs(u) - 1.0) > 1e-5, axis=(1, 2))
        want = ap.query(refs[b], xb[keep], rnd=RND[precision])
        got = f[off[b]:off[b + 1]][pick][keep]
        # forward values are continuous in the operand rounding, so no kink filter is needed
        assert rel_l2(got, want) <= TOL[precision], (b, rel_l2(got, want))


def test_eight_brick_training_pass_gradients():
    """The benchmark's BF16 training pass as it runs there (8 uneven bricks, 2 653 469
    points, the density passes on the second stream beside the scatter): losses and every
    gradient of the two smallest bricks (81 524 and 131 669 points) against the oracle.
    Those bricks' points are kept off grid faces and ReLU kinks; the other bricks'
    points are the sampler's as they come."""
    import torch
    counts = synth.uneven_counts(8, 1 << 16, 1 << 19, seed=1)
    check = [int(b) for b in np.argsort(counts)[:2]]
    m, refs = make_model(SHAPE, 8, "bf16", int(counts.sum()), seed=43, shrink=0.3)
    r = np.random.default_rng(17)
    xs, vs = [], []
    for b, c in enumerate(counts):
        c = int(c)
        if b in check:
            x = osp.sample_points(11, 0, b, c + c // 2)
            u = ap.local_coords(refs[b]["G"], x.astype(np.float64))
            x = points_off_kinks(refs[b], x[np.all(np.abs(np.abs(u) - 1.0) > 1e-5, axis=(1, 2))], RND["bf16"])
            assert len(x) >= c
            x = x[:c]
        else:
            x = osp.sample_points(11, 0, b, c)
        xs.append(morton_sorted(x))
        vs.append(r.uniform(-0.5, 1.5, c).astype(np.float32))
    off = m.offsets_of(counts)
    losses = m.backward(torch.as_tensor(np.concatenate(xs), device="cuda"),
                        torch.as_tensor(np.concatenate(vs), device="cuda"), off, density=True).cpu().numpy()
    grads = m.get("grads")
    tol = TOL["bf16"]
    for b in check:
        x = xs[b].astype(np.float64)
        o = ap.grad_rec(refs[b], x, vs[b].astype(np.float64), rnd=RND["bf16"])
        d = ap.grad_density(refs[b]["G"], x, o["h"])
        assert losses[b, 3] == counts[b]
        assert abs(losses[b, 0] - o["L_rec"]) <= tol * o["L_rec"], b
        assert abs(losses[b, 1] - d["L_den"]) <= tol * abs(d["L_den"]), b
        g = grads[b]
        errs = {k: rel_l2(g[k], want) for k, want in (("F", o["dF"]), ("W1", o["dW1"]), ("W2", o["dW2"]),
                                                      ("w3", o["dw3"]))}
        errs["G"] = dG_error(g["G"], d["dG"], density_grad_scale(refs[b]["G"], x, o["h"]))
        assert all(e <= tol for e in errs.values()), (b, errs)
