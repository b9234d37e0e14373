"""Pins of the oracle's mixed-precision backward (grad_rec with rnd=bf16).

The reading pinned here: the decoder's matrix products take bfloat16 operands with a
wide accumulator (the features y and ReLU(z1) in the forward pass; dL/dz2 and dL/dz1
in the backward pass, together with the y and ReLU(z1) factors of the weight
gradients), the ReLU masks are decided on the unrounded pre-activations, dL/dw3 is
formed from the unrounded dL/dm, and dL/dy is handed on to the adjoint of Eq. 2 as
bfloat16 (Sec. 4.1.2 decoder, Sec. 4.3.1 L_rec).

None of the expected values below comes from the oracle: the worked example is
evaluated with exact rationals and a round-to-nearest-even of its own, and the
representability checks read the float32 bit pattern directly.
"""
import math
from fractions import Fraction as Fr

import numpy as np

from oracle import apmgsrn as ap


def rne_bf16(v: Fr) -> Fr:
    """Nearest number with 8 significant bits (ties to even) of an exact rational."""
    if v == 0:
        return Fr(0)
    a = abs(v)
    e = math.floor(math.log2(a))
    while Fr(2) ** e > a:
        e -= 1
    while Fr(2) ** (e + 1) <= a:
        e += 1
    m = round(a / Fr(2) ** e * 128)   # Fraction.__round__ rounds halves to even
    return (1 if v > 0 else -1) * Fr(m, 128) * Fr(2) ** e


def representable(a) -> bool:
    """Every entry of a is a bfloat16 number (a float32 with 16 zero low bits)."""
    a = np.asarray(a, dtype=np.float64)
    f = a.astype(np.float32)
    return bool(np.all(f.astype(np.float64) == a) and np.all((f.view(np.uint32) & 0xFFFF) == 0))


def _one_node_case(v):
    """M = 1 grid of 2^3 nodes, C = 2, two hidden units, one point on node (0, 0, 0)
    under the identity transform: y is that node's pair of features exactly, and the
    whole of dL/dy lands on that node."""
    F = np.full((1, 2, 2, 2, 2), 0.3)
    F[0, 0, 0, 0] = (1.0, 0.5)
    params = {"F": F, "G": np.eye(3, 4)[None].copy(),
              "W1": np.array([[1.0, 1.0], [1.0, -0.5]]),
              "W2": np.array([[1.0, 0.0], [3.0, 1.25]]),
              "w3": np.array([1 + 2 ** -7, 1 - 2 ** -7]), "vmin": 0.0, "vmax": 1.0}
    return params, np.array([[-1.0, -1.0, -1.0]]), np.array([float(v)])


def _exact_chain(v: Fr, q):
    """The same case by hand in exact arithmetic, with q the operand rounding."""
    y = [Fr(1), Fr(1, 2)]
    W1 = [[Fr(1), Fr(1)], [Fr(1), Fr(-1, 2)]]
    W2 = [[Fr(1), Fr(0)], [Fr(3), Fr(5, 4)]]
    w3 = [1 + Fr(1, 128), 1 - Fr(1, 128)]
    yq = [q(a) for a in y]
    z1 = [W1[j][0] * yq[0] + W1[j][1] * yq[1] for j in range(2)]
    h1q = [q(max(Fr(0), a)) for a in z1]
    z2 = [W2[j][0] * h1q[0] + W2[j][1] * h1q[1] for j in range(2)]
    h2 = [max(Fr(0), a) for a in z2]
    r = w3[0] * h2[0] + w3[1] * h2[1] - v        # f - v with min = 0, max = 1
    dm = 2 * r                                    # dL/dm for one point
    out = {"r": r, "dw3": [dm * a for a in h2]}
    out["dz2_raw"] = [dm * w3[j] * (z2[j] > 0) for j in range(2)]
    dz2 = [q(a) for a in out["dz2_raw"]]
    out["dW2"] = [[dz2[j] * h1q[k] for k in range(2)] for j in range(2)]
    out["dz1_raw"] = [(W2[0][k] * dz2[0] + W2[1][k] * dz2[1]) * (z1[k] > 0) for k in range(2)]
    dz1 = [q(a) for a in out["dz1_raw"]]
    out["dW1"] = [[dz1[j] * yq[k] for k in range(2)] for j in range(2)]
    out["dy_raw"] = [W1[0][k] * dz1[0] + W1[1][k] * dz1[1] for k in range(2)]
    out["dy"] = [q(a) for a in out["dy_raw"]]
    return out


V = Fr(26753, 4096)   # chosen so that r = 1537/4096 and every rounding below is not a tie


def _check_against(o, want):
    np.testing.assert_array_equal(o["dw3"], [float(a) for a in want["dw3"]])
    np.testing.assert_array_equal(o["dW2"], [[float(a) for a in row] for row in want["dW2"]])
    np.testing.assert_array_equal(o["dW1"], [[float(a) for a in row] for row in want["dW1"]])
    np.testing.assert_array_equal(o["dy"][0], [float(a) for a in want["dy"]])
    dF = np.zeros((1, 2, 2, 2, 2))
    dF[0, 0, 0, 0] = [float(a) for a in want["dy"]]
    np.testing.assert_array_equal(o["dF"], dF)
    assert o["L_rec"] == float(want["r"] ** 2)


def test_worked_example_rounds_dz2_dz1_and_dy():
    want = _exact_chain(V, rne_bf16)
    # the example is sensitive: each of dz2, dz1 and dy changes when rounded
    for k in ("dz2", "dz1", "dy"):
        raw = want[k + "_raw"]
        rounded = [rne_bf16(a) for a in raw]
        assert all(a != b for a, b in zip(raw, rounded)), k
    assert [str(a) for a in want["dW2"][0]] == ["291/256", "291/512"]        # dz2_0 -> 97/128
    assert [str(a) for a in want["dW1"][0]] == ["3", "3/2"]                 # dz1_0 = 767/256 -> 3
    assert [str(a) for a in want["dy"]] == ["63/16", "81/32"]               # 1007/256, 1297/512 rounded
    params, x, v = _one_node_case(V)
    _check_against(ap.grad_rec(params, x, v, rnd=ap.bf16), want)


def test_worked_example_without_rounding_is_the_exact_chain():
    want = _exact_chain(V, lambda a: a)
    params, x, v = _one_node_case(V)
    _check_against(ap.grad_rec(params, x, v), want)


def test_small_perturbation_moves_only_the_unrounded_outputs():
    # dL/dm moves by 2^-19: the rounded dz2, dz1 and dy keep their values (each lies
    # far from a rounding boundary), so dW2, dW1 and dF must not move, while dw3 (formed
    # from the unrounded dL/dm) and the exact branch's dW2 must.
    params, x, v = _one_node_case(V)
    a = ap.grad_rec(params, x, v, rnd=ap.bf16)
    b = ap.grad_rec(params, x, v - 2.0 ** -20, rnd=ap.bf16)
    for k in ("dW2", "dW1", "dF", "dy"):
        np.testing.assert_array_equal(a[k], b[k])
    assert np.all(a["dw3"] != b["dw3"])
    e0, e1 = ap.grad_rec(params, x, v), ap.grad_rec(params, x, v - 2.0 ** -20)
    assert np.all(e0["dW2"] != e1["dW2"]) and np.all(e0["dy"] != e1["dy"])


def test_rounding_is_a_no_op_when_every_operand_is_representable():
    # Two grids of 3^3 nodes (C = 2) with quarter-step features, weights in {0, +-1/2,
    # +-1}, points on the nodes of grid 0 (grid 1 is half as large: its weights are 1/2),
    # targets on a 1/64 grid: every operand of every product is a bfloat16 number, so
    # the rounded backward must equal the exact one bit for bit.
    r = np.random.default_rng(2)   # a draw whose operands all have few enough bits
    M, R, C, H = 2, 3, 2, 4
    F = r.integers(-4, 5, size=(M, R, R, R, C)) / 4.0
    G = np.stack([np.eye(3, 4), 0.5 * np.eye(3, 4)])
    W1 = r.integers(-2, 3, size=(H, M * C)) / 2.0
    W2 = r.integers(-2, 3, size=(H, H)) / 2.0
    w3 = r.integers(-2, 3, size=H) / 2.0
    x = np.array([[-1.0, 0.0, 1.0], [0.0, 0.0, 0.0], [1.0, -1.0, 0.0], [0.0, 1.0, -1.0]])
    v = np.array([0.25, -0.5, 0.75, 0.125]) + r.integers(-8, 9, size=4) / 64.0
    params = {"F": F, "G": G, "W1": W1, "W2": W2, "w3": w3, "vmin": 0.0, "vmax": 1.0}
    ex = ap.grad_rec(params, x, v)
    y = ap.encode(F, G, x)
    _, c = ap.mlp_forward(W1, W2, w3, y)
    dm = 2.0 * (ex["f"] - v) / len(x)
    dz2 = dm[:, None] * w3[None, :] * (c["z2"] > 0)
    dz1 = (dz2 @ W2) * (c["z1"] > 0)
    for name, a in (("y", y), ("h1", c["h1"]), ("dz2", dz2), ("dz1", dz1), ("dy", ex["dy"])):
        assert representable(a), name
    assert np.count_nonzero(dz2) >= 4 and np.count_nonzero(dz1) >= 4
    rd = ap.grad_rec(params, x, v, rnd=ap.bf16)
    for k in ("f", "dF", "dW1", "dW2", "dw3", "dy"):
        np.testing.assert_array_equal(rd[k], ex[k])
