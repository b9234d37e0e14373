"""Pins of the oracle's decoder (Sec. 4.1.2), L_rec (Sec. 4.3.1) and Adam (Sec. 6)."""
import numpy as np

from oracle import apmgsrn as ap


def test_mlp_matches_explicit_loops():
    # Plain scalar loops over the definition: two bias-free ReLU layers, linear output.
    r = np.random.default_rng(0)
    N, K, H = 4, 6, 5
    y = r.normal(size=(N, K))
    W1, W2, w3 = r.normal(size=(H, K)), r.normal(size=(H, H)), r.normal(size=H)
    m, _ = ap.mlp_forward(W1, W2, w3, y)
    for n in range(N):
        h1 = [max(0.0, sum(W1[j, k] * y[n, k] for k in range(K))) for j in range(H)]
        h2 = [max(0.0, sum(W2[j, k] * h1[k] for k in range(H))) for j in range(H)]
        ref = sum(w3[j] * h2[j] for j in range(H))
        assert abs(m[n] - ref) < 1e-12


def test_mlp_selection_weights_and_relu_cut():
    # One-hot rows of W1 pick features; W2 = I passes them on; w3 = 1 sums them.
    K, H = 8, 8
    W1 = np.eye(H, K)
    W2 = np.eye(H)
    w3 = np.ones(H)
    y = np.array([[1.0, -2.0, 3.0, -4.0, 0.5, 0.0, -0.1, 2.0]])
    m, c = ap.mlp_forward(W1, W2, w3, y)
    assert m[0] == 1.0 + 3.0 + 0.5 + 2.0          # negatives cut by ReLU
    assert np.all(c["h1"][0][y[0] < 0] == 0.0)
    # no activation after the last layer: the output can be negative
    m2, _ = ap.mlp_forward(W1, W2, -w3, y)
    assert m2[0] == -(1.0 + 3.0 + 0.5 + 2.0)


def test_output_scaling():
    m = np.array([0.0, 0.25, 1.0, 1.7])
    np.testing.assert_array_equal(ap.scale_output(m, 0.0, 1.0), m)
    np.testing.assert_allclose(ap.scale_output(m, -2.0, 6.0), m * 8.0 - 2.0)


def test_loss_rec_closed_form():
    f = np.array([1.0, 2.0, 3.0, 4.0])
    v = np.array([1.0, 0.0, 3.0, 8.0])
    assert ap.loss_rec(f, v) == (0 + 4 + 0 + 16) / 4


def test_adam_first_step_closed_form():
    # From zero state, m_hat = g and v_hat = g^2, so the step is -lr g / (|g| + eps).
    g = np.array([1e-3, -2.0, 0.5, 0.0])
    p = np.zeros(4)
    p1, m1, v1 = ap.adam_update(p, g, np.zeros(4), np.zeros(4), 1, lr=0.01)
    np.testing.assert_allclose(p1, -0.01 * g / (np.abs(g) + 1e-8), rtol=1e-12, atol=0)
    np.testing.assert_allclose(m1, 0.1 * g)
    np.testing.assert_allclose(v1, 0.01 * g * g)


def test_adam_constant_gradient_keeps_unit_steps():
    # With a constant gradient, bias correction makes every step -lr g/(|g| + eps).
    g = np.array([0.3, -4.0])
    p, m, v = np.zeros(2), np.zeros(2), np.zeros(2)
    for t in range(1, 30):
        p_new, m, v = ap.adam_update(p, g, m, v, t, lr=1e-3)
        np.testing.assert_allclose(p_new - p, -1e-3 * g / (np.abs(g) + 1e-8), rtol=1e-9)
        p = p_new


def test_bf16_rounding_closed_form():
    # bfloat16 keeps 8 significant bits; halfway cases go to the even neighbour.
    from oracle.apmgsrn import bf16
    vals = np.array([1.0, 1 + 2 ** -8, 1 + 3 * 2 ** -8, 1 + 2 ** -7, -2.5, 3.14159265, 0.0,
                     1 + 2 ** -8 + 2 ** -20, 255.5])
    want = np.array([1.0, 1.0, 1 + 2 ** -6, 1 + 2 ** -7, -2.5, 3.140625, 0.0,
                     1 + 2 ** -7, 256.0])
    np.testing.assert_array_equal(bf16(vals), want)
    tiny = bf16(np.array([1e-30]))[0]
    assert tiny != 0.0 and abs(tiny - 1e-30) <= 2 ** -8 * 1e-30


def test_bf16_operand_rounding_only_touches_activations():
    # With operands already representable in bfloat16 the rounded decoder is the exact one.
    from oracle.apmgsrn import bf16
    r = np.random.default_rng(3)
    y = bf16(r.normal(size=(5, 8)))
    W1, W2, w3 = r.normal(size=(4, 8)), np.eye(4), r.normal(size=4)
    W1 = bf16(W1)
    m_exact, c = ap.mlp_forward(W1, W2, w3, y)
    m_rnd, _ = ap.mlp_forward(W1, W2, w3, y, rnd=bf16)
    # h1 is rounded in the second product: equal iff h1 is representable
    same = np.all(bf16(c["h1"]) == c["h1"], axis=1)
    np.testing.assert_array_equal(m_rnd[same], m_exact[same])
    assert not np.allclose(m_rnd, m_exact, rtol=1e-12, atol=0) or np.all(same)
